// Host runtime of libhp: contexts, the stream pool, the caching allocators,
// events with exactly-once completion callbacks, and the C ABI of hp.h.
//
// Execution model (arXiv:2004.04334 Sec. 2 and Sec. 4.1): an enqueue call
// is the non-blocking acquire(): it stages the inputs in pooled pinned
// memory, queues copies and kernels on one stream of the pool and a host
// function after them, and returns.  The host function (the holder of
// Sec. 2) runs when the device work is done, marks the event complete and
// fires the user's callback; produce() is hp_fetch_clusters on the pinned
// results.  No allocation, synchronisation or device assert happens on this
// path once the pools are warm (Sec. 4.1): every buffer comes from a
// caching pool whose cudaMalloc / cudaHostAlloc calls only happen while it
// grows.
//
// Also here: consumers of a product (hits, transfers) under the stream
// rules of Sec. 4.2, the device-resident entry and its CUDA-graph form, the
// autotuner of the clustering kernel's launch parameters, and the
// continuous-batching serving loop with its native load driver.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "hp.h"
#include "hp_internal.h"

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Bin sizes: four bins per power of two, 4 KiB minimum (at most 25% slack).
// Serving sizes vary from batch to batch and request to request: rounding
// them up to a power of two keeps the number of distinct pool bins small, and
// request staging may take any cached block up to kServeRatio times its
// size, and a batch any cached block at all (the smallest that fits; the
// blocks reserved at hp_serve_start, one of the largest batch per batch in
// flight, always leave one), so a steady stream reuses cached blocks instead
// of allocating: cudaMalloc synchronises the device and cudaHostAlloc takes
// milliseconds, and one such call on the admitter thread stalled every
// request behind it for tens of milliseconds.
constexpr size_t kServeRatio = 256;
constexpr size_t kAnyRatio = 0; // Pool::alloc: any cached block that fits
size_t round_pow2(size_t bytes)
{
    size_t p = 4096;
    while (p < bytes) p <<= 1;
    return p;
}

size_t round_bin(size_t bytes)
{
    if (bytes <= 4096) return 4096;
    int lg = 63 - __builtin_clzll((unsigned long long)bytes);
    size_t step = ((size_t)1 << lg) / 4;
    return (bytes + step - 1) / step * step;
}

struct Block {
    void *ptr = nullptr;  // host address (host pool) or device address
    void *dptr = nullptr; // device alias of the block
    size_t bytes = 0;
};

// Caching allocator for device or mapped pinned host memory.  Blocks return
// to a per-size free list and are reused by later requests of the same bin;
// the backend is only called when no cached block fits.  free() makes no
// CUDA call, so blocks can be returned from a CUDA host-function thread.
class Pool {
  public:
    explicit Pool(bool host) : host_(host) {}

    // max_ratio: the largest cached block (relative to the request) that may
    // serve it, 0 for any; a large ratio trades memory for fewer backend calls.
    hp_status alloc(size_t bytes, Block *out, size_t max_ratio = 2)
    {
        const size_t b = round_bin(bytes);
        {
            std::lock_guard<std::mutex> g(mu_);
            if (fail_next_ > 0) {
                --fail_next_;
                return HP_ENOMEM;
            }
            auto it = free_.lower_bound(b); // best fit among cached blocks of up to max_ratio times the size
            if (it != free_.end() && (max_ratio == 0 || it->first / max_ratio <= b)) {
                *out = it->second;
                free_.erase(it);
                ++hits_;
                return HP_OK;
            }
        }
        Block blk;
        if (!backend_alloc(b, &blk)) {
            trim();
            if (!backend_alloc(b, &blk)) return HP_ENOMEM;
        }
        std::lock_guard<std::mutex> g(mu_);
        ++backend_allocs_;
        total_ += b;
        *out = blk;
        return HP_OK;
    }

    void free(const Block &b)
    {
        if (!b.ptr) return;
        std::lock_guard<std::mutex> g(mu_);
        free_.emplace(b.bytes, b);
    }

    // Release every cached block (CUDA calls; never on the event path).
    void trim()
    {
        std::multimap<size_t, Block> f;
        {
            std::lock_guard<std::mutex> g(mu_);
            f.swap(free_);
            for (auto &kv : f) total_ -= kv.first;
        }
        for (auto &kv : f) {
            if (host_)
                cudaFreeHost(kv.second.ptr);
            else
                cudaFree(kv.second.ptr);
        }
    }

    void fail_next(uint32_t n)
    {
        std::lock_guard<std::mutex> g(mu_);
        fail_next_ = n;
    }
    uint64_t backend_allocs()
    {
        std::lock_guard<std::mutex> g(mu_);
        return backend_allocs_;
    }
    uint64_t hits()
    {
        std::lock_guard<std::mutex> g(mu_);
        return hits_;
    }
    uint64_t total_bytes()
    {
        std::lock_guard<std::mutex> g(mu_);
        return total_;
    }

  private:
    bool backend_alloc(size_t b, Block *blk)
    {
        void *p = nullptr;
        cudaError_t e = host_ ? cudaHostAlloc(&p, b, cudaHostAllocMapped | cudaHostAllocPortable) : cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        void *d = p;
        if (host_ && cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(p);
            return false;
        }
        blk->ptr = p;
        blk->dptr = d;
        blk->bytes = b;
        return true;
    }

    bool host_;
    std::mutex mu_;
    std::multimap<size_t, Block> free_;
    uint64_t backend_allocs_ = 0, hits_ = 0, total_ = 0;
    uint32_t fail_next_ = 0;
};

// Event state word: completion, callback and release bits, and in bits 8
// and up the number of consumers (hp_enqueue_hits) that still read the
// event's outputs.  Every change is one atomic read-modify-write of this
// word; the change that makes the event destroyable (complete, callback run,
// released, no consumer left) is the one that frees it, exactly once.
// Build identifier reported in the provenance of every product.
constexpr const char *kLibraryId = "libhp 1 (sm_103a)";

constexpr uint32_t kDone = 1u, kCbSet = 2u, kCbDone = 4u, kReleaseReq = 8u;
constexpr uint32_t kHold = 1u << 8;

bool destroyable(uint32_t s)
{
    return (s & kDone) && (s & kReleaseReq) && (!(s & kCbSet) || (s & kCbDone)) && (s >> 8) == 0;
}

struct Serve;
struct Batch;

} // namespace

struct hp_ctx {
    hp_config cfg{};
    int device = 0;
    int sm_count = 0;
    uint32_t max_tile[4] = {0, 0, 0, 0}; // largest tile per resident-blocks count (init_kernels)
    char device_name[256] = {0};
    int cc_major = 0, cc_minor = 0;
    // autotuner (hp_autotune): tuning per launch-shape bucket, optional cache file
    std::mutex tune_mu;
    std::map<std::pair<int, int>, hp::Tuning> tuned;
    int tune_mode = 1; // 0 off (defaults only), 1 use tuned buckets, 2 also search on first device call
    std::string tune_cache;
    int32_t *d_gain = nullptr, *d_ped = nullptr;
    std::vector<cudaStream_t> streams;
    std::atomic<uint32_t> next_stream{0};
    Pool dpool{false}, hpool{true};
    std::atomic<uint64_t> inflight{0}, dev_in_use{0};
    std::atomic<int> failed{0};
    std::atomic<uint64_t> enqueued{0}, completed{0}, h2d{0}, d2h{0}, kernels{0}, ws_mallocs{0};
    // clusters per digi of recent launches (x 65536): sizes the part of the
    // cluster outputs that goes to the host by DMA (see head_count)
    std::atomic<uint32_t> clus_ratio{6554};
    bool pageable_access = false; // the device reads pageable host memory (cudaDevAttrPageableMemoryAccess)
    std::mutex live_mu;
    std::set<hp_event *> live;
    std::mutex cev_mu;
    std::vector<cudaEvent_t> cev_free;
    std::mutex ws_mu;
    std::map<cudaStream_t, Block> stream_ws;
    // stage timers (hp_profile_enable / hp_profile_read)
    struct ProfRec {
        cudaEvent_t ev[hp::kNumKernels + 1];
    };
    std::mutex prof_mu;
    uint32_t prof_left = 0;
    std::vector<ProfRec> prof_used;
    std::vector<cudaEvent_t> prof_pool;
    // serving loop (hp_serve_start / hp_submit / hp_serve_stop)
    std::mutex serve_mu;
    Serve *serve = nullptr;
    std::atomic<uint64_t> serve_batches{0}, serve_requests{0};
    std::atomic<uint64_t> serve_submit_ns{0}, serve_launch_ns{0}, serve_complete_ns{0}, serve_max_batch{0};
    // serving trace (hp_serve_trace_enable / hp_serve_trace_read)
    std::mutex trace_mu;
    std::vector<hp_serve_trace_record> trace;
    std::vector<std::array<cudaEvent_t, 4>> trace_ev; // device marks of each record (or null)
    std::vector<cudaEvent_t> trace_spare;             // marks of batches past the cap, destroyed later
    uint64_t trace_cap = 0;
    // hits: module placement (every version stays until hp_destroy, so queued
    // work keeps the one it was queued with) and the consumer streams
    std::mutex geom_mu;
    std::vector<void *> placements;
    hp::Placement place{};
    bool has_place = false;
    std::mutex aux_mu;
    std::vector<cudaStream_t> aux_streams;
    std::atomic<uint32_t> next_aux{0};
    std::atomic<uint64_t> consumer_reuses{0}, consumer_waits{0};
    std::atomic<uint32_t> debug_withhold{0}; // hp_debug_expire_waits: launches left to withhold ticket 0
    // captured device passes (hp_graph_capture), destroyed with the context
    std::mutex graph_mu;
    std::set<hp_graph *> graphs;
};

struct hp_graph {
    hp_ctx *ctx = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *ws = nullptr;    // the graph's own scratch (its launches are serialised by CUDA)
    uint64_t kernels = 0;  // kernels per launch
};

struct hp_event {
    hp_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Block dev, host;
    size_t dev_charge = 0;
    uint32_t E = 0;
    uint64_t N = 0;
    uint32_t flags = 0;
    uint64_t tag = 0;
    uint64_t *h_coff = nullptr;
    int32_t *h_status = nullptr;
    uint32_t *h_module = nullptr;
    int32_t *h_id = nullptr, *h_charge = nullptr, *h_npix = nullptr, *h_label = nullptr;
    float *h_x = nullptr, *h_y = nullptr;
    uint16_t *h_label16 = nullptr; // compact labels (HP_LABELS_U16)
    uint32_t *h_ifirst = nullptr;
    std::atomic<uint32_t> state{0};
    hp_status status = HP_OK;
    hp_callback cb = nullptr;
    void *user = nullptr;
    uint64_t t_enq = 0, t_done = 0;
    // provenance (Sec. 3): which path made the product, with which clustering settings
    uint32_t path = 0;
    hp::Tuning tune_used{};
    // serving requests: the batch that carries the request and its index in it
    bool request = false;
    int32_t status_local = 0;
    Batch *batch = nullptr;
    uint32_t index = 0;
    Block staging;               // the request's inputs (pinned), until its batch completes
    const uint32_t *in_words = nullptr;  // inputs of the request: device alias of the staging, or the
    const uint16_t *in_mods = nullptr;   // caller's buffers (in_direct, HP_INPUT_NOCOPY)
    bool in_direct = false;
    uint64_t coff_local[2] = {0, 0};
    // Product<T> stream rule (Sec. 4.2): set by the first consumer, which takes this event's stream
    std::atomic<bool> stream_taken{false};
    // device-visible addresses of the outputs: aliases of the mapped host
    // arrays, or device memory (dout) with HP_KEEP_ON_DEVICE; label is set
    // only while the labels stay on the device
    hp::Outputs dv{};
    bool on_device = false;
    Block dout;
    size_t dout_charge = 0;
    // consumers: hits events and transfer events hold the consumed clusters
    // event until their own work has run
    bool hits = false;
    bool transfer = false;
    hp_event *product = nullptr;
    uint32_t *h_hmodule = nullptr;
    float *h_hx = nullptr, *h_hy = nullptr, *h_hz = nullptr;
};

namespace {

hp_status fail(hp_ctx *ctx)
{
    ctx->failed.store(1);
    return HP_ECUDA;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void release_batch_ref(Batch *b);

// Free the host side of a completed, released event (no CUDA call).
void destroy_event(hp_event *ev)
{
    hp_ctx *ctx = ev->ctx;
    if (ev->request) {
        ctx->hpool.free(ev->staging);
        if (ev->batch) release_batch_ref(ev->batch);
    } else {
        ctx->hpool.free(ev->host);
        if (ev->dout.ptr) {
            ctx->dpool.free(ev->dout);
            ctx->dev_in_use.fetch_sub(ev->dout_charge);
        }
        std::lock_guard<std::mutex> g(ctx->cev_mu);
        ctx->cev_free.push_back(ev->done);
    }
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        ctx->live.erase(ev);
    }
    delete ev;
}

// Set `bits` in the state word; free the event if that made it destroyable.
uint32_t set_state(hp_event *ev, uint32_t bits)
{
    const uint32_t prev = ev->state.fetch_or(bits, std::memory_order_acq_rel);
    if (!destroyable(prev) && destroyable(prev | bits)) destroy_event(ev);
    return prev;
}

// A consumer no longer reads the event's outputs.
void drop_hold(hp_event *ev)
{
    const uint32_t prev = ev->state.fetch_sub(kHold, std::memory_order_acq_rel);
    if (!destroyable(prev) && destroyable(prev - kHold)) destroy_event(ev);
}

// Completion of one event on the host-function thread: the exactly-once
// hand-off to the callback (Sec. 2 holder) and a deferred release.
void complete_event(hp_event *ev)
{
    const uint32_t prev = set_state(ev, kDone);
    if (prev & kCbSet) {
        ev->cb(ev->user, ev, ev->status);
        set_state(ev, kCbDone);
    }
}

// Destroy the serving trace's device marks (not from a host function).
void clear_trace_marks(hp_ctx *ctx)
{
    for (auto &a : ctx->trace_ev)
        for (cudaEvent_t e : a)
            if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->trace_spare) cudaEventDestroy(e);
    ctx->trace_ev.clear();
    ctx->trace_spare.clear();
    cudaGetLastError();
}

// Cluster outputs bound for mapped host memory: how many leading positions
// go through device columns and one DMA each (Outputs::head) instead of
// being stored over the host link by the copy kernel.  15/16 of the clusters
// expected from the recent clusters-per-digi ratio, at most a quarter of the
// digis, in whole copy chunks; the rest of a launch that has more clusters
// still goes straight to the host.
uint32_t head_count(const hp_ctx *ctx, uint64_t N)
{
    const uint64_t expect = (N * ctx->clus_ratio.load(std::memory_order_relaxed)) >> 16;
    const uint64_t h = std::min<uint64_t>(N / 4, expect - expect / 16);
    return (uint32_t)(h & ~(uint64_t)(hp::kOutChunk - 1));
}

void note_clusters(hp_ctx *ctx, uint64_t clusters, uint64_t N)
{
    if (N < 4096) return;
    const uint32_t now = (uint32_t)std::min<uint64_t>(65536, (std::min(clusters, N) << 16) / N);
    const uint32_t old = ctx->clus_ratio.load(std::memory_order_relaxed);
    ctx->clus_ratio.store((3 * old + now) / 4, std::memory_order_relaxed);
}

// Runs on the CUDA host-function thread once the event's stream work is done.
void CUDART_CB trampoline(void *p)
{
    hp_event *ev = static_cast<hp_event *>(p);
    hp_ctx *ctx = ev->ctx;
    if (!ev->on_device) note_clusters(ctx, ev->h_coff[ev->E], ev->N);
    hp_status st = HP_OK;
    for (uint32_t e = 0; e < ev->E; ++e)
        if (ev->h_status[e] != 0) {
            st = (hp_status)ev->h_status[e];
            break;
        }
    ev->status = st;
    ev->t_done = now_ns();
    ctx->dpool.free(ev->dev);
    ev->dev = Block();
    ctx->dev_in_use.fetch_sub(ev->dev_charge);
    ctx->inflight.fetch_sub(1);
    ctx->completed.fetch_add(1);
    complete_event(ev);
}

// Completion of a consumer (hits or transfer) event: its status is that of
// the consumed product (copied per event by its kernel); then the product
// loses this hold.
void CUDART_CB consumer_trampoline(void *p)
{
    hp_event *ev = static_cast<hp_event *>(p);
    hp_status st = HP_OK;
    for (uint32_t e = 0; e < ev->E; ++e)
        if (ev->h_status[e] != 0) {
            st = (hp_status)ev->h_status[e];
            break;
        }
    ev->status = st;
    ev->t_done = now_ns();
    hp_event *prod = ev->product;
    ev->product = nullptr;
    drop_hold(prod);
    complete_event(ev);
}

cudaEvent_t take_cuda_event(hp_ctx *ctx)
{
    {
        std::lock_guard<std::mutex> g(ctx->cev_mu);
        if (!ctx->cev_free.empty()) {
            cudaEvent_t e = ctx->cev_free.back();
            ctx->cev_free.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

hp_status validate_config(const hp_config *c)
{
    if (!c || !c->gain || !c->pedestal) return HP_EINVAL;
    if (c->n_modules < 1 || c->n_modules > 65536) return HP_EINVAL;
    if (c->rows < 1 || c->rows > 256 || c->cols < 1 || c->cols > 512) return HP_EINVAL;
    if ((uint64_t)c->rows * c->cols > 131072) return HP_EINVAL;
    if (c->pixel_thr < 1) return HP_EINVAL;
    const int64_t qmax_allowed = (int64_t)INT32_MAX / ((int64_t)c->rows * c->cols);
    for (uint32_t m = 0; m < c->n_modules; ++m) {
        if (c->gain[m] < 0) return HP_EINVAL;
        if (255 * (int64_t)c->gain[m] - c->pedestal[m] > qmax_allowed) return HP_EINVAL;
    }
    return HP_OK;
}

hp::Geometry geometry(const hp_ctx *ctx)
{
    hp::Geometry g;
    g.M = ctx->cfg.n_modules;
    g.R = ctx->cfg.rows;
    g.C = ctx->cfg.cols;
    g.pixel_thr = ctx->cfg.pixel_thr;
    g.cluster_thr = ctx->cfg.cluster_thr;
    g.gain = ctx->d_gain;
    g.ped = ctx->d_ped;
    return g;
}

// Launch shape bucket of the autotuner: log2 of the (event, module) items
// and log2 of the mean digis per item.
std::pair<int, int> tune_bucket(const hp_ctx *ctx, uint32_t E, uint64_t N)
{
    const uint64_t EM = std::max<uint64_t>(1, (uint64_t)E * ctx->cfg.n_modules);
    const uint64_t per = std::max<uint64_t>(1, N / EM);
    return {63 - __builtin_clzll((unsigned long long)EM), 63 - __builtin_clzll((unsigned long long)per)};
}

// Launch parameters of the clustering kernel for a launch of E events and N
// digis: the tuned entry of its bucket, else the defaults.
struct Shape {
    hp::Tuning tune;
    int grid = 1;
};

Shape shape_with(const hp_ctx *ctx, uint32_t E, const hp::Tuning &t)
{
    Shape sh;
    sh.tune = t;
    // enough blocks for tickets of the smallest size (see ticket_items)
    const uint64_t groups = ((uint64_t)E * ctx->cfg.n_modules + 3) / 4;
    const uint64_t resident = (uint64_t)ctx->sm_count * t.blocks_per_sm;
    sh.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(groups, resident));
    return sh;
}

// Settings of a bucket the autotuner has not seen: those of the nearest
// tuned bucket (the mean item size weighs four times the item count, since
// it decides which tier the items take), else a size default: items of a
// thousand digis or more on average get the single-block tile, so that the
// large ones among them stay in shared memory instead of global scratch.
hp::Tuning untuned_default(const hp_ctx *ctx, std::pair<int, int> b)
{
    hp::Tuning t;
    if (ctx->tune_mode != 0) {
        int best = 1 << 30;
        for (const auto &kv : ctx->tuned) {
            const int d = std::abs(kv.first.first - b.first) + 4 * std::abs(kv.first.second - b.second);
            if (d < best) {
                best = d;
                t = kv.second;
            }
        }
        if (best <= 4 * 2) return t;
        t = hp::Tuning{};
    }
    if (b.second >= 10 && ctx->max_tile[1] >= hp::kSmemSlots) {
        t.tile_slots = ctx->max_tile[1];
        t.blocks_per_sm = 1;
        t.ticket_max = 4;
        t.warp_max = 32;
    }
    return t;
}

Shape shape_for(hp_ctx *ctx, uint32_t E, uint64_t N)
{
    const std::pair<int, int> b = tune_bucket(ctx, E, N);
    hp::Tuning t;
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        auto it = ctx->tune_mode != 0 ? ctx->tuned.find(b) : ctx->tuned.end();
        t = it != ctx->tuned.end() ? it->second : untuned_default(ctx, b);
    }
    return shape_with(ctx, E, t);
}

// Test hooks for the next launch (hp_debug_expire_waits).
uint32_t take_debug(hp_ctx *ctx)
{
    uint32_t n = ctx->debug_withhold.load();
    while (n > 0 && !ctx->debug_withhold.compare_exchange_weak(n, n - 1)) {
    }
    return n > 0 ? hp::kDebugWithholdTicket0 : 0u;
}

bool valid_tuning(const hp_ctx *ctx, const hp::Tuning &t)
{
    if (t.blocks_per_sm < 1 || t.blocks_per_sm > 3) return false;
    if (t.tile_slots < 256 || t.tile_slots > ctx->max_tile[t.blocks_per_sm] || t.tile_slots % 256) return false;
    if (t.ticket_max != 2 && t.ticket_max != 4 && t.ticket_max != 8 && t.ticket_max != 16) return false;
    return t.warp_max == 32 || t.warp_max == 64;
}

// The autotuner's search space on this device: the default tile at two
// resident blocks per SM, the largest tile that keeps three resident, and
// the largest tile of a single block, each with tickets of 16, 8, 4 or 2
// items and a warp tier up to 64 or 32 digis.
std::vector<hp::Tuning> tuning_candidates(const hp_ctx *ctx)
{
    std::vector<hp::Tuning> c;
    for (uint32_t b = 1; b <= 3; ++b) {
        const uint32_t tile = b == 2 ? (uint32_t)hp::kSmemSlots : ctx->max_tile[b];
        if (tile < 256) continue;
        for (uint32_t tk : {16u, 8u, 4u, 2u})
            for (uint32_t wm : {64u, 32u}) {
                hp::Tuning t;
                t.tile_slots = tile;
                t.blocks_per_sm = b;
                t.ticket_max = tk;
                t.warp_max = wm;
                c.push_back(t);
            }
    }
    return c;
}

// Value of "key": in a one-line JSON object (numbers only), or -1.
double json_number(const std::string &line, const char *key)
{
    const std::string k = std::string("\"") + key + "\":";
    const size_t p = line.find(k);
    if (p == std::string::npos) return -1;
    return std::strtod(line.c_str() + p + k.size(), nullptr);
}

std::string json_string(const std::string &line, const char *key)
{
    const std::string k = std::string("\"") + key + "\": \"";
    const size_t p = line.find(k);
    if (p == std::string::npos) return "";
    const size_t q = line.find('"', p + k.size());
    return q == std::string::npos ? "" : line.substr(p + k.size(), q - p - k.size());
}

// HP_TUNE = off | cache (default) | search; HP_TUNE_CACHE = path of the
// cache file (one JSON object per line, appended by hp_autotune).  Entries
// for another device or module size are ignored.
void load_tuning(hp_ctx *ctx)
{
    const char *mode = std::getenv("HP_TUNE");
    if (mode && !std::strcmp(mode, "off")) ctx->tune_mode = 0;
    if (mode && !std::strcmp(mode, "search")) ctx->tune_mode = 2;
    const char *path = std::getenv("HP_TUNE_CACHE");
    if (!path || !*path) return;
    ctx->tune_cache = path;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char buf[1024];
    while (std::fgets(buf, sizeof buf, f)) {
        const std::string line(buf);
        if (json_string(line, "device") != ctx->device_name) continue;
        if (json_number(line, "rows") != ctx->cfg.rows || json_number(line, "cols") != ctx->cfg.cols) continue;
        hp::Tuning t;
        t.tile_slots = (uint32_t)json_number(line, "tile_slots");
        t.blocks_per_sm = (uint32_t)json_number(line, "blocks_per_sm");
        t.ticket_max = (uint32_t)json_number(line, "ticket_items");
        t.warp_max = (uint32_t)json_number(line, "warp_max");
        const int a = (int)json_number(line, "items_log2"), b = (int)json_number(line, "digis_per_item_log2");
        if (a < 0 || b < 0 || !valid_tuning(ctx, t)) continue;
        ctx->tuned[{a, b}] = t; // later lines win
    }
    std::fclose(f);
}

void save_tuning(hp_ctx *ctx, std::pair<int, int> bucket, const hp::Tuning &t, double ms)
{
    if (ctx->tune_cache.empty()) return;
    FILE *f = std::fopen(ctx->tune_cache.c_str(), "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"device\": \"%s\", \"rows\": %u, \"cols\": %u, \"items_log2\": %d, "
                 "\"digis_per_item_log2\": %d, \"tile_slots\": %u, \"blocks_per_sm\": %u, \"ticket_items\": %u, "
                 "\"warp_max\": %u, \"ms\": %.4f}\n",
                 ctx->device_name, ctx->cfg.rows, ctx->cfg.cols, bucket.first, bucket.second, t.tile_slots,
                 t.blocks_per_sm, t.ticket_max, t.warp_max, ms);
    std::fclose(f);
}

void to_public(const hp::Tuning &t, hp_tuning *o)
{
    o->tile_slots = t.tile_slots;
    o->blocks_per_sm = t.blocks_per_sm;
    o->ticket_items = t.ticket_max;
    o->warp_max = t.warp_max;
}

// Page-locked host memory (cudaHostAlloc or registered).
bool pinned_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// The address by which the device reads p: device, managed and pinned
// (mapped) host memory, and any host memory where the device reads pageable
// memory (hardware-coherent hosts); null where it cannot.
const void *device_view(const hp_ctx *ctx, const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost)
        return a.devicePointer;
    return ctx->pageable_access ? p : nullptr;
}

bool device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Most blocks of the output copy.  Into device memory: eight an SM.  Into
// mapped host memory the chip-to-chip link bounds it, and half an SM's worth
// of blocks already fill the link with whole-line stores (about 190 GB/s
// from 16 blocks of 512 threads on a GB300), so the copy leaves the other
// SMs to the next launch's kernels instead of holding all of them while its
// stores drain.
int copy_grid(const hp_ctx *ctx, bool host_outputs)
{
    return host_outputs ? std::max(16, ctx->sm_count / 2) : ctx->sm_count * 8;
}

// Timing marks for the next launch, or null when stage timers are off.
cudaEvent_t *profile_marks(hp_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    if (ctx->prof_left == 0) return nullptr;
    hp_ctx::ProfRec rec;
    for (int i = 0; i <= hp::kNumKernels; ++i) {
        if (!ctx->prof_pool.empty()) {
            rec.ev[i] = ctx->prof_pool.back();
            ctx->prof_pool.pop_back();
        } else if (cudaEventCreate(&rec.ev[i]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) ctx->prof_pool.push_back(rec.ev[j]);
            return nullptr;
        }
    }
    --ctx->prof_left;
    ctx->prof_used.push_back(rec);
    return ctx->prof_used.back().ev;
}

hp_status enqueue_impl(hp_ctx *ctx, uint32_t E, const uint64_t *offsets, uint64_t n_single, const uint32_t *words,
                       const uint16_t *mods, uint64_t tag, uint32_t flags, hp_event **out)
{
    hp::NvtxRange range("hp_enqueue");
    if (!ctx || !out) return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    if (E < 1) return HP_EINVAL;
    uint64_t N = n_single;
    if (offsets) {
        if (offsets[0] != 0) return HP_EINVAL;
        for (uint32_t e = 0; e < E; ++e)
            if (offsets[e + 1] < offsets[e]) return HP_EINVAL;
        N = offsets[E];
    }
    if (N >= 0xFFFFFFFFull) return HP_EINVAL;
    if (N > 0 && (!words || !mods)) return HP_EINVAL;
    const uint64_t EM = (uint64_t)E * ctx->cfg.n_modules;
    if (EM > (1ull << 31)) return HP_EINVAL;
    flags |= ctx->cfg.flags;
    const bool compact = (flags & HP_LABELS_U16) != 0;
    const bool labels = compact || (flags & HP_WANT_LABELS) != 0;
    const bool nocopy = (flags & HP_INPUT_NOCOPY) != 0;
    const bool keep = (flags & HP_KEEP_ON_DEVICE) != 0;
    if (compact && keep) return HP_EINVAL;

    // device block: inputs, labels, workspace
    const Shape sh = shape_for(ctx, E, N);
    const int grid = sh.grid;
    const size_t ws_bytes = hp::carve_workspace(nullptr, E, ctx->cfg.n_modules, N, ctx->cfg.rows, ctx->cfg.cols,
                                                grid, sh.tune, nullptr, ctx->sm_count);
    size_t doff = 0;
    const size_t d_words = doff;
    doff = align_up(doff + 4 * N, 256);
    const size_t d_mods = doff;
    doff = align_up(doff + 2 * N, 256);
    const size_t d_offs = doff;
    doff = align_up(doff + 8 * (E + 1), 256);
    const size_t d_label = doff;
    if (labels && !compact) doff = align_up(doff + 4 * N, 256);
    const size_t d_label16 = doff; // compact labels and item offsets, staged for one copy each
    if (compact) doff = align_up(doff + 2 * N, 256);
    const size_t d_ifirst = doff;
    if (compact) doff = align_up(doff + 4 * EM, 256);
    const uint32_t head = keep ? 0u : head_count(ctx, N);
    size_t d_head[6];
    for (int i = 0; i < 6; ++i) {
        d_head[i] = doff;
        doff = align_up(doff + 4 * (size_t)head, 256);
    }
    const size_t d_ws = doff;
    doff += ws_bytes;
    // outputs kept in device memory (HP_KEEP_ON_DEVICE): their own block, held until release
    size_t ooff = 0, o_arr[6], o_coff = 0, o_status = 0, o_label = 0;
    if (keep) {
        for (int i = 0; i < 6; ++i) {
            o_arr[i] = ooff;
            ooff = align_up(ooff + 4 * N, 256);
        }
        o_coff = ooff;
        ooff = align_up(ooff + 8 * (size_t)(E + 1), 256);
        o_status = ooff;
        ooff = align_up(ooff + 4 * (size_t)E, 256);
        o_label = ooff;
        if (labels) ooff = align_up(ooff + 4 * N, 256);
    }
    const size_t out_bytes = keep ? round_bin(ooff) : 0;
    const size_t dev_bytes = round_bin(doff) + out_bytes;

    // pinned host block: staged inputs, outputs
    size_t hoff = 0;
    const size_t h_words = hoff;
    hoff = align_up(hoff + (nocopy ? 0 : 4 * N), 256);
    const size_t h_mods = hoff;
    hoff = align_up(hoff + (nocopy ? 0 : 2 * N), 256);
    const size_t h_offs = hoff;
    hoff = align_up(hoff + 8 * (E + 1), 256);
    const size_t h_coff = hoff;
    hoff = align_up(hoff + 8 * (E + 1), 256);
    const size_t h_status = hoff;
    hoff = align_up(hoff + 4 * E, 256);
    size_t h_arr[6];
    for (int i = 0; i < 6; ++i) {
        h_arr[i] = hoff;
        if (!keep) hoff = align_up(hoff + 4 * N, 256);
    }
    const size_t h_label = hoff;
    if (labels && !keep) hoff = align_up(hoff + (compact ? 2 : 4) * N, 256);
    const size_t h_ifirst = hoff;
    if (compact) hoff = align_up(hoff + 4 * EM, 256);

    // admission: in-flight limit and device budget (non-blocking: HP_EAGAIN)
    const uint64_t maxin = ctx->cfg.max_inflight ? ctx->cfg.max_inflight : 256;
    if (ctx->inflight.fetch_add(1) >= maxin) {
        ctx->inflight.fetch_sub(1);
        return HP_EAGAIN;
    }
    const uint64_t used = ctx->dev_in_use.fetch_add(dev_bytes);
    if (ctx->cfg.device_budget_bytes && used + dev_bytes > ctx->cfg.device_budget_bytes && used > 0) {
        ctx->dev_in_use.fetch_sub(dev_bytes);
        ctx->inflight.fetch_sub(1);
        return HP_EAGAIN;
    }
    auto rollback = [&](hp_status st) {
        ctx->dev_in_use.fetch_sub(dev_bytes);
        ctx->inflight.fetch_sub(1);
        return st;
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) return rollback(fail(ctx));

    hp_event *ev = new (std::nothrow) hp_event();
    if (!ev) return rollback(HP_ENOMEM);
    ev->ctx = ctx;
    ev->E = E;
    ev->N = N;
    ev->flags = flags;
    ev->tag = tag;
    ev->dev_charge = dev_bytes - out_bytes;
    ev->dout_charge = out_bytes;
    if (ctx->dpool.alloc(doff, &ev->dev) != HP_OK) {
        delete ev;
        return rollback(HP_ENOMEM);
    }
    if (keep && ctx->dpool.alloc(ooff, &ev->dout) != HP_OK) {
        ctx->dpool.free(ev->dev);
        delete ev;
        return rollback(HP_ENOMEM);
    }
    if (ctx->hpool.alloc(hoff, &ev->host) != HP_OK) {
        ctx->dpool.free(ev->dev);
        ctx->dpool.free(ev->dout);
        delete ev;
        return rollback(HP_ENOMEM);
    }
    ev->done = take_cuda_event(ctx);
    if (!ev->done) {
        ctx->dpool.free(ev->dev);
        ctx->dpool.free(ev->dout);
        ctx->hpool.free(ev->host);
        delete ev;
        return rollback(fail(ctx));
    }
    unsigned char *hb = static_cast<unsigned char *>(ev->host.ptr);
    unsigned char *hd = static_cast<unsigned char *>(ev->host.dptr);
    unsigned char *db = static_cast<unsigned char *>(ev->dev.ptr);
    uint64_t *hoffs = reinterpret_cast<uint64_t *>(hb + h_offs);
    if (offsets)
        std::memcpy(hoffs, offsets, 8 * (size_t)(E + 1));
    else {
        hoffs[0] = 0;
        hoffs[1] = N;
    }
    const void *src_words = words, *src_mods = mods;
    bool dev_input = false;
    if (!nocopy) {
        if (N) {
            std::memcpy(hb + h_words, words, 4 * N);
            std::memcpy(hb + h_mods, mods, 2 * N);
        }
        src_words = hb + h_words;
        src_mods = hb + h_mods;
    } else if (N) {
        dev_input = device_pointer(words) && device_pointer(mods);
    }
    ev->h_coff = reinterpret_cast<uint64_t *>(hb + h_coff);
    ev->h_status = reinterpret_cast<int32_t *>(hb + h_status);
    if (!keep) {
        ev->h_module = reinterpret_cast<uint32_t *>(hb + h_arr[0]);
        ev->h_id = reinterpret_cast<int32_t *>(hb + h_arr[1]);
        ev->h_charge = reinterpret_cast<int32_t *>(hb + h_arr[2]);
        ev->h_npix = reinterpret_cast<int32_t *>(hb + h_arr[3]);
        ev->h_x = reinterpret_cast<float *>(hb + h_arr[4]);
        ev->h_y = reinterpret_cast<float *>(hb + h_arr[5]);
        ev->h_label = labels && !compact ? reinterpret_cast<int32_t *>(hb + h_label) : nullptr;
        ev->h_label16 = compact ? reinterpret_cast<uint16_t *>(hb + h_label) : nullptr;
        ev->h_ifirst = compact ? reinterpret_cast<uint32_t *>(hb + h_ifirst) : nullptr;
    }
    ev->on_device = keep;

    hp::Launch L;
    L.g = geometry(ctx);
    L.E = E;
    L.N = N;
    L.offsets = reinterpret_cast<const uint64_t *>(db + d_offs);
    L.words = dev_input ? static_cast<const uint32_t *>(words) : reinterpret_cast<const uint32_t *>(db + d_words);
    L.modules = dev_input ? static_cast<const uint16_t *>(mods) : reinterpret_cast<const uint16_t *>(db + d_mods);
    // cluster outputs go straight to mapped pinned host memory (written once
    // by the kernel), or stay in device memory until a transfer asks for them
    unsigned char *ob = keep ? static_cast<unsigned char *>(ev->dout.ptr) : hd;
    L.out.capacity = N;
    L.out.module = reinterpret_cast<uint32_t *>(ob + (keep ? o_arr[0] : h_arr[0]));
    L.out.id = reinterpret_cast<int32_t *>(ob + (keep ? o_arr[1] : h_arr[1]));
    L.out.charge = reinterpret_cast<int32_t *>(ob + (keep ? o_arr[2] : h_arr[2]));
    L.out.npix = reinterpret_cast<int32_t *>(ob + (keep ? o_arr[3] : h_arr[3]));
    L.out.x = reinterpret_cast<float *>(ob + (keep ? o_arr[4] : h_arr[4]));
    L.out.y = reinterpret_cast<float *>(ob + (keep ? o_arr[5] : h_arr[5]));
    L.out.cluster_offsets = reinterpret_cast<uint64_t *>(ob + (keep ? o_coff : h_coff));
    L.out.event_status = reinterpret_cast<int32_t *>(ob + (keep ? o_status : h_status));
    L.out.label = labels && !compact ? reinterpret_cast<int32_t *>(keep ? ob + o_label : db + d_label) : nullptr;
    if (compact) {
        L.out.label16 = reinterpret_cast<uint16_t *>(db + d_label16);
        L.out.item_first = reinterpret_cast<uint32_t *>(db + d_ifirst);
    }
    L.out.head = {reinterpret_cast<uint32_t *>(db + d_head[0]), reinterpret_cast<int32_t *>(db + d_head[1]),
                  reinterpret_cast<int32_t *>(db + d_head[2]), reinterpret_cast<int32_t *>(db + d_head[3]),
                  reinterpret_cast<float *>(db + d_head[4]), reinterpret_cast<float *>(db + d_head[5])};
    L.out.head_n = head;
    ev->dv = L.out;
    ev->dv.head_n = 0;
    if (!keep) ev->dv.label = nullptr; // the device labels go back to the pool at completion
    ev->dv.label16 = nullptr;
    ev->dv.item_first = nullptr;
    hp::carve_workspace(db + d_ws, E, ctx->cfg.n_modules, N, ctx->cfg.rows, ctx->cfg.cols, grid, sh.tune, &L.ws, ctx->sm_count);
    L.cc_grid = grid;
    L.copy_grid = copy_grid(ctx, !keep);
    L.sm_count = ctx->sm_count;
    L.tune = sh.tune;
    L.debug = take_debug(ctx);
    ev->path = offsets ? HP_PATH_BATCH : HP_PATH_EVENT;
    ev->tune_used = sh.tune;

    const uint32_t si = ctx->next_stream.fetch_add(1) % (uint32_t)ctx->streams.size();
    cudaStream_t s = ctx->streams[si];
    ev->stream = s;
    ev->t_enq = now_ns();
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        ctx->live.insert(ev);
    }
    uint64_t h2d = 8ull * (E + 1);
    cudaError_t err = cudaMemcpyAsync(db + d_offs, hoffs, 8 * (size_t)(E + 1), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && N && !dev_input) {
        err = cudaMemcpyAsync(db + d_words, src_words, 4 * N, cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(db + d_mods, src_mods, 2 * N, cudaMemcpyHostToDevice, s);
        h2d += 6 * N;
    }
    uint64_t nk = 0;
    if (err == cudaSuccess) err = hp::launch_reconstruct(L, s, &nk, profile_marks(ctx));
    if (err == cudaSuccess && head) { // the leading clusters, by DMA (see head_count)
        void *dst[6] = {ev->h_module, ev->h_id, ev->h_charge, ev->h_npix, ev->h_x, ev->h_y};
        for (int i = 0; i < 6 && err == cudaSuccess; ++i)
            err = cudaMemcpyAsync(dst[i], db + d_head[i], 4 * (size_t)head, cudaMemcpyDeviceToHost, s);
        ctx->d2h.fetch_add(24ull * head);
    }
    if (err == cudaSuccess && labels && !keep) {
        if (compact) {
            if (N) err = cudaMemcpyAsync(ev->h_label16, db + d_label16, 2 * N, cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(ev->h_ifirst, db + d_ifirst, 4 * EM, cudaMemcpyDeviceToHost, s);
            ctx->d2h.fetch_add(2 * N + 4 * EM);
        } else if (N) {
            err = cudaMemcpyAsync(ev->h_label, db + d_label, 4 * N, cudaMemcpyDeviceToHost, s);
            ctx->d2h.fetch_add(4 * N);
        }
    }
    if (err == cudaSuccess && keep) { // per-event status and offsets only: the completion needs them
        err = cudaMemcpyAsync(ev->h_coff, L.out.cluster_offsets, 8 * (size_t)(E + 1), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(ev->h_status, L.out.event_status, 4 * (size_t)E, cudaMemcpyDeviceToHost, s);
        ctx->d2h.fetch_add(8ull * (E + 1) + 4ull * E);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev->done, s);
    if (err == cudaSuccess) err = cudaLaunchHostFunc(s, trampoline, ev);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx); // the context is unusable; its memory is reclaimed by hp_destroy
    }
    ctx->h2d.fetch_add(h2d);
    ctx->kernels.fetch_add(nk);
    ctx->enqueued.fetch_add(1);
    *out = ev;
    return HP_OK;
}


// ------------------------------------------------------------------ serving

// A batch of serving requests that runs as one device pass.
struct Batch {
    hp_ctx *ctx = nullptr;
    Serve *sv = nullptr;
    Block dev, host;
    size_t dev_charge = 0;
    uint32_t E = 0;
    uint64_t N = 0;
    bool labels = false;
    uint32_t si = 0; // its stream (index into the pool)
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr}; // serving trace: device marks
    std::vector<hp_event *> reqs;
    std::atomic<uint32_t> refs{0}; // one per request, plus one while in flight
    hp_serve_trace_record rec{};   // serving trace record of this batch
    uint64_t *h_offs = nullptr, *h_coff = nullptr;
    int32_t *h_status = nullptr, *h_id = nullptr, *h_charge = nullptr, *h_npix = nullptr, *h_label = nullptr;
    uint16_t *h_label16 = nullptr; // compact labels (HP_LABELS_U16)
    uint32_t *h_ifirst = nullptr;
    uint32_t *h_module = nullptr;
    float *h_x = nullptr, *h_y = nullptr;
};

// The continuous-batching admission loop of a context: requests queue here
// and an admitter thread launches everything pending as one batch whenever a
// batch slot is free and the batch fits the device budget.
struct Serve {
    hp_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<hp_event *> pending;
    uint32_t inflight_batches = 0;
    std::vector<uint32_t> stream_load; // batches in flight on each stream of the pool
    bool stop = false;
    std::thread admitter;
};

void release_batch_ref(Batch *b)
{
    if (b->refs.fetch_sub(1) == 1) {
        b->ctx->hpool.free(b->host);
        delete b;
    }
}

// Complete requests that never reached the device (allocation or CUDA error).
void fail_requests(hp_ctx *ctx, std::vector<hp_event *> &reqs, hp_status st)
{
    const uint64_t now = now_ns();
    for (hp_event *r : reqs) {
        r->status = st;
        r->status_local = st;
        r->coff_local[0] = r->coff_local[1] = 0;
        r->h_coff = r->coff_local;
        r->h_status = &r->status_local;
        r->t_done = now;
        ctx->completed.fetch_add(1);
        complete_event(r);
    }
}

// Host function after a batch: per-request status and result views, buffers
// back to the pools, a free batch slot for the admitter, then every request's
// completion hand-off.  No CUDA call.
void CUDART_CB batch_done(void *p)
{
    Batch *b = static_cast<Batch *>(p);
    hp_ctx *ctx = b->ctx;
    const uint64_t now = now_ns();
    struct Timer { // time spent in this host function
        hp_ctx *c;
        uint64_t t;
        ~Timer() { c->serve_complete_ns.fetch_add(now_ns() - t); }
    } timer{ctx, now};
    note_clusters(ctx, b->h_coff[b->E], b->N);
    for (uint32_t e = 0; e < b->E; ++e) {
        hp_event *r = b->reqs[e];
        const uint64_t c0 = b->h_coff[e], c1 = b->h_coff[e + 1];
        r->status = (hp_status)b->h_status[e];
        r->coff_local[0] = 0;
        r->coff_local[1] = c1 >= c0 ? c1 - c0 : 0;
        r->h_coff = r->coff_local;
        r->h_status = b->h_status + e;
        r->h_module = b->h_module + c0;
        r->h_id = b->h_id + c0;
        r->h_charge = b->h_charge + c0;
        r->h_npix = b->h_npix + c0;
        r->h_x = b->h_x + c0;
        r->h_y = b->h_y + c0;
        r->h_label = b->h_label ? b->h_label + b->h_offs[e] : nullptr;
        r->h_label16 = b->h_label16 ? b->h_label16 + b->h_offs[e] : nullptr;
        r->h_ifirst = b->h_ifirst ? b->h_ifirst + (uint64_t)e * ctx->cfg.n_modules : nullptr;
        r->t_done = now;
        ctx->hpool.free(r->staging);
        r->staging = Block();
    }
    ctx->dpool.free(b->dev);
    b->dev = Block();
    ctx->dev_in_use.fetch_sub(b->dev_charge);
    ctx->completed.fetch_add(b->E);
    {
        std::lock_guard<std::mutex> g(b->sv->mu);
        b->sv->inflight_batches--;
        b->sv->stream_load[b->si]--;
        b->sv->cv.notify_all();
    }
    for (uint32_t e = 0; e < b->E; ++e) complete_event(b->reqs[e]);
    {
        std::lock_guard<std::mutex> g(ctx->trace_mu);
        if (ctx->trace.size() < ctx->trace_cap) {
            b->rec.t_done_start = now;
            b->rec.t_done_end = now_ns();
            ctx->trace.push_back(b->rec);
            ctx->trace_ev.push_back({b->tev[0], b->tev[1], b->tev[2], b->tev[3]});
        } else {
            for (cudaEvent_t e : b->tev)
                if (e) ctx->trace_spare.push_back(e);
        }
    }
    release_batch_ref(b);
}

struct BatchLayout {
    size_t d_words, d_mods, d_offs, d_label, d_label16, d_ifirst, d_head[6], d_ws, dev_bytes;
    uint32_t head;
    size_t h_offs, h_coff, h_status, h_arr[6], h_label, h_ifirst, h_table, host_bytes;
    Shape sh;
};

// Labels a batch returns: 0 none, 1 int32 (HP_WANT_LABELS), 2 compact (HP_LABELS_U16).
int label_mode(uint32_t flags)
{
    return (flags & HP_LABELS_U16) ? 2 : (flags & HP_WANT_LABELS) ? 1 : 0;
}

BatchLayout batch_layout(hp_ctx *ctx, uint32_t E, uint64_t N, int lmode, uint32_t head)
{
    const bool labels = lmode != 0, compact = lmode == 2;
    const uint64_t EM = (uint64_t)E * ctx->cfg.n_modules;
    BatchLayout l;
    l.sh = shape_for(ctx, E, N);
    const size_t ws = hp::carve_workspace(nullptr, E, ctx->cfg.n_modules, N, ctx->cfg.rows, ctx->cfg.cols,
                                          l.sh.grid, l.sh.tune, nullptr, ctx->sm_count);
    size_t d = 0;
    l.d_words = d;
    d = align_up(d + 4 * N, 256);
    l.d_mods = d;
    d = align_up(d + 2 * N, 256);
    l.d_offs = d;
    d = align_up(d + 8 * (size_t)(E + 1), 256);
    l.d_label = d;
    if (labels && !compact) d = align_up(d + 4 * N, 256);
    l.d_label16 = d;
    if (compact) d = align_up(d + 2 * N, 256);
    l.d_ifirst = d;
    if (compact) d = align_up(d + 4 * EM, 256);
    l.head = head;
    for (int i = 0; i < 6; ++i) {
        l.d_head[i] = d;
        d = align_up(d + 4 * (size_t)head, 256);
    }
    l.d_ws = d;
    l.dev_bytes = d + ws;
    size_t h = 0;
    l.h_offs = h;
    h = align_up(h + 8 * (size_t)(E + 1), 256);
    l.h_coff = h;
    h = align_up(h + 8 * (size_t)(E + 1), 256);
    l.h_status = h;
    h = align_up(h + 4 * (size_t)E, 256);
    for (int i = 0; i < 6; ++i) {
        l.h_arr[i] = h;
        h = align_up(h + 4 * N, 256);
    }
    l.h_label = h;
    if (labels) h = align_up(h + (compact ? 2 : 4) * N, 256);
    l.h_ifirst = h;
    if (compact) h = align_up(h + 4 * EM, 256);
    l.h_table = h;
    h = align_up(h + sizeof(hp::GatherEntry) * E, 256);
    l.host_bytes = h;
    return l;
}

void launch_batch(hp_ctx *ctx, Serve *sv, std::vector<hp_event *> &take)
{
    hp::NvtxRange range("hp_serve_batch");
    const uint32_t E = (uint32_t)take.size();
    const uint64_t t_start = now_ns();
    uint64_t N = 0;
    for (hp_event *r : take) N += r->N;
    const int lmode = label_mode(sv->cfg.flags | ctx->cfg.flags);
    const bool labels = lmode != 0, compact = lmode == 2;
    const BatchLayout l = batch_layout(ctx, E, N, lmode, head_count(ctx, N));
    Batch *b = new (std::nothrow) Batch();
    auto give_up = [&](hp_status st) {
        {
            std::lock_guard<std::mutex> g(sv->mu);
            sv->inflight_batches--;
            sv->cv.notify_all();
        }
        fail_requests(ctx, take, st);
    };
    if (!b) return give_up(HP_ENOMEM);
    b->ctx = ctx;
    b->sv = sv;
    b->E = E;
    b->N = N;
    b->labels = labels;
    b->reqs = take;
    b->rec.t_admit = t_start;
    b->rec.n_events = E;
    b->rec.n_digis = N;
    b->rec.t_first_submit = ~0ull;
    for (hp_event *r : take) b->rec.t_first_submit = std::min<uint64_t>(b->rec.t_first_submit, r->t_enq);
    if (ctx->dpool.alloc(round_pow2(l.dev_bytes), &b->dev, kAnyRatio) != HP_OK) {
        delete b;
        return give_up(HP_ENOMEM);
    }
    if (ctx->hpool.alloc(round_pow2(l.host_bytes), &b->host, kAnyRatio) != HP_OK) {
        ctx->dpool.free(b->dev);
        delete b;
        return give_up(HP_ENOMEM);
    }
    b->dev_charge = round_pow2(l.dev_bytes);
    ctx->dev_in_use.fetch_add(b->dev_charge);
    b->refs.store(E + 1);
    b->rec.t_pooled = now_ns();
    for (hp_event *r : take) {
        r->batch = b;
        r->path = HP_PATH_SERVING;
        r->tune_used = l.sh.tune;
    }
    unsigned char *hb = static_cast<unsigned char *>(b->host.ptr);
    unsigned char *hd = static_cast<unsigned char *>(b->host.dptr);
    unsigned char *db = static_cast<unsigned char *>(b->dev.ptr);
    b->h_offs = reinterpret_cast<uint64_t *>(hb + l.h_offs);
    b->h_coff = reinterpret_cast<uint64_t *>(hb + l.h_coff);
    b->h_status = reinterpret_cast<int32_t *>(hb + l.h_status);
    b->h_module = reinterpret_cast<uint32_t *>(hb + l.h_arr[0]);
    b->h_id = reinterpret_cast<int32_t *>(hb + l.h_arr[1]);
    b->h_charge = reinterpret_cast<int32_t *>(hb + l.h_arr[2]);
    b->h_npix = reinterpret_cast<int32_t *>(hb + l.h_arr[3]);
    b->h_x = reinterpret_cast<float *>(hb + l.h_arr[4]);
    b->h_y = reinterpret_cast<float *>(hb + l.h_arr[5]);
    b->h_label = labels && !compact ? reinterpret_cast<int32_t *>(hb + l.h_label) : nullptr;
    b->h_label16 = compact ? reinterpret_cast<uint16_t *>(hb + l.h_label) : nullptr;
    b->h_ifirst = compact ? reinterpret_cast<uint32_t *>(hb + l.h_ifirst) : nullptr;
    hp::GatherEntry *table = reinterpret_cast<hp::GatherEntry *>(hb + l.h_table);
    b->h_offs[0] = 0;
    uint32_t n_gather = 0;
    uint64_t max_gather = 0;
    for (uint32_t e = 0; e < E; ++e) {
        hp_event *r = take[e];
        b->h_offs[e + 1] = b->h_offs[e] + r->N;
        if (r->in_direct || !r->N) continue;
        table[n_gather].words = r->in_words;
        table[n_gather].modules = r->in_mods;
        table[n_gather].n = r->N;
        table[n_gather].off = b->h_offs[e];
        max_gather = std::max<uint64_t>(max_gather, r->N);
        ++n_gather;
    }

    hp::Launch L;
    L.g = geometry(ctx);
    L.E = E;
    L.N = N;
    L.offsets = reinterpret_cast<const uint64_t *>(db + l.d_offs);
    L.words = reinterpret_cast<const uint32_t *>(db + l.d_words);
    L.modules = reinterpret_cast<const uint16_t *>(db + l.d_mods);
    L.out.capacity = N;
    L.out.module = reinterpret_cast<uint32_t *>(hd + l.h_arr[0]);
    L.out.id = reinterpret_cast<int32_t *>(hd + l.h_arr[1]);
    L.out.charge = reinterpret_cast<int32_t *>(hd + l.h_arr[2]);
    L.out.npix = reinterpret_cast<int32_t *>(hd + l.h_arr[3]);
    L.out.x = reinterpret_cast<float *>(hd + l.h_arr[4]);
    L.out.y = reinterpret_cast<float *>(hd + l.h_arr[5]);
    L.out.cluster_offsets = reinterpret_cast<uint64_t *>(hd + l.h_coff);
    L.out.event_status = reinterpret_cast<int32_t *>(hd + l.h_status);
    L.out.label = labels && !compact ? reinterpret_cast<int32_t *>(db + l.d_label) : nullptr;
    if (compact) {
        L.out.label16 = reinterpret_cast<uint16_t *>(db + l.d_label16);
        L.out.item_first = reinterpret_cast<uint32_t *>(db + l.d_ifirst);
    }
    L.out.head = {reinterpret_cast<uint32_t *>(db + l.d_head[0]), reinterpret_cast<int32_t *>(db + l.d_head[1]),
                  reinterpret_cast<int32_t *>(db + l.d_head[2]), reinterpret_cast<int32_t *>(db + l.d_head[3]),
                  reinterpret_cast<float *>(db + l.d_head[4]), reinterpret_cast<float *>(db + l.d_head[5])};
    L.out.head_n = l.head;
    hp::carve_workspace(db + l.d_ws, E, ctx->cfg.n_modules, N, ctx->cfg.rows, ctx->cfg.cols, l.sh.grid, l.sh.tune,
                        &L.ws, ctx->sm_count);
    L.cc_grid = l.sh.grid;
    L.copy_grid = copy_grid(ctx, true);
    L.sm_count = ctx->sm_count;
    L.tune = l.sh.tune;

    // the stream with the fewest batches in flight, so that a batch does not
    // queue behind another while a stream is idle
    uint32_t si = 0;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        for (uint32_t i = 1; i < (uint32_t)sv->stream_load.size(); ++i)
            if (sv->stream_load[i] < sv->stream_load[si]) si = i;
        sv->stream_load[si]++;
    }
    b->si = si;
    cudaStream_t s = ctx->streams[si];
    uint64_t nk = 0;
    bool traced;
    {
        std::lock_guard<std::mutex> g(ctx->trace_mu);
        traced = ctx->trace.size() < ctx->trace_cap;
    }
    for (int i = 0; traced && i < 4; ++i)
        if (cudaEventCreate(&b->tev[i]) != cudaSuccess) {
            cudaGetLastError();
            b->tev[i] = nullptr;
        }
    auto mark = [&](int i) {
        if (b->tev[i]) cudaEventRecord(b->tev[i], s);
    };
    mark(0);
    cudaError_t err = cudaMemcpyAsync(db + l.d_offs, b->h_offs, 8 * (size_t)(E + 1), cudaMemcpyHostToDevice, s);
    uint32_t *dw = reinterpret_cast<uint32_t *>(db + l.d_words);
    uint16_t *dm = reinterpret_cast<uint16_t *>(db + l.d_mods);
    for (uint32_t e = 0; e < E && err == cudaSuccess; ++e) {
        hp_event *r = take[e];
        if (!r->in_direct || !r->N) continue;
        err = cudaMemcpyAsync(dw + b->h_offs[e], r->in_words, 4 * r->N, cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(dm + b->h_offs[e], r->in_mods, 2 * r->N, cudaMemcpyHostToDevice, s);
    }
    if (err == cudaSuccess && n_gather) {
        err = hp::launch_gather(reinterpret_cast<const hp::GatherEntry *>(hd + l.h_table), n_gather, max_gather, dw,
                                dm, s);
        ++nk;
    }
    b->rec.t_inputs = now_ns();
    mark(1);
    if (err == cudaSuccess) err = hp::launch_reconstruct(L, s, &nk, profile_marks(ctx));
    mark(2);
    b->rec.t_kernels = now_ns();
    const uint64_t EM = (uint64_t)E * ctx->cfg.n_modules;
    if (err == cudaSuccess && l.head) { // the leading clusters, by DMA (see head_count)
        void *dst[6] = {b->h_module, b->h_id, b->h_charge, b->h_npix, b->h_x, b->h_y};
        for (int i = 0; i < 6 && err == cudaSuccess; ++i)
            err = cudaMemcpyAsync(dst[i], db + l.d_head[i], 4 * (size_t)l.head, cudaMemcpyDeviceToHost, s);
        ctx->d2h.fetch_add(24ull * l.head);
    }
    if (err == cudaSuccess && compact) {
        if (N) err = cudaMemcpyAsync(b->h_label16, db + l.d_label16, 2 * N, cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(b->h_ifirst, db + l.d_ifirst, 4 * EM, cudaMemcpyDeviceToHost, s);
    } else if (err == cudaSuccess && labels && N) {
        err = cudaMemcpyAsync(b->h_label, db + l.d_label, 4 * N, cudaMemcpyDeviceToHost, s);
    }
    mark(3);
    b->rec.stream = si;
    b->rec.t_launched = now_ns();
    if (err == cudaSuccess) err = cudaLaunchHostFunc(s, batch_done, b);
    if (err != cudaSuccess) {
        cudaGetLastError();
        fail(ctx);
        for (hp_event *r : take) r->batch = nullptr; // the batch's memory is not reclaimed: the context is failed
        {
            std::lock_guard<std::mutex> g(sv->mu);
            sv->stream_load[si]--;
        }
        return give_up(HP_ECUDA);
    }
    ctx->h2d.fetch_add(6 * N + 8 * (uint64_t)(E + 1));
    if (labels) ctx->d2h.fetch_add(compact ? 2 * N + 4 * EM : 4 * N);
    ctx->kernels.fetch_add(nk);
    ctx->serve_batches.fetch_add(1);
    ctx->serve_launch_ns.fetch_add(now_ns() - t_start);
    uint64_t mb = ctx->serve_max_batch.load();
    while (E > mb && !ctx->serve_max_batch.compare_exchange_weak(mb, E)) {
    }
}

void admitter_main(hp_ctx *ctx, Serve *sv)
{
    cudaSetDevice(ctx->device);
    const uint32_t max_events = sv->cfg.max_batch_events ? sv->cfg.max_batch_events : 256;
    const uint64_t max_digis = sv->cfg.max_batch_digis ? sv->cfg.max_batch_digis : (32ull << 20);
    const uint32_t max_batches = sv->cfg.max_inflight_batches ? sv->cfg.max_inflight_batches : 3;
    const size_t budget = sv->cfg.device_budget_bytes;
    const int lmode = label_mode(sv->cfg.flags | ctx->cfg.flags);
    for (;;) {
        std::vector<hp_event *> take;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                return (sv->stop && sv->pending.empty()) ||
                       (!sv->pending.empty() && sv->inflight_batches < max_batches);
            });
            if (sv->pending.empty()) break; // stopping, and everything queued was launched
            uint64_t nd = 0;
            while (!sv->pending.empty() && take.size() < max_events) {
                hp_event *r = sv->pending.front();
                if (!take.empty() && nd + r->N > max_digis) break;
                nd += r->N;
                take.push_back(r);
                sv->pending.pop_front();
            }
            if (budget) {
                const size_t need = round_pow2(batch_layout(ctx, (uint32_t)take.size(), nd, lmode, head_count(ctx, nd)).dev_bytes);
                sv->cv.wait(lk, [&] {
                    return sv->inflight_batches == 0 || ctx->dev_in_use.load() + need <= budget;
                });
            }
            sv->inflight_batches++;
        }
        launch_batch(ctx, sv, take);
    }
}

// Before the loop starts: one cached block of the largest batch the loop
// can form, per in-flight batch (within the device budget), in the device
// and the pinned host pool, so that no batch of the loop calls cudaMalloc
// (which synchronises the device) or cudaHostAlloc (milliseconds for large
// blocks) on the admitter thread while every request waits.  Best effort: a
// block that cannot be reserved is left to the loop.
void reserve_serving(hp_ctx *ctx, const hp_serve_config &cfg)
{
    const uint32_t max_events = cfg.max_batch_events ? cfg.max_batch_events : 256;
    const uint64_t max_digis = cfg.max_batch_digis ? cfg.max_batch_digis : (32ull << 20);
    const uint32_t max_batches = cfg.max_inflight_batches ? cfg.max_inflight_batches : 3;
    const BatchLayout l = batch_layout(ctx, max_events, max_digis, label_mode(cfg.flags | ctx->cfg.flags),
                                       (uint32_t)(max_digis / 4)); // the largest head (head_count)
    // the workspace of another clustering setting may be larger (its 64-bit
    // moment scratch scales with tile and grid): leave room for the largest
    const size_t dev = round_pow2(l.dev_bytes + 16ull * hp::kMaxTileSlots * (size_t)ctx->sm_count * 3);
    const size_t host = round_pow2(l.host_bytes);
    uint32_t n = max_batches;
    if (cfg.device_budget_bytes) n = (uint32_t)std::min<uint64_t>(n, cfg.device_budget_bytes / dev);
    // A batch's host block (its results) stays taken until its requests are
    // released, which is after its slot frees up (the completion host
    // function hands the slot to the admitter before it runs the requests'
    // callbacks): two more host blocks cover the batches that complete while
    // the admitter launches the next ones.
    const uint32_t nh = max_batches + 2;
    std::vector<Block> d(n), h(nh);
    for (uint32_t i = 0; i < n; ++i)
        if (ctx->dpool.alloc(dev, &d[i]) != HP_OK) d[i] = Block();
    for (uint32_t i = 0; i < nh; ++i)
        if (ctx->hpool.alloc(host, &h[i]) != HP_OK) h[i] = Block();
    for (uint32_t i = 0; i < n; ++i) ctx->dpool.free(d[i]);
    for (uint32_t i = 0; i < nh; ++i) ctx->hpool.free(h[i]);
}

hp_status serve_stop(hp_ctx *ctx)
{
    Serve *sv = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        sv = ctx->serve;
        ctx->serve = nullptr;
    }
    if (!sv) return HP_EINVAL;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    sv->admitter.join();
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv.wait(lk, [&] { return sv->inflight_batches == 0; });
    }
    delete sv;
    return HP_OK;
}

} // namespace

namespace {

bool current_placement(hp_ctx *ctx, hp::Placement *p)
{
    std::lock_guard<std::mutex> g(ctx->geom_mu);
    if (!ctx->has_place) return false;
    *p = ctx->place;
    return true;
}

// A stream for a consumer that cannot take its product's stream: one of a
// second pool, disjoint from the producers' streams (created on first use).
cudaStream_t consumer_stream(hp_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->aux_mu);
    if (ctx->aux_streams.empty()) {
        for (size_t i = 0; i < ctx->streams.size(); ++i) {
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            ctx->aux_streams.push_back(s);
        }
        if (ctx->aux_streams.empty()) return nullptr;
    }
    return ctx->aux_streams[ctx->next_aux.fetch_add(1) % ctx->aux_streams.size()];
}

// ScopedContext (Sec. 4.2) for consumer `ev` of product `prod`: the first
// consumer takes the product's stream; a later one takes another stream and,
// unless the product's CUDA event has completed, must queue a wait on it
// (*wait).  On success the consumer holds the product and is live; on
// failure `ev` and its buffers are freed.
hp_status scope_consumer(hp_ctx *ctx, hp_event *prod, hp_event *ev, bool *wait)
{
    cudaStream_t s = prod->stream;
    *wait = false;
    hp_status st = HP_OK;
    if (prod->stream_taken.exchange(true)) {
        s = consumer_stream(ctx);
        if (!s) {
            st = fail(ctx);
        } else {
            const cudaError_t q = cudaEventQuery(prod->done);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();
                *wait = true;
            } else if (q != cudaSuccess) {
                cudaGetLastError();
                st = fail(ctx);
            }
        }
    }
    if (st != HP_OK) {
        ctx->hpool.free(ev->host);
        {
            std::lock_guard<std::mutex> g(ctx->cev_mu);
            ctx->cev_free.push_back(ev->done);
        }
        delete ev;
        return st;
    }
    ev->stream = s;
    ev->product = prod;
    prod->state.fetch_add(kHold, std::memory_order_acq_rel); // the product outlives this consumer's work
    ev->t_enq = now_ns();
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        ctx->live.insert(ev);
    }
    if (*wait)
        ctx->consumer_waits.fetch_add(1);
    else if (s == prod->stream)
        ctx->consumer_reuses.fetch_add(1);
    return HP_OK;
}

// Device alias of a pointer into an event's mapped pinned host block.
template <class T> T *device_alias(const Block &b, T *host)
{
    return reinterpret_cast<T *>(static_cast<unsigned char *>(b.dptr) +
                                 (reinterpret_cast<unsigned char *>(host) - static_cast<unsigned char *>(b.ptr)));
}

} // namespace

namespace {

hp_status check_device_args(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                            const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out)
{
    if (!ctx || !out || !d_offsets || n_events < 1) return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    if (n_digis >= 0xFFFFFFFFull) return HP_EINVAL;
    if (n_digis > 0 && (!d_words || !d_module_ids)) return HP_EINVAL;
    if (((uintptr_t)d_words & 3) || ((uintptr_t)d_module_ids & 1) || ((uintptr_t)d_offsets & 7)) return HP_EINVAL;
    if (!out->module || !out->id || !out->charge || !out->npix || !out->x || !out->y || !out->cluster_offsets ||
        !out->event_status)
        return HP_EINVAL;
    const uint64_t EM = (uint64_t)n_events * ctx->cfg.n_modules;
    if (EM > (1ull << 31)) return HP_EINVAL;
    return HP_OK;
}

// Queue one device-resident pass with its scratch at `base`.
cudaError_t device_pass(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                        const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                        const Shape &sh, void *base, cudaStream_t s, uint64_t *nk, cudaEvent_t *marks,
                        uint32_t debug = 0)
{
    hp::Launch L;
    L.g = geometry(ctx);
    L.E = n_events;
    L.N = n_digis;
    L.offsets = d_offsets;
    L.words = d_words;
    L.modules = d_module_ids;
    L.out.capacity = out->capacity;
    L.out.module = out->module;
    L.out.id = out->id;
    L.out.charge = out->charge;
    L.out.npix = out->npix;
    L.out.x = out->x;
    L.out.y = out->y;
    L.out.cluster_offsets = out->cluster_offsets;
    L.out.event_status = out->event_status;
    L.out.label = out->label;
    hp::carve_workspace(base, n_events, ctx->cfg.n_modules, n_digis, ctx->cfg.rows, ctx->cfg.cols, sh.grid, sh.tune,
                        &L.ws, ctx->sm_count);
    L.cc_grid = sh.grid;
    L.copy_grid = ctx->sm_count * 8;
    L.sm_count = ctx->sm_count;
    L.tune = sh.tune;
    L.debug = debug;
    return hp::launch_reconstruct(L, s, nk, marks);
}

void destroy_graph(hp_graph *g)
{
    cudaSetDevice(g->ctx->device);
    cudaGraphExecDestroy(g->exec);
    cudaFree(g->ws); // synchronises the device: no launch of the graph is left running
    cudaGetLastError();
    delete g;
}

} // namespace

bool hp::context_launch_params(hp_ctx *ctx, hp::Geometry *g, int *device, int *cc_grid, int *sm_count)
{
    if (!ctx || ctx->failed.load()) return false;
    *g = geometry(ctx);
    *device = ctx->device;
    *cc_grid = ctx->sm_count * (int)hp::Tuning().blocks_per_sm;
    *sm_count = ctx->sm_count;
    return true;
}

int hp::check_device_call(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                          const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out)
{
    return check_device_args(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out);
}

int hp::context_fail(hp_ctx *ctx) { return fail(ctx); }


extern "C" {

const char *hp_status_string(hp_status st)
{
    switch (st) {
    case HP_OK: return "HP_OK";
    case HP_EAGAIN: return "HP_EAGAIN";
    case HP_ENOTREADY: return "HP_ENOTREADY";
    case HP_EINVAL: return "HP_EINVAL";
    case HP_EBADDIGI: return "HP_EBADDIGI";
    case HP_EDUP: return "HP_EDUP";
    case HP_ECAPACITY: return "HP_ECAPACITY";
    case HP_ENOMEM: return "HP_ENOMEM";
    case HP_ETIMEOUT: return "HP_ETIMEOUT";
    case HP_ECUDA: return "HP_ECUDA";
    }
    return "HP_UNKNOWN";
}

hp_status hp_create(const hp_config *cfg, hp_ctx **out)
{
    if (!out) return HP_EINVAL;
    *out = nullptr;
    hp_status st = validate_config(cfg);
    if (st != HP_OK) return st;
    hp_ctx *ctx = new (std::nothrow) hp_ctx();
    if (!ctx) return HP_ENOMEM;
    ctx->cfg = *cfg;
    ctx->cfg.gain = nullptr;
    ctx->cfg.pedestal = nullptr;
    ctx->device = cfg->device;
    auto bail = [&](hp_status s) {
        if (ctx->d_gain) cudaFree(ctx->d_gain);
        for (cudaStream_t x : ctx->streams) cudaStreamDestroy(x);
        delete ctx;
        cudaGetLastError();
        return s;
    };
    if (cudaSetDevice(cfg->device) != cudaSuccess) return bail(HP_ECUDA);
    if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess)
        return bail(HP_ECUDA);
    if (hp::init_kernels(cfg->device, cfg->rows, cfg->cols, ctx->max_tile) != cudaSuccess) return bail(HP_ECUDA);
    if (ctx->max_tile[2] < (uint32_t)hp::kSmemSlots) return bail(HP_EINVAL); // the default tile must fit
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, cfg->device) == cudaSuccess) {
            std::snprintf(ctx->device_name, sizeof ctx->device_name, "%s", prop.name);
            ctx->cc_major = prop.major;
            ctx->cc_minor = prop.minor;
        }
        int pageable = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, cfg->device) != cudaSuccess)
            cudaGetLastError();
        ctx->pageable_access = pageable != 0;
    }
    load_tuning(ctx);
    const size_t M = cfg->n_modules;
    if (cudaMalloc(&ctx->d_gain, 8 * M) != cudaSuccess) return bail(HP_ENOMEM);
    ctx->d_ped = ctx->d_gain + M;
    if (cudaMemcpy(ctx->d_gain, cfg->gain, 4 * M, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_ped, cfg->pedestal, 4 * M, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(HP_ECUDA);
    const uint32_t ns = cfg->n_streams ? cfg->n_streams : 4;
    for (uint32_t i = 0; i < ns; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(HP_ECUDA);
        ctx->streams.push_back(s);
    }
    *out = ctx;
    return HP_OK;
}

hp_status hp_destroy(hp_ctx *ctx)
{
    if (!ctx) return HP_EINVAL;
    serve_stop(ctx); // drains a running serving loop (no-op otherwise)
    cudaSetDevice(ctx->device);
    for (hp_graph *g : ctx->graphs) destroy_graph(g);
    ctx->graphs.clear();
    for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s);
    for (cudaStream_t s : ctx->aux_streams) cudaStreamSynchronize(s);
    {
        std::lock_guard<std::mutex> g(ctx->ws_mu);
        for (auto &kv : ctx->stream_ws) {
            cudaStreamSynchronize(kv.first);
            cudaFree(kv.second.ptr);
        }
        ctx->stream_ws.clear();
    }
    std::vector<hp_event *> left;
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        left.assign(ctx->live.begin(), ctx->live.end());
    }
    for (hp_event *ev : left) destroy_event(ev);
    ctx->dpool.trim();
    ctx->hpool.trim();
    for (cudaEvent_t e : ctx->cev_free) cudaEventDestroy(e);
    for (auto &r : ctx->prof_used)
        for (cudaEvent_t e : r.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    clear_trace_marks(ctx);
    for (cudaStream_t s : ctx->streams) cudaStreamDestroy(s);
    for (cudaStream_t s : ctx->aux_streams) cudaStreamDestroy(s);
    for (void *p : ctx->placements) cudaFree(p);
    cudaFree(ctx->d_gain);
    const bool failed = ctx->failed.load() != 0;
    delete ctx;
    cudaGetLastError();
    return failed ? HP_ECUDA : HP_OK;
}

hp_status hp_enqueue_event(hp_ctx *ctx, const uint32_t *words, const uint16_t *module_ids, uint64_t n_digis,
                           uint64_t tag, uint32_t flags, hp_event **out)
{
    return enqueue_impl(ctx, 1, nullptr, n_digis, words, module_ids, tag, flags, out);
}

hp_status hp_enqueue_batch(hp_ctx *ctx, uint32_t n_events, const uint64_t *offsets, const uint32_t *words,
                           const uint16_t *module_ids, uint64_t tag, uint32_t flags, hp_event **out)
{
    if (!offsets) return HP_EINVAL;
    return enqueue_impl(ctx, n_events, offsets, 0, words, module_ids, tag, flags, out);
}

hp_status hp_on_complete(hp_event *ev, hp_callback cb, void *user)
{
    if (!ev || !cb) return HP_EINVAL;
    if (ev->cb) return HP_EINVAL;
    ev->cb = cb;
    ev->user = user;
    const uint32_t prev = ev->state.fetch_or(kCbSet, std::memory_order_acq_rel);
    if (prev & kCbSet) return HP_EINVAL;
    if (prev & kDone) {
        cb(user, ev, ev->status);
        set_state(ev, kCbDone);
    }
    return HP_OK;
}

hp_status hp_event_query(hp_event *ev)
{
    if (!ev) return HP_EINVAL;
    if (!(ev->state.load(std::memory_order_acquire) & kDone)) return HP_ENOTREADY;
    return ev->status;
}

hp_status hp_fetch_clusters(hp_event *ev, hp_clusters *v)
{
    if (!ev || !v || ev->hits || ev->on_device) return HP_EINVAL;
    if (!(ev->state.load(std::memory_order_acquire) & kDone)) return HP_ENOTREADY;
    v->n_events = ev->E;
    v->n_digis = ev->N;
    v->n_clusters = ev->h_coff[ev->E];
    if (v->n_clusters > ev->N) v->n_clusters = ev->N;
    v->tag = ev->tag;
    v->cluster_offsets = ev->h_coff;
    v->event_status = ev->h_status;
    v->module = ev->h_module;
    v->id = ev->h_id;
    v->charge = ev->h_charge;
    v->npix = ev->h_npix;
    v->x = ev->h_x;
    v->y = ev->h_y;
    v->label = ev->h_label;
    v->label16 = ev->h_label16;
    v->item_first = ev->h_ifirst;
    return ev->status;
}

hp_status hp_release_event(hp_event *ev)
{
    if (!ev) return HP_EINVAL;
    const uint32_t prev = set_state(ev, kReleaseReq);
    if (prev & kReleaseReq) return HP_EINVAL;
    return HP_OK;
}

hp_status hp_event_provenance(const hp_event *ev, hp_provenance *o)
{
    if (!ev || !o) return HP_EINVAL;
    const hp_ctx *ctx = ev->ctx;
    std::memset(o, 0, sizeof *o);
    std::snprintf(o->device_name, sizeof o->device_name, "%s", ctx->device_name);
    o->device = ctx->device;
    o->cc_major = ctx->cc_major;
    o->cc_minor = ctx->cc_minor;
    o->library = kLibraryId;
    o->path = ev->path;
    if (ev->path != HP_PATH_HITS && ev->path != HP_PATH_TRANSFER) to_public(ev->tune_used, &o->tuning);
    return HP_OK;
}

int hp_event_device(const hp_event *ev) { return ev ? ev->ctx->device : -1; }
void *hp_event_stream(const hp_event *ev) { return ev ? (void *)ev->stream : nullptr; }
void *hp_event_cuda_event(const hp_event *ev) { return ev ? (void *)ev->done : nullptr; }
uint64_t hp_event_latency_ns(const hp_event *ev)
{
    if (!ev || !(ev->state.load(std::memory_order_acquire) & kDone)) return 0;
    return ev->t_done - ev->t_enq;
}

hp_status hp_set_geometry(hp_ctx *ctx, const float *origin, const float *rot, float pitch_row, float pitch_col)
{
    if (!ctx || !origin || !rot) return HP_EINVAL;
    if (!(pitch_row > 0.f) || !(pitch_col > 0.f) || !std::isfinite(pitch_row) || !std::isfinite(pitch_col))
        return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    const uint32_t M = ctx->cfg.n_modules;
    // affine rows (r_i0, r_i1, o_i, 0) of each module
    std::vector<float> rows(12 * (size_t)M);
    for (uint32_t m = 0; m < M; ++m)
        for (int i = 0; i < 3; ++i) {
            float *r = &rows[12 * (size_t)m + 4 * i];
            r[0] = rot[9 * (size_t)m + 3 * i];
            r[1] = rot[9 * (size_t)m + 3 * i + 1];
            r[2] = origin[3 * (size_t)m + i];
            r[3] = 0.f;
        }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    void *d = nullptr;
    if (cudaMalloc(&d, rows.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return HP_ENOMEM;
    }
    if (cudaMemcpy(d, rows.data(), rows.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return fail(ctx);
    }
    std::lock_guard<std::mutex> g(ctx->geom_mu);
    ctx->placements.push_back(d);
    ctx->place.rows = static_cast<const float4 *>(d);
    ctx->place.M = M;
    ctx->place.pitch_row = pitch_row;
    ctx->place.pitch_col = pitch_col;
    ctx->place.half_rows = 0.5f * (float)(ctx->cfg.rows - 1);
    ctx->place.half_cols = 0.5f * (float)(ctx->cfg.cols - 1);
    ctx->has_place = true;
    return HP_OK;
}

hp_status hp_enqueue_hits(hp_event *prod, uint32_t flags, hp_event **out)
{
    hp::NvtxRange range("hp_enqueue_hits");
    if (!prod || !out || flags != 0) return HP_EINVAL;
    if (prod->request || prod->hits || prod->transfer) return HP_EINVAL;
    hp_ctx *ctx = prod->ctx;
    if (ctx->failed.load()) return HP_ECUDA;
    hp::Placement place;
    if (!current_placement(ctx, &place)) return HP_EINVAL;
    const uint32_t E = prod->E;
    const uint64_t N = prod->N;

    size_t hoff = 0;
    const size_t h_coff = hoff;
    hoff = align_up(hoff + 8 * (size_t)(E + 1), 256);
    const size_t h_status = hoff;
    hoff = align_up(hoff + 4 * (size_t)E, 256);
    size_t h_arr[4];
    for (int i = 0; i < 4; ++i) {
        h_arr[i] = hoff;
        hoff = align_up(hoff + 4 * N, 256);
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx); // the product's device (Sec. 4.2)
    hp_event *ev = new (std::nothrow) hp_event();
    if (!ev) return HP_ENOMEM;
    ev->ctx = ctx;
    ev->E = E;
    ev->N = N;
    ev->tag = prod->tag;
    ev->hits = true;
    ev->path = HP_PATH_HITS;
    if (ctx->hpool.alloc(hoff, &ev->host) != HP_OK) {
        delete ev;
        return HP_ENOMEM;
    }
    ev->done = take_cuda_event(ctx);
    if (!ev->done) {
        ctx->hpool.free(ev->host);
        delete ev;
        return fail(ctx);
    }
    unsigned char *hb = static_cast<unsigned char *>(ev->host.ptr);
    ev->h_coff = reinterpret_cast<uint64_t *>(hb + h_coff);
    ev->h_status = reinterpret_cast<int32_t *>(hb + h_status);
    ev->h_hmodule = reinterpret_cast<uint32_t *>(hb + h_arr[0]);
    ev->h_hx = reinterpret_cast<float *>(hb + h_arr[1]);
    ev->h_hy = reinterpret_cast<float *>(hb + h_arr[2]);
    ev->h_hz = reinterpret_cast<float *>(hb + h_arr[3]);

    bool wait = false;
    const hp_status sst = scope_consumer(ctx, prod, ev, &wait);
    if (sst != HP_OK) return sst;
    cudaStream_t s = ev->stream;
    hp::HitsLaunch h;
    h.p = place;
    h.E = E;
    h.capacity = N;
    h.cluster_offsets = prod->dv.cluster_offsets;
    h.event_status = prod->dv.event_status;
    h.module = prod->dv.module;
    h.x = prod->dv.x;
    h.y = prod->dv.y;
    h.hit_offsets = device_alias(ev->host, ev->h_coff);
    h.hit_status = device_alias(ev->host, ev->h_status);
    h.hit_module = device_alias(ev->host, ev->h_hmodule);
    h.hx = device_alias(ev->host, ev->h_hx);
    h.hy = device_alias(ev->host, ev->h_hy);
    h.hz = device_alias(ev->host, ev->h_hz);
    cudaError_t err = cudaSuccess;
    if (wait) err = cudaStreamWaitEvent(s, prod->done, 0);
    if (err == cudaSuccess) err = hp::launch_hits(h, 8 * ctx->sm_count, s);
    if (err == cudaSuccess) err = cudaEventRecord(ev->done, s);
    if (err == cudaSuccess) err = cudaLaunchHostFunc(s, consumer_trampoline, ev);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx); // the context is unusable; its memory is reclaimed by hp_destroy
    }
    ctx->kernels.fetch_add(1);
    *out = ev;
    return HP_OK;
}

hp_status hp_fetch_hits(hp_event *ev, hp_hits *v)
{
    if (!ev || !v || !ev->hits) return HP_EINVAL;
    if (!(ev->state.load(std::memory_order_acquire) & kDone)) return HP_ENOTREADY;
    v->n_events = ev->E;
    v->n_hits = ev->h_coff[ev->E];
    if (v->n_hits > ev->N) v->n_hits = ev->N;
    v->tag = ev->tag;
    v->hit_offsets = ev->h_coff;
    v->event_status = ev->h_status;
    v->module = ev->h_hmodule;
    v->x = ev->h_hx;
    v->y = ev->h_hy;
    v->z = ev->h_hz;
    return ev->status;
}

hp_status hp_event_device_clusters(hp_event *ev, hp_device_clusters *v)
{
    if (!ev || !v || !ev->on_device) return HP_EINVAL;
    v->capacity = ev->dv.capacity;
    v->module = ev->dv.module;
    v->id = ev->dv.id;
    v->charge = ev->dv.charge;
    v->npix = ev->dv.npix;
    v->x = ev->dv.x;
    v->y = ev->dv.y;
    v->cluster_offsets = ev->dv.cluster_offsets;
    v->event_status = ev->dv.event_status;
    v->label = ev->dv.label;
    return HP_OK;
}

hp_status hp_enqueue_transfer(hp_event *prod, uint32_t what, hp_event **out)
{
    hp::NvtxRange range("hp_enqueue_transfer");
    if (!prod || !out) return HP_EINVAL;
    if (!prod->on_device || prod->hits || prod->transfer || prod->request) return HP_EINVAL;
    if (what == 0 || (what & ~(uint32_t)(HP_TRANSFER_CLUSTERS | HP_TRANSFER_LABELS))) return HP_EINVAL;
    const bool clusters = (what & HP_TRANSFER_CLUSTERS) != 0, labels = (what & HP_TRANSFER_LABELS) != 0;
    if (labels && !prod->dv.label) return HP_EINVAL;
    hp_ctx *ctx = prod->ctx;
    if (ctx->failed.load()) return HP_ECUDA;
    const uint32_t E = prod->E;
    const uint64_t N = prod->N;
    size_t hoff = 0;
    const size_t h_coff = hoff;
    hoff = align_up(hoff + 8 * (size_t)(E + 1), 256);
    const size_t h_status = hoff;
    hoff = align_up(hoff + 4 * (size_t)E, 256);
    size_t h_arr[6];
    for (int i = 0; i < 6; ++i) {
        h_arr[i] = hoff;
        if (clusters) hoff = align_up(hoff + 4 * N, 256);
    }
    const size_t h_label = hoff;
    if (labels) hoff = align_up(hoff + 4 * N, 256);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx); // the product's device (Sec. 4.2)
    hp_event *ev = new (std::nothrow) hp_event();
    if (!ev) return HP_ENOMEM;
    ev->ctx = ctx;
    ev->E = E;
    ev->N = N;
    ev->tag = prod->tag;
    ev->transfer = true;
    ev->path = HP_PATH_TRANSFER;
    if (ctx->hpool.alloc(hoff, &ev->host) != HP_OK) {
        delete ev;
        return HP_ENOMEM;
    }
    ev->done = take_cuda_event(ctx);
    if (!ev->done) {
        ctx->hpool.free(ev->host);
        delete ev;
        return fail(ctx);
    }
    unsigned char *hb = static_cast<unsigned char *>(ev->host.ptr);
    ev->h_coff = reinterpret_cast<uint64_t *>(hb + h_coff);
    ev->h_status = reinterpret_cast<int32_t *>(hb + h_status);
    if (clusters) {
        ev->h_module = reinterpret_cast<uint32_t *>(hb + h_arr[0]);
        ev->h_id = reinterpret_cast<int32_t *>(hb + h_arr[1]);
        ev->h_charge = reinterpret_cast<int32_t *>(hb + h_arr[2]);
        ev->h_npix = reinterpret_cast<int32_t *>(hb + h_arr[3]);
        ev->h_x = reinterpret_cast<float *>(hb + h_arr[4]);
        ev->h_y = reinterpret_cast<float *>(hb + h_arr[5]);
    }
    ev->h_label = labels ? reinterpret_cast<int32_t *>(hb + h_label) : nullptr;
    bool wait = false;
    const hp_status sst = scope_consumer(ctx, prod, ev, &wait);
    if (sst != HP_OK) return sst;
    cudaStream_t s = ev->stream;
    hp::Outputs dst{};
    dst.capacity = N;
    dst.cluster_offsets = device_alias(ev->host, ev->h_coff);
    dst.event_status = device_alias(ev->host, ev->h_status);
    if (clusters) {
        dst.module = device_alias(ev->host, ev->h_module);
        dst.id = device_alias(ev->host, ev->h_id);
        dst.charge = device_alias(ev->host, ev->h_charge);
        dst.npix = device_alias(ev->host, ev->h_npix);
        dst.x = device_alias(ev->host, ev->h_x);
        dst.y = device_alias(ev->host, ev->h_y);
    }
    cudaError_t err = cudaSuccess;
    if (wait) err = cudaStreamWaitEvent(s, prod->done, 0);
    if (err == cudaSuccess) err = hp::launch_copy_out(prod->dv, dst, E, clusters, 8 * ctx->sm_count, s);
    if (err == cudaSuccess && labels && N) {
        err = cudaMemcpyAsync(ev->h_label, prod->dv.label, 4 * N, cudaMemcpyDeviceToHost, s);
        ctx->d2h.fetch_add(4 * N);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev->done, s);
    if (err == cudaSuccess) err = cudaLaunchHostFunc(s, consumer_trampoline, ev);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx); // the context is unusable; its memory is reclaimed by hp_destroy
    }
    ctx->kernels.fetch_add(1);
    *out = ev;
    return HP_OK;
}

hp_status hp_hits_device(hp_ctx *ctx, uint32_t n_events, uint64_t capacity, const uint64_t *d_cluster_offsets,
                         const uint32_t *d_module, const float *d_x, const float *d_y, float *d_hx, float *d_hy,
                         float *d_hz, void *stream)
{
    if (!ctx || !d_cluster_offsets) return HP_EINVAL;
    if (capacity > 0 && (!d_module || !d_x || !d_y || !d_hx || !d_hy || !d_hz)) return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    hp::Placement place;
    if (!current_placement(ctx, &place)) return HP_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    hp::HitsLaunch h;
    h.p = place;
    h.E = n_events;
    h.capacity = capacity;
    h.cluster_offsets = d_cluster_offsets;
    h.event_status = nullptr;
    h.module = d_module;
    h.x = d_x;
    h.y = d_y;
    h.hit_offsets = nullptr;
    h.hit_status = nullptr;
    h.hit_module = nullptr;
    h.hx = d_hx;
    h.hy = d_hy;
    h.hz = d_hz;
    if (hp::launch_hits(h, 8 * ctx->sm_count, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx);
    }
    ctx->kernels.fetch_add(1);
    return HP_OK;
}

hp_status hp_reconstruct_device(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                                const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                                void *stream)
{
    hp_status st = check_device_args(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out);
    if (st != HP_OK) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ctx->tune_mode == 2) {
        bool known;
        {
            std::lock_guard<std::mutex> g(ctx->tune_mu);
            known = ctx->tuned.count(tune_bucket(ctx, n_events, n_digis)) != 0;
        }
        if (!known) { // search mode: tune this bucket once, on this call's inputs (blocking)
            hp_tuning best;
            st = hp_autotune(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out, 3, 0, nullptr, &best,
                             nullptr);
            if (st != HP_OK) return st;
        }
    }
    const Shape sh = shape_for(ctx, n_events, n_digis);
    const size_t need = hp::carve_workspace(nullptr, n_events, ctx->cfg.n_modules, n_digis, ctx->cfg.rows,
                                            ctx->cfg.cols, sh.grid, sh.tune, nullptr, ctx->sm_count);
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->ws_mu);
        Block &b = ctx->stream_ws[s];
        if (b.bytes < need) {
            if (b.ptr) {
                if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ctx);
                cudaFree(b.ptr);
                b = Block();
            }
            void *p = nullptr;
            if (cudaMalloc(&p, need) != cudaSuccess) {
                cudaGetLastError();
                return HP_ENOMEM;
            }
            ctx->ws_mallocs.fetch_add(1);
            b.ptr = b.dptr = p;
            b.bytes = need;
        }
        base = b.ptr;
    }
    uint64_t nk = 0;
    if (device_pass(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out, sh, base, s, &nk,
                    profile_marks(ctx), take_debug(ctx)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx);
    }
    ctx->kernels.fetch_add(nk);
    return HP_OK;
}

hp_status hp_tuning_candidates(hp_ctx *ctx, uint32_t cap, hp_tuning *list, uint32_t *n)
{
    if (!ctx || !n || (cap && !list)) return HP_EINVAL;
    const std::vector<hp::Tuning> c = tuning_candidates(ctx);
    *n = (uint32_t)c.size();
    for (uint32_t i = 0; i < c.size() && i < cap; ++i) to_public(c[i], &list[i]);
    return HP_OK;
}

hp_status hp_get_tuning(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, hp_tuning *out)
{
    if (!ctx || !out || n_events < 1) return HP_EINVAL;
    to_public(shape_for(ctx, n_events, n_digis).tune, out);
    return HP_OK;
}

hp_status hp_set_tuning(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const hp_tuning *t)
{
    if (!ctx || n_events < 1) return HP_EINVAL;
    const auto bucket = tune_bucket(ctx, n_events, n_digis);
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    if (!t) {
        ctx->tuned.erase(bucket);
        return HP_OK;
    }
    hp::Tuning x;
    x.tile_slots = t->tile_slots;
    x.blocks_per_sm = t->blocks_per_sm;
    x.ticket_max = t->ticket_items;
    x.warp_max = t->warp_max;
    if (!valid_tuning(ctx, x)) return HP_EINVAL;
    ctx->tuned[bucket] = x;
    return HP_OK;
}

hp_status hp_autotune(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                      const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                      uint32_t reps, uint32_t cap, double *cand_ms, hp_tuning *best, double *best_ms)
{
    hp::NvtxRange range("hp_autotune");
    hp_status st = check_device_args(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out);
    if (st != HP_OK) return st;
    if (reps < 1) reps = 1;
    const std::vector<hp::Tuning> cands = tuning_candidates(ctx);
    if (cands.empty()) return HP_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    size_t need = 0;
    for (const hp::Tuning &t : cands) {
        const Shape sh = shape_with(ctx, n_events, t);
        need = std::max(need, hp::carve_workspace(nullptr, n_events, ctx->cfg.n_modules, n_digis, ctx->cfg.rows,
                                                  ctx->cfg.cols, sh.grid, sh.tune, nullptr, ctx->sm_count));
    }
    void *ws = nullptr;
    if (cudaMalloc(&ws, need) != cudaSuccess) {
        cudaGetLastError();
        return HP_ENOMEM;
    }
    ctx->ws_mallocs.fetch_add(1);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](hp_status r) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
        cudaFree(ws);
        cudaGetLastError();
        return r;
    };
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        return done(fail(ctx));
    double best_t = 1e300;
    size_t bi = 0;
    uint64_t nk = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        const Shape sh = shape_with(ctx, n_events, cands[i]);
        cudaError_t err = device_pass(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out, sh, ws, s, &nk,
                                      nullptr); // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        for (uint32_t r = 0; r < reps && err == cudaSuccess; ++r)
            err = device_pass(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out, sh, ws, s, &nk, nullptr);
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err != cudaSuccess) return done(fail(ctx));
        const double per = (double)ms / reps;
        if (cand_ms && i < cap) cand_ms[i] = per;
        if (per < best_t) {
            best_t = per;
            bi = i;
        }
    }
    ctx->kernels.fetch_add(nk);
    const auto bucket = tune_bucket(ctx, n_events, n_digis);
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tuned[bucket] = cands[bi];
    }
    save_tuning(ctx, bucket, cands[bi], best_t);
    if (best) to_public(cands[bi], best);
    if (best_ms) *best_ms = best_t;
    return done(HP_OK);
}

hp_status hp_graph_capture(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                           const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                           hp_graph **graph)
{
    if (!graph) return HP_EINVAL;
    *graph = nullptr;
    hp_status st = check_device_args(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out);
    if (st != HP_OK) return st;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    hp_graph *g = new (std::nothrow) hp_graph();
    if (!g) return HP_ENOMEM;
    g->ctx = ctx;
    const Shape sh = shape_for(ctx, n_events, n_digis);
    const size_t need = hp::carve_workspace(nullptr, n_events, ctx->cfg.n_modules, n_digis, ctx->cfg.rows,
                                            ctx->cfg.cols, sh.grid, sh.tune, nullptr, ctx->sm_count);
    if (cudaMalloc(&g->ws, need) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return HP_ENOMEM;
    }
    ctx->ws_mallocs.fetch_add(1);
    cudaStream_t s = nullptr;
    cudaGraph_t cg = nullptr;
    auto bail = [&](hp_status r) {
        cudaGetLastError();
        if (cg) cudaGraphDestroy(cg);
        if (s) cudaStreamDestroy(s);
        cudaFree(g->ws);
        delete g;
        cudaGetLastError();
        return r;
    };
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(ctx));
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return bail(fail(ctx));
    const cudaError_t le = device_pass(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out, sh, g->ws, s,
                                       &g->kernels, nullptr);
    const cudaError_t ce = cudaStreamEndCapture(s, &cg);
    if (le != cudaSuccess || ce != cudaSuccess || !cg) return bail(fail(ctx));
    if (cudaGraphInstantiate(&g->exec, cg, 0) != cudaSuccess) return bail(fail(ctx));
    cudaGraphDestroy(cg);
    cudaStreamDestroy(s);
    {
        std::lock_guard<std::mutex> l(ctx->graph_mu);
        ctx->graphs.insert(g);
    }
    *graph = g;
    return HP_OK;
}

hp_status hp_graph_launch(hp_graph *g, void *stream)
{
    if (!g) return HP_EINVAL;
    hp_ctx *ctx = g->ctx;
    if (ctx->failed.load()) return HP_ECUDA;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx);
    if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx);
    }
    ctx->kernels.fetch_add(g->kernels);
    return HP_OK;
}

hp_status hp_graph_destroy(hp_graph *g)
{
    if (!g) return HP_EINVAL;
    hp_ctx *ctx = g->ctx;
    {
        std::lock_guard<std::mutex> l(ctx->graph_mu);
        ctx->graphs.erase(g);
    }
    destroy_graph(g);
    return HP_OK;
}

hp_status hp_serve_start(hp_ctx *ctx, const hp_serve_config *cfg)
{
    if (!ctx || !cfg) return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    if (ctx->serve) return HP_EINVAL;
    Serve *sv = new (std::nothrow) Serve();
    if (!sv) return HP_ENOMEM;
    sv->cfg = *cfg;
    sv->stream_load.assign(ctx->streams.size(), 0);
    reserve_serving(ctx, *cfg);
    try {
        sv->admitter = std::thread(admitter_main, ctx, sv);
    } catch (...) {
        delete sv;
        return HP_ENOMEM;
    }
    ctx->serve = sv;
    return HP_OK;
}

hp_status hp_submit(hp_ctx *ctx, const uint32_t *words, const uint16_t *module_ids, uint64_t n_digis, uint64_t tag,
                    hp_callback cb, void *user, hp_event **out)
{
    if (!ctx || !out) return HP_EINVAL;
    if (ctx->failed.load()) return HP_ECUDA;
    if (n_digis >= 0xFFFFFFFFull) return HP_EINVAL;
    if (n_digis > 0 && (!words || !module_ids)) return HP_EINVAL;
    const uint64_t t_start = now_ns();
    Serve *sv = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        sv = ctx->serve;
    }
    if (!sv) return HP_EINVAL;
    const uint32_t max_pending = sv->cfg.max_pending ? sv->cfg.max_pending : 65536;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->stop) return HP_EINVAL;
        if (sv->pending.size() >= max_pending) return HP_EAGAIN;
    }
    hp_event *ev = new (std::nothrow) hp_event();
    if (!ev) return HP_ENOMEM;
    ev->ctx = ctx;
    ev->request = true;
    ev->E = 1;
    ev->N = n_digis;
    ev->tag = tag;
    ev->flags = sv->cfg.flags | ctx->cfg.flags;
    if (ev->flags & HP_INPUT_NOCOPY) {
        // the caller's buffers stay where they are until the batch reads
        // them: in place by its gather kernel where the device can address
        // them, else by one cudaMemcpyAsync each.  (Two DMA commands per
        // request made large batches queue hundreds of small copies, and the
        // copy engines then fell behind.)
        const void *dw = n_digis ? device_view(ctx, words) : nullptr;
        const void *dm = n_digis ? device_view(ctx, module_ids) : nullptr;
        ev->in_direct = !(dw && dm);
        ev->in_words = ev->in_direct ? words : static_cast<const uint32_t *>(dw);
        ev->in_mods = ev->in_direct ? module_ids : static_cast<const uint16_t *>(dm);
    } else {
        const size_t wbytes = align_up(4 * n_digis, 256);
        if (ctx->hpool.alloc(round_pow2(wbytes + 2 * n_digis + 256), &ev->staging, kServeRatio) != HP_OK) {
            delete ev;
            return HP_ENOMEM;
        }
        unsigned char *st = static_cast<unsigned char *>(ev->staging.ptr);
        if (n_digis) {
            std::memcpy(st, words, 4 * n_digis);
            std::memcpy(st + wbytes, module_ids, 2 * n_digis);
        }
        const unsigned char *sd = static_cast<const unsigned char *>(ev->staging.dptr);
        ev->in_words = reinterpret_cast<const uint32_t *>(sd);
        ev->in_mods = reinterpret_cast<const uint16_t *>(sd + wbytes);
    }
    if (cb) {
        ev->cb = cb;
        ev->user = user;
        ev->state.store(kCbSet);
    }
    ev->coff_local[0] = ev->coff_local[1] = 0;
    ev->h_coff = ev->coff_local;
    ev->h_status = &ev->status_local;
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        ctx->live.insert(ev);
    }
    ev->t_enq = now_ns();
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->pending.push_back(ev);
    }
    sv->cv.notify_one();
    ctx->serve_requests.fetch_add(1);
    ctx->enqueued.fetch_add(1);
    ctx->serve_submit_ns.fetch_add(now_ns() - t_start);
    *out = ev;
    return HP_OK;
}

hp_status hp_serve_stop(hp_ctx *ctx)
{
    if (!ctx) return HP_EINVAL;
    return serve_stop(ctx);
}

hp_status hp_serve_replay(hp_ctx *ctx, uint32_t n_threads, uint64_t n_requests, const uint64_t *arrival_ns,
                          const uint32_t *event_index, uint32_t n_pool, const uint32_t *const *pool_words,
                          const uint16_t *const *pool_modules, const uint64_t *pool_n, uint64_t *latency_ns,
                          int32_t *status, uint64_t *span_ns)
{
    if (!ctx || !arrival_ns || !event_index || !pool_words || !pool_modules || !pool_n || !latency_ns || !status ||
        !span_ns || n_threads < 1 || n_pool < 1)
        return HP_EINVAL;
    for (uint64_t i = 0; i < n_requests; ++i)
        if (event_index[i] >= n_pool) return HP_EINVAL;
    struct Shared {
        std::mutex mu;
        std::condition_variable cv;
        uint64_t remaining;
        uint64_t last_done = 0;
        uint64_t *latency;
        int32_t *status;
        hp_status submit_error = HP_OK;
    } sh;
    sh.remaining = n_requests;
    sh.latency = latency_ns;
    sh.status = status;
    struct Slot {
        Shared *sh;
        uint64_t i;
    };
    std::vector<Slot> slots(n_requests);
    // a serving loop that reads inputs in place (HP_INPUT_NOCOPY) needs them
    // in pinned memory: the driver then submits from a pinned copy of the pool
    bool nocopy = false;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        nocopy = ctx->serve && ((ctx->serve->cfg.flags | ctx->cfg.flags) & HP_INPUT_NOCOPY);
    }
    std::vector<const uint32_t *> pw(pool_words, pool_words + n_pool);
    std::vector<const uint16_t *> pm(pool_modules, pool_modules + n_pool);
    void *pinned = nullptr;
    bool copy_pool = false; // a pool the caller already keeps in pinned memory is used as it is
    for (uint32_t e = 0; nocopy && e < n_pool && !copy_pool; ++e)
        copy_pool = pool_n[e] && (!pinned_host(pool_words[e]) || !pinned_host(pool_modules[e]));
    if (copy_pool) {
        size_t total = 0;
        for (uint32_t e = 0; e < n_pool; ++e) total += align_up(4 * pool_n[e], 256) + align_up(2 * pool_n[e], 256);
        if (cudaHostAlloc(&pinned, std::max<size_t>(total, 256), cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return HP_ENOMEM;
        }
        unsigned char *q = static_cast<unsigned char *>(pinned);
        for (uint32_t e = 0; e < n_pool; ++e) {
            std::memcpy(q, pool_words[e], 4 * pool_n[e]);
            pw[e] = reinterpret_cast<const uint32_t *>(q);
            q += align_up(4 * pool_n[e], 256);
            std::memcpy(q, pool_modules[e], 2 * pool_n[e]);
            pm[e] = reinterpret_cast<const uint16_t *>(q);
            q += align_up(2 * pool_n[e], 256);
        }
    }
    auto unregister = [&]() {
        if (pinned) cudaFreeHost(pinned);
        cudaGetLastError();
    };
    auto cb = [](void *user, hp_event *ev, hp_status st) {
        Slot *sl = static_cast<Slot *>(user);
        sl->sh->latency[sl->i] = hp_event_latency_ns(ev);
        sl->sh->status[sl->i] = st;
        hp_release_event(ev);
        const uint64_t t = now_ns();
        std::lock_guard<std::mutex> g(sl->sh->mu);
        if (t > sl->sh->last_done) sl->sh->last_done = t;
        if (--sl->sh->remaining == 0) sl->sh->cv.notify_all();
    };
    const uint64_t t0 = now_ns() + 1000000; // start 1 ms from now
    auto worker = [&](uint32_t tid) {
        for (uint64_t i = tid; i < n_requests; i += n_threads) {
            const uint64_t due = t0 + arrival_ns[i];
            uint64_t now = now_ns();
            if (due > now + 100000) std::this_thread::sleep_for(std::chrono::nanoseconds(due - now - 50000));
            while (now_ns() < due) {
            }
            slots[i] = Slot{&sh, i};
            const uint32_t e = event_index[i];
            hp_event *ev = nullptr;
            for (;;) {
                const hp_status st = hp_submit(ctx, pw[e], pm[e], pool_n[e], i, +cb, &slots[i], &ev);
                if (st == HP_OK) break;
                if (st != HP_EAGAIN) {
                    std::lock_guard<std::mutex> g(sh.mu);
                    sh.submit_error = st;
                    status[i] = st;
                    latency_ns[i] = 0;
                    if (--sh.remaining == 0) sh.cv.notify_all();
                    break;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    };
    std::vector<std::thread> ts;
    for (uint32_t t = 0; t < n_threads; ++t) ts.emplace_back(worker, t);
    for (auto &t : ts) t.join();
    {
        std::unique_lock<std::mutex> lk(sh.mu);
        sh.cv.wait(lk, [&] { return sh.remaining == 0; });
    }
    unregister();
    *span_ns = sh.last_done > t0 ? sh.last_done - t0 : 0;
    return sh.submit_error;
}

hp_status hp_get_stats(hp_ctx *ctx, hp_stats *o)
{
    if (!ctx || !o) return HP_EINVAL;
    o->device_mallocs = ctx->dpool.backend_allocs() + ctx->ws_mallocs.load();
    o->host_mallocs = ctx->hpool.backend_allocs();
    o->pool_hits = ctx->dpool.hits() + ctx->hpool.hits();
    o->device_bytes_in_use = ctx->dev_in_use.load();
    o->device_bytes_cached = ctx->dpool.total_bytes();
    o->events_enqueued = ctx->enqueued.load();
    o->events_completed = ctx->completed.load();
    o->inflight = ctx->inflight.load();
    o->h2d_bytes = ctx->h2d.load();
    o->d2h_bytes = ctx->d2h.load();
    o->kernel_launches = ctx->kernels.load();
    o->serve_batches = ctx->serve_batches.load();
    o->serve_requests = ctx->serve_requests.load();
    o->serve_submit_ns = ctx->serve_submit_ns.load();
    o->serve_launch_ns = ctx->serve_launch_ns.load();
    o->serve_complete_ns = ctx->serve_complete_ns.load();
    o->serve_max_batch = ctx->serve_max_batch.load();
    o->consumer_stream_reuses = ctx->consumer_reuses.load();
    o->consumer_stream_waits = ctx->consumer_waits.load();
    return ctx->failed.load() ? HP_ECUDA : HP_OK;
}

hp_status hp_serve_trace_enable(hp_ctx *ctx, uint64_t cap)
{
    if (!ctx) return HP_EINVAL;
    std::lock_guard<std::mutex> g(ctx->trace_mu);
    clear_trace_marks(ctx);
    ctx->trace.clear();
    ctx->trace.reserve(cap);
    ctx->trace_cap = cap;
    return HP_OK;
}

hp_status hp_serve_trace_read(hp_ctx *ctx, hp_serve_trace_record *out, uint64_t cap, uint64_t *n)
{
    if (!ctx || !n || (cap && !out)) return HP_EINVAL;
    std::lock_guard<std::mutex> g(ctx->trace_mu);
    *n = ctx->trace.size();
    cudaEvent_t base = nullptr; // the first traced batch's start
    for (auto &a : ctx->trace_ev)
        if (a[0]) {
            base = a[0];
            break;
        }
    for (uint64_t i = 0; i < cap && i < ctx->trace.size(); ++i) {
        out[i] = ctx->trace[i];
        int64_t *g[4] = {&out[i].gpu_start, &out[i].gpu_inputs, &out[i].gpu_kernels, &out[i].gpu_outputs};
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            const cudaEvent_t e = ctx->trace_ev[i][k];
            *g[k] = base && e && cudaEventElapsedTime(&ms, base, e) == cudaSuccess ? (int64_t)(ms * 1e6) : -1;
        }
    }
    cudaGetLastError();
    return HP_OK;
}

hp_status hp_profile_enable(hp_ctx *ctx, uint32_t max_launches)
{
    if (!ctx) return HP_EINVAL;
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    ctx->prof_left = max_launches;
    if (max_launches == 0) {
        for (auto &r : ctx->prof_used)
            for (cudaEvent_t e : r.ev) ctx->prof_pool.push_back(e);
        ctx->prof_used.clear();
    }
    return HP_OK;
}

hp_status hp_profile_read(hp_ctx *ctx, uint32_t cap, const char **names, double *total_ms, uint64_t *launches,
                          uint32_t *n_kernels)
{
    if (!ctx || !n_kernels) return HP_EINVAL;
    double ms[hp::kNumKernels] = {0};
    uint64_t cnt[hp::kNumKernels] = {0};
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    for (auto &r : ctx->prof_used) {
        if (cudaEventSynchronize(r.ev[hp::kNumKernels]) != cudaSuccess) return fail(ctx);
        for (int i = 0; i < hp::kNumKernels; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.ev[i], r.ev[i + 1]) != cudaSuccess) return fail(ctx);
            ms[i] += t;
            cnt[i] += 1;
        }
    }
    *n_kernels = hp::kNumKernels;
    for (uint32_t i = 0; i < cap && i < (uint32_t)hp::kNumKernels; ++i) {
        if (names) names[i] = hp::kKernelNames[i];
        if (total_ms) total_ms[i] = ms[i];
        if (launches) launches[i] = cnt[i];
    }
    return HP_OK;
}

hp_status hp_debug_expire_waits(hp_ctx *ctx, uint32_t count)
{
    if (!ctx) return HP_EINVAL;
    ctx->debug_withhold.store(count);
    return HP_OK;
}

hp_status hp_debug_fail_allocations(hp_ctx *ctx, uint32_t count)
{
    if (!ctx) return HP_EINVAL;
    ctx->dpool.fail_next(count);
    return HP_OK;
}

} // extern "C"
