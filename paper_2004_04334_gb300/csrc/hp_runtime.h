// Private header of libhp's host runtime, shared by its three parts:
// hp_runtime.cpp (contexts, the caching pools, events with exactly-once
// completion, the enqueue paths and their consumers, the device-resident
// entry and its CUDA graphs, the C ABI of those), hp_serving.cpp (the
// continuous-batching serving loop, its load driver and trace) and
// hp_tuning.cpp (the autotuner of the clustering kernel's launch settings).
#pragma once
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
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>
#include <utility>

#include "hp.h"
#include "hp_cpu.h"
#include "hp_internal.h"

namespace hp {
namespace rt {

inline uint64_t now_ns()
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
constexpr uint64_t kMinHead = 4096; // fewer leading clusters than this go straight to the host (see head_count)
inline size_t round_pow2(size_t bytes)
{
    size_t p = 4096;
    while (p < bytes) p <<= 1;
    return p;
}

inline size_t round_bin(size_t bytes)
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

inline bool destroyable(uint32_t s)
{
    return (s & kDone) && (s & kReleaseReq) && (!(s & kCbSet) || (s & kCbDone)) && (s >> 8) == 0;
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Serve;
struct Batch;

} // namespace rt
} // namespace hp

// the runtime's own types and helpers, used unqualified by its three parts
using namespace hp::rt;

struct hp_ctx {
    hp_config cfg{};
    int device = 0;
    int sm_count = 0;
    uint32_t max_tile[4] = {0, 0, 0, 0}; // largest tile per resident-blocks count (init_kernels)
    uint32_t hash_tile[4] = {0, 0, 0, 0}; // the same for the hash label store's kernel instance
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
    // CPU case (Sec. 3, the SwitchProducer): no usable GPU, or HP_FORCE_CPU.
    // Enqueued events run in order on one dispatcher thread, each spread
    // over the host thread pool; completion callbacks run on the dispatcher.
    bool cpu = false;
    std::vector<int32_t> h_gain, h_ped;
    std::unique_ptr<hp::cpu::ThreadPool> cpu_pool;
    std::mutex cpu_mu;
    std::condition_variable cpu_cv;
    std::deque<hp_event *> cpu_jobs;
    bool cpu_stop = false, cpu_busy = false;
    std::thread cpu_thread;
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
    // CPU case (Sec. 3): the job's offsets, inputs (copied unless
    // HP_INPUT_NOCOPY) and outputs in plain host memory
    std::vector<uint64_t> cpu_offsets;
    std::vector<uint32_t> cpu_words;
    std::vector<uint16_t> cpu_mods;
    std::unique_ptr<unsigned char[]> cpu_out; // not zeroed: the reconstruction writes every used byte
};

namespace hp {
namespace rt {

// Launch parameters of the clustering kernel for a launch of E events and N
// digis: the tuned entry of its bucket, else the defaults.
struct Shape {
    hp::Tuning tune;
    int grid = 1;
};

// hp_runtime.cpp
hp_status fail(hp_ctx *ctx);
void destroy_event(hp_event *ev);
uint32_t set_state(hp_event *ev, uint32_t bits);
void complete_event(hp_event *ev);
uint32_t head_count(const hp_ctx *ctx, uint64_t N);
void note_clusters(hp_ctx *ctx, uint64_t clusters, uint64_t N);
hp::Geometry geometry(const hp_ctx *ctx);
bool pinned_host(const void *p);
const void *device_view(const hp_ctx *ctx, const void *p);
int copy_grid(const hp_ctx *ctx, bool host_outputs);
cudaEvent_t *profile_marks(hp_ctx *ctx);
hp_status cpu_create(hp_ctx *ctx, const hp_config *cfg);
void cpu_destroy(hp_ctx *ctx);
hp_status cpu_enqueue(hp_ctx *ctx, uint32_t E, const uint64_t *offsets, uint64_t N, const uint32_t *words,
                      const uint16_t *mods, uint64_t tag, uint32_t flags, hp_event **out);
hp_status check_device_args(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                            const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out);
cudaError_t device_pass(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                        const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                        const Shape &sh, void *base, cudaStream_t s, uint64_t *nk, cudaEvent_t *marks,
                        uint32_t debug = 0);

// hp_tuning.cpp
std::pair<int, int> tune_bucket(const hp_ctx *ctx, uint32_t E, uint64_t N);
Shape shape_with(const hp_ctx *ctx, uint32_t E, uint64_t N, const hp::Tuning &t);
Shape shape_for(hp_ctx *ctx, uint32_t E, uint64_t N);
bool valid_tuning(const hp_ctx *ctx, const hp::Tuning &t);
std::vector<hp::Tuning> tuning_candidates(const hp_ctx *ctx);
void load_tuning(hp_ctx *ctx);
void save_tuning(hp_ctx *ctx, std::pair<int, int> bucket, const hp::Tuning &t, double ms);
void to_public(const hp::Tuning &t, hp_tuning *o);

// hp_serving.cpp
void release_batch_ref(Batch *b);
void clear_trace_marks(hp_ctx *ctx);
hp_status serve_stop(hp_ctx *ctx);

} // namespace rt
} // namespace hp
