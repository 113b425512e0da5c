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
// rules of Sec. 4.2, and the device-resident entry and its CUDA-graph form.
// The serving loop is in hp_serving.cpp, the autotuner in hp_tuning.cpp.
#include "hp_runtime.h"

namespace hp {
namespace rt {

hp_status fail(hp_ctx *ctx)
{
    ctx->failed.store(1);
    return HP_ECUDA;
}

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
        if (ev->done) ctx->cev_free.push_back(ev->done);
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
    // below ~100 KB of records one DMA costs more than the stores it saves
    return h < kMinHead ? 0u : (uint32_t)(h & ~(uint64_t)(hp::kOutChunk - 1));
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

// Test hooks for the next launch (hp_debug_expire_waits).
uint32_t take_debug(hp_ctx *ctx)
{
    uint32_t n = ctx->debug_withhold.load();
    while (n > 0 && !ctx->debug_withhold.compare_exchange_weak(n, n - 1)) {
    }
    return n > 0 ? hp::kDebugWithholdTicket0 : 0u;
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
    if (ctx->cpu) return cpu_enqueue(ctx, E, offsets, N, words, mods, tag, flags, out);

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
    cudaError_t err = cudaSuccess;
    if (!nocopy && d_words == h_words && d_mods == h_mods && d_offs == h_offs) {
        // staged words, module ids and offsets sit at the same offsets in
        // the pinned and the device block: one copy for all three
        err = cudaMemcpyAsync(db, hb, h_offs + 8 * (size_t)(E + 1), cudaMemcpyHostToDevice, s);
        h2d += 6 * N;
    } else {
        err = cudaMemcpyAsync(db + d_offs, hoffs, 8 * (size_t)(E + 1), cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess && N && !dev_input) {
            err = cudaMemcpyAsync(db + d_words, src_words, 4 * N, cudaMemcpyHostToDevice, s);
            if (err == cudaSuccess) err = cudaMemcpyAsync(db + d_mods, src_mods, 2 * N, cudaMemcpyHostToDevice, s);
            h2d += 6 * N;
        }
    }
    uint64_t nk = 0;
    if (err == cudaSuccess) err = hp::launch_reconstruct(L, s, &nk, profile_marks(ctx));
    if (err == cudaSuccess && head) { // the leading clusters, by DMA (see head_count): one 2D copy of six rows
        err = cudaMemcpy2DAsync(ev->h_module, h_arr[1] - h_arr[0], db + d_head[0], d_head[1] - d_head[0],
                                4 * (size_t)head, 6, cudaMemcpyDeviceToHost, s);
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

hp_status check_device_args(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                            const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out)
{
    if (!ctx || !out || !d_offsets || n_events < 1 || ctx->cpu) return HP_EINVAL;
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
                        uint32_t debug)
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

} // namespace rt
} // namespace hp

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
    // the SwitchProducer's choice (Sec. 3), made only when asked for: the
    // CPU case with HP_FORCE_CPU, or with HP_ALLOW_CPU where no device is
    // usable.  Without either, a missing device fails here (HP_ECUDA): the
    // library never falls back to the host on its own.
    {
        const char *force = std::getenv("HP_FORCE_CPU");
        int ndev = 0;
        const bool no_gpu = cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev;
        cudaGetLastError();
        const bool forced = force && *force && std::strcmp(force, "0") != 0;
        if (forced || (no_gpu && (cfg->flags & HP_ALLOW_CPU))) {
            const hp_status cs = cpu_create(ctx, cfg);
            if (cs != HP_OK) {
                cpu_destroy(ctx);
                delete ctx;
                return cs;
            }
            *out = ctx;
            return HP_OK;
        }
    }
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
    if (hp::init_kernels(cfg->device, cfg->rows, cfg->cols, ctx->max_tile, ctx->hash_tile) != cudaSuccess) return bail(HP_ECUDA);
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
    if (ctx->cpu) {
        cpu_destroy(ctx); // completes what is queued
        std::vector<hp_event *> left;
        {
            std::lock_guard<std::mutex> g(ctx->live_mu);
            left.assign(ctx->live.begin(), ctx->live.end());
        }
        for (hp_event *ev : left) destroy_event(ev);
        delete ctx;
        return HP_OK;
    }
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
    if (ev->path != HP_PATH_HITS && ev->path != HP_PATH_TRANSFER && ev->path != HP_PATH_CPU)
        to_public(ev->tune_used, &o->tuning);
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
    if (!ctx || !origin || !rot || ctx->cpu) return HP_EINVAL;
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
    if (!prod || !out || flags != 0 || prod->ctx->cpu) return HP_EINVAL;
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
    if (!ctx || !d_cluster_offsets || ctx->cpu) return HP_EINVAL;
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
