// Continuous batching (serving) of libhp: requests submitted one event at a
// time (hp_submit, the non-blocking acquire() of Sec. 2) are gathered by an
// admitter thread into batches that run as one device pass each, under a
// device budget and a limit of batches in flight (the pools of Sec. 4.1);
// a host function after each batch hands every request its slice of the
// results and fires its callback.  Also the native load driver
// (hp_serve_replay) and the serving trace.
#include "hp_runtime.h"

namespace hp {
namespace rt {

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
    if (err == cudaSuccess && l.head) { // the leading clusters, by DMA (see head_count): one 2D copy of six rows
        err = cudaMemcpy2DAsync(b->h_module, l.h_arr[1] - l.h_arr[0], db + l.d_head[0], l.d_head[1] - l.d_head[0],
                                4 * (size_t)l.head, 6, cudaMemcpyDeviceToHost, s);
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

} // namespace rt
} // namespace hp

extern "C" {

hp_status hp_serve_start(hp_ctx *ctx, const hp_serve_config *cfg)
{
    if (!ctx || !cfg || ctx->cpu) return HP_EINVAL;
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
    // times from `base`, then shifted so that the earliest traced start is 0
    // (records are in completion order, which need not be launch order)
    const uint64_t n_out = std::min<uint64_t>(cap, ctx->trace.size());
    std::vector<std::array<int64_t, 4>> t(n_out);
    int64_t t0 = INT64_MAX;
    for (uint64_t i = 0; i < n_out; ++i)
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            const cudaEvent_t e = ctx->trace_ev[i][k];
            const bool ok = base && e && cudaEventElapsedTime(&ms, base, e) == cudaSuccess;
            t[i][k] = ok ? (int64_t)((double)ms * 1e6) : INT64_MIN;
            if (ok && k == 0) t0 = std::min(t0, t[i][k]);
        }
    for (uint64_t i = 0; i < n_out; ++i) {
        out[i] = ctx->trace[i];
        int64_t *g[4] = {&out[i].gpu_start, &out[i].gpu_inputs, &out[i].gpu_kernels, &out[i].gpu_outputs};
        for (int k = 0; k < 4; ++k) *g[k] = t[i][k] == INT64_MIN ? -1 : t[i][k] - t0;
    }
    cudaGetLastError();
    return HP_OK;
}

} // extern "C"
