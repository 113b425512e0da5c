// The runtime side of the CPU case (Sec. 3, the SwitchProducer): the
// contexts hp_create makes when the caller asks for the CPU case
// (HP_FORCE_CPU set to anything but "0", or HP_ALLOW_CPU where no device is
// usable), their job queue and the events they produce.
// The product is the same hp_clusters view as on the GPU, and its
// provenance says HP_PATH_CPU and names the host, so that a consumer does
// not depend on the choice and a reader can tell afterwards which one ran.
#include "hp_runtime.h"

namespace hp {
namespace rt {

namespace {

// Run the queued events in order; each spreads over the thread pool.
void cpu_dispatch(hp_ctx *ctx)
{
    for (;;) {
        hp_event *ev = nullptr;
        {
            std::unique_lock<std::mutex> lk(ctx->cpu_mu);
            ctx->cpu_cv.wait(lk, [&] { return ctx->cpu_stop || !ctx->cpu_jobs.empty(); });
            if (ctx->cpu_jobs.empty()) return; // stopping, and the queue is drained
            ev = ctx->cpu_jobs.front();
            ctx->cpu_jobs.pop_front();
            ctx->cpu_busy = true;
        }
        hp::cpu::Geometry g{ctx->cfg.n_modules, ctx->cfg.rows, ctx->cfg.cols, ctx->cfg.pixel_thr,
                            ctx->cfg.cluster_thr, ctx->h_gain.data(), ctx->h_ped.data()};
        hp::cpu::Outputs o;
        o.module = ev->h_module;
        o.id = ev->h_id;
        o.charge = ev->h_charge;
        o.npix = ev->h_npix;
        o.x = ev->h_x;
        o.y = ev->h_y;
        o.cluster_offsets = ev->h_coff;
        o.event_status = ev->h_status;
        o.label = ev->h_label;
        o.label16 = ev->h_label16;
        o.item_first = ev->h_ifirst;
        hp::cpu::reconstruct(g, ev->E, ev->cpu_offsets.data(), ev->in_words, ev->in_mods, o, *ctx->cpu_pool);
        hp_status st = HP_OK;
        for (uint32_t e = 0; e < ev->E && st == HP_OK; ++e) st = (hp_status)ev->h_status[e];
        ev->status = st;
        ev->t_done = now_ns();
        ctx->inflight.fetch_sub(1);
        ctx->completed.fetch_add(1);
        complete_event(ev);
        {
            std::lock_guard<std::mutex> g2(ctx->cpu_mu);
            ctx->cpu_busy = false;
        }
        ctx->cpu_cv.notify_all();
    }
}

} // namespace

hp_status cpu_create(hp_ctx *ctx, const hp_config *cfg)
{
    ctx->cpu = true;
    ctx->device = -1;
    ctx->h_gain.assign(cfg->gain, cfg->gain + cfg->n_modules);
    ctx->h_ped.assign(cfg->pedestal, cfg->pedestal + cfg->n_modules);
    unsigned threads = 0;
    if (const char *t = std::getenv("HP_CPU_THREADS")) threads = (unsigned)std::strtoul(t, nullptr, 10);
    try {
        ctx->cpu_pool.reset(new hp::cpu::ThreadPool(threads));
        ctx->cpu_thread = std::thread(cpu_dispatch, ctx);
    } catch (...) {
        return HP_ENOMEM;
    }
    std::snprintf(ctx->device_name, sizeof ctx->device_name, "host CPU (%u threads)", ctx->cpu_pool->size());
    return HP_OK;
}

void cpu_destroy(hp_ctx *ctx)
{
    {
        std::lock_guard<std::mutex> g(ctx->cpu_mu);
        ctx->cpu_stop = true;
    }
    ctx->cpu_cv.notify_all();
    if (ctx->cpu_thread.joinable()) ctx->cpu_thread.join(); // runs what is queued first
    ctx->cpu_pool.reset();
}

hp_status cpu_enqueue(hp_ctx *ctx, uint32_t E, const uint64_t *offsets, uint64_t N, const uint32_t *words,
                      const uint16_t *mods, uint64_t tag, uint32_t flags, hp_event **out)
{
    const bool compact = (flags & HP_LABELS_U16) != 0;
    const bool labels = compact || (flags & HP_WANT_LABELS) != 0;
    if (flags & HP_KEEP_ON_DEVICE) return HP_EINVAL; // no device to keep anything on
    const uint32_t max_inflight = ctx->cfg.max_inflight ? ctx->cfg.max_inflight : 256;
    if (ctx->inflight.load() >= max_inflight) return HP_EAGAIN;
    hp_event *ev = new (std::nothrow) hp_event();
    if (!ev) return HP_ENOMEM;
    const uint64_t EM = (uint64_t)E * ctx->cfg.n_modules;
    try {
        if (offsets) ev->cpu_offsets.assign(offsets, offsets + E + 1);
        else ev->cpu_offsets = {0, N};
        if (flags & HP_INPUT_NOCOPY) {
            ev->in_words = words;
            ev->in_mods = mods;
        } else {
            ev->cpu_words.assign(words, words + N);
            ev->cpu_mods.assign(mods, mods + N);
            ev->in_words = ev->cpu_words.data();
            ev->in_mods = ev->cpu_mods.data();
        }
        // outputs: six cluster columns (capacity N), offsets, statuses, labels
        size_t off = 0;
        auto take = [&](size_t bytes) { off = align_up(off + bytes, 64); };
        for (int i = 0; i < 6; ++i) take(4 * N);
        take(8 * (size_t)(E + 1));
        take(4 * (size_t)E);
        take(labels && !compact ? 4 * N : 0);
        take(compact ? 2 * N : 0);
        take(compact ? 4 * EM : 0);
        ev->cpu_out.reset(new unsigned char[off + 64]); // laid out below in the same order
    } catch (...) {
        delete ev;
        return HP_ENOMEM;
    }
    unsigned char *b = ev->cpu_out.get();
    size_t o = 0;
    auto next = [&](size_t bytes) {
        unsigned char *p = b + o;
        o = align_up(o + bytes, 64);
        return p;
    };
    ev->h_module = reinterpret_cast<uint32_t *>(next(4 * N));
    ev->h_id = reinterpret_cast<int32_t *>(next(4 * N));
    ev->h_charge = reinterpret_cast<int32_t *>(next(4 * N));
    ev->h_npix = reinterpret_cast<int32_t *>(next(4 * N));
    ev->h_x = reinterpret_cast<float *>(next(4 * N));
    ev->h_y = reinterpret_cast<float *>(next(4 * N));
    ev->h_coff = reinterpret_cast<uint64_t *>(next(8 * (size_t)(E + 1)));
    ev->h_status = reinterpret_cast<int32_t *>(next(4 * (size_t)E));
    unsigned char *l32 = next(labels && !compact ? 4 * N : 0);
    unsigned char *l16 = next(compact ? 2 * N : 0);
    unsigned char *ifi = next(compact ? 4 * EM : 0);
    ev->h_label = labels && !compact ? reinterpret_cast<int32_t *>(l32) : nullptr;
    ev->h_label16 = compact ? reinterpret_cast<uint16_t *>(l16) : nullptr;
    ev->h_ifirst = compact ? reinterpret_cast<uint32_t *>(ifi) : nullptr;
    ev->ctx = ctx;
    ev->E = E;
    ev->N = N;
    ev->flags = flags;
    ev->tag = tag;
    ev->path = HP_PATH_CPU;
    ev->t_enq = now_ns();
    {
        std::lock_guard<std::mutex> g(ctx->live_mu);
        ctx->live.insert(ev);
    }
    ctx->inflight.fetch_add(1);
    ctx->enqueued.fetch_add(1);
    {
        std::lock_guard<std::mutex> g(ctx->cpu_mu);
        ctx->cpu_jobs.push_back(ev);
    }
    ctx->cpu_cv.notify_all();
    *out = ev;
    return HP_OK;
}

} // namespace rt
} // namespace hp
