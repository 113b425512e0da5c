// Autotuner of libhp's clustering kernel: launch settings (shared-memory
// tile, resident blocks, items per ticket, warp-tier limit, bitmap or hash
// label store and the hash store's threads per item) per launch-shape
// bucket, chosen by timing every candidate on device-resident inputs; an
// optional cache file; untuned buckets take the nearest tuned entry.
#include "hp_runtime.h"

namespace hp {
namespace rt {

// Launch shape bucket of the autotuner: log2 of the (event, module) items
// and log2 of the mean digis per item.
std::pair<int, int> tune_bucket(const hp_ctx *ctx, uint32_t E, uint64_t N)
{
    const uint64_t EM = std::max<uint64_t>(1, (uint64_t)E * ctx->cfg.n_modules);
    const uint64_t per = std::max<uint64_t>(1, N / EM);
    return {63 - __builtin_clzll((unsigned long long)EM), 63 - __builtin_clzll((unsigned long long)per)};
}

Shape shape_with(const hp_ctx *ctx, uint32_t E, uint64_t N, const hp::Tuning &t)
{
    Shape sh;
    sh.tune = t;
    // enough blocks for tickets of the smallest size (see ticket_items): one
    // item for block-tier items, four for warp-tier ones
    const uint64_t EM = (uint64_t)E * ctx->cfg.n_modules;
    const uint64_t groups = hp::large_items(N, EM) ? EM : (EM + 3) / 4;
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
    return shape_with(ctx, E, N, t);
}

bool valid_tuning(const hp_ctx *ctx, const hp::Tuning &t)
{
    if (t.blocks_per_sm < 1 || t.blocks_per_sm > 3) return false;
    if (t.tile_slots < 256 || t.tile_slots > ctx->max_tile[t.blocks_per_sm] || t.tile_slots % 256) return false;
    if (t.ticket_max != 2 && t.ticket_max != 4 && t.ticket_max != 8 && t.ticket_max != 16) return false;
    if (t.warp_max != 32 && t.warp_max != 64) return false;
    if (t.label_store == hp::kStoreBitmap) return t.item_threads == (uint32_t)hp::kCCThreads; // a block an item
    if (t.label_store != hp::kStoreHash || t.tile_slots > ctx->hash_tile[t.blocks_per_sm]) return false;
    return t.item_threads == 128 || t.item_threads == 256 || t.item_threads == 512;
}

// The autotuner's search space on this device: the default tile at two
// resident blocks per SM, the largest tile that keeps three resident, and
// the largest tile of a single block, each with the bitmap label store
// (tickets of 16, 8, 4 or 2 items, a warp tier up to 64 or 32 digis) and
// with the hash label store at 128, 256 or 512 threads an item (tickets of
// 16 or 4 items, a warp tier up to 64 digis).
std::vector<hp::Tuning> tuning_candidates(const hp_ctx *ctx)
{
    std::vector<hp::Tuning> c;
    for (uint32_t b = 1; b <= 3; ++b) {
        const uint32_t tile = b == 2 ? (uint32_t)hp::kSmemSlots : ctx->max_tile[b];
        if (tile < 256) continue;
        hp::Tuning t;
        t.tile_slots = tile;
        t.blocks_per_sm = b;
        for (uint32_t tk : {16u, 8u, 4u, 2u})
            for (uint32_t wm : {64u, 32u}) {
                t.ticket_max = tk;
                t.warp_max = wm;
                c.push_back(t);
            }
        if (tile > ctx->hash_tile[b]) continue; // the hash instance keeps fewer blocks resident with this tile
        t.label_store = hp::kStoreHash;
        t.warp_max = 64;
        for (uint32_t it : {128u, 256u, 512u})
            for (uint32_t tk : {16u, 4u}) {
                t.item_threads = it;
                t.ticket_max = tk;
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
        const double store = json_number(line, "label_store"), threads = json_number(line, "item_threads");
        if (store >= 0) t.label_store = (uint32_t)store;
        if (threads >= 0) t.item_threads = (uint32_t)threads;
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
                 "\"warp_max\": %u, \"label_store\": %u, \"item_threads\": %u, \"ms\": %.4f}\n",
                 ctx->device_name, ctx->cfg.rows, ctx->cfg.cols, bucket.first, bucket.second, t.tile_slots,
                 t.blocks_per_sm, t.ticket_max, t.warp_max, t.label_store, t.item_threads, ms);
    std::fclose(f);
}

void to_public(const hp::Tuning &t, hp_tuning *o)
{
    o->tile_slots = t.tile_slots;
    o->blocks_per_sm = t.blocks_per_sm;
    o->ticket_items = t.ticket_max;
    o->warp_max = t.warp_max;
    o->label_store = t.label_store;
    o->item_threads = t.item_threads;
}

} // namespace rt
} // namespace hp

extern "C" {

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
    x.label_store = t->label_store;
    x.item_threads = t->item_threads;
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
        const Shape sh = shape_with(ctx, n_events, n_digis, t);
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
        const Shape sh = shape_with(ctx, n_events, n_digis, cands[i]);
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

} // extern "C"
