// The CPU case of libhp (Sec. 3, the SwitchProducer): the same product —
// clusters ordered by (event, module, id), per-event status, labels in
// either form — computed on the host's cores, for contexts created where no
// GPU is usable or HP_FORCE_CPU asks for it.  The choice is made at runtime
// and recorded in each product's provenance, and consumers see the same
// hp_clusters view either way.
//
// Per event and module (an item), from the operation's definition:
//   decode each digi word (row = bits 0-7, column = bits 8-16, adc = bits
//   17-24, bits 25-31 zero; row < rows, column < cols, adc >= 1 and module <
//   n_modules, else the event is invalid), calibrate q = adc * gain -
//   pedestal, keep pixels with q >= pixel_thr, join kept pixels that touch
//   by an edge or a corner, and keep the components whose charge reaches
//   cluster_thr: id = smallest row * cols + col, Q, pixel count, and the
//   charge-weighted mean row and column.  A position given twice makes the
//   event invalid too (HP_EDUP); an invalid event has no clusters and every
//   label -1.
//
// The components are found in one raster pass over the item's kept pixels
// (ascending linear index) with a dense occupancy grid of the module: each
// pixel looks back at the four neighbours already visited (left, and the
// three of the row above) and joins their sets; a set's representative is
// kept at its smallest member, which is then the cluster id.  Items run in
// parallel on a pool of host threads; a prefix over the per-item cluster
// counts then places every item's clusters in the output.
#include "hp_cpu.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace hp {
namespace cpu {

namespace {

constexpr int32_t kStatusBadDigi = 4; // HP_EBADDIGI
constexpr int32_t kStatusDup = 5;     // HP_EDUP

struct Decoded {
    uint32_t row, col, adc;
    bool ok;
};

Decoded decode(uint32_t w, uint32_t R, uint32_t C)
{
    Decoded d;
    d.row = w & 0xFFu;
    d.col = (w >> 8) & 0x1FFu;
    d.adc = (w >> 17) & 0xFFu;
    d.ok = (w >> 25) == 0 && d.row < R && d.col < C && d.adc >= 1;
    return d;
}

// Correctly rounded float of s / Q for the centroid (s >= 0, Q > 0).
float ratio(long long s, long long Q)
{
    return (float)((double)s / (double)Q);
}

// One kept cluster of an item.
struct Cluster {
    int32_t id, q, np;
    float x, y;
};

// Scratch of one worker: the module's occupancy grid (digi of each pixel,
// or -1) and per-item arrays, reused across items.
struct Scratch {
    std::vector<int32_t> grid;    // the module's pixels: item digi index, or -1
    std::vector<uint32_t> lin, kpos; // per item digi: linear index; position among the kept pixels, or ~0
    std::vector<int32_t> q;          // per item digi: calibrated charge
    std::vector<uint64_t> keys;      // kept pixels as (linear index << 32 | item digi index), raster order
    std::vector<uint32_t> parent;    // union-find over positions in `keys`
    std::vector<long long> sq, sr, sc;
    std::vector<int32_t> np, rank;
};

uint32_t find(std::vector<uint32_t> &p, uint32_t a)
{
    while (p[a] != a) {
        p[a] = p[p[a]];
        a = p[a];
    }
    return a;
}

} // namespace

// ------------------------------------------------------------ thread pool

ThreadPool::ThreadPool(unsigned n)
{
    if (n == 0) n = std::max(1u, std::thread::hardware_concurrency());
    for (unsigned i = 0; i < n; ++i) workers_.emplace_back([this, i] { loop(i); });
}

ThreadPool::~ThreadPool()
{
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : workers_) t.join();
}

void ThreadPool::loop(unsigned self)
{
    uint64_t seen = 0;
    for (;;) {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        lk.unlock();
        work(self);
        lk.lock();
        if (--busy_ == 0) done_.notify_all();
    }
}

void ThreadPool::work(unsigned self)
{
    for (;;) {
        const uint64_t t = next_.fetch_add(1);
        if (t >= n_) return;
        (*fn_)(t, self);
    }
}

void ThreadPool::parallel_for(uint64_t n, const std::function<void(uint64_t, unsigned)> &fn)
{
    if (n == 0) return;
    std::lock_guard<std::mutex> one(call_mu_); // one parallel loop at a time
    {
        std::lock_guard<std::mutex> g(mu_);
        fn_ = &fn;
        n_ = n;
        next_.store(0);
        busy_ = (unsigned)workers_.size();
        ++gen_;
    }
    cv_.notify_all();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return busy_ == 0; });
    fn_ = nullptr;
}

// ------------------------------------------------------------ reconstruction

void reconstruct(const Geometry &g, uint32_t E, const uint64_t *offsets, const uint32_t *words,
                 const uint16_t *modules, const Outputs &o, ThreadPool &pool)
{
    const uint32_t M = g.M, R = g.R, C = g.C;
    const uint64_t N = offsets[E];
    const uint64_t EM = (uint64_t)E * M;
    // 1: per event, validate the digis and list them by module (stable)
    // (not zeroed up front: every entry used is written first, in parallel)
    std::unique_ptr<uint32_t[]> item_start(new uint32_t[EM + E]); // per event M + 1 starts into `bucket`
    std::unique_ptr<uint32_t[]> bucket(new uint32_t[N + 1]);       // in-event digi indices, module by module
    std::vector<std::atomic<int32_t>> status(E);
    pool.parallel_for(E, [&](uint64_t e, unsigned) {
        const uint64_t a = offsets[e], n = offsets[e + 1] - a;
        uint32_t *st = item_start.get() + e * (M + 1);
        std::fill(st, st + M + 1, 0u);
        int32_t s = 0;
        for (uint64_t i = 0; i < n && !s; ++i) {
            if (!decode(words[a + i], R, C).ok || modules[a + i] >= M) s = kStatusBadDigi;
            else ++st[modules[a + i] + 1];
        }
        status[e].store(s);
        if (s) return;
        for (uint32_t m = 0; m < M; ++m) st[m + 1] += st[m];
        std::vector<uint32_t> cur(st, st + M);
        for (uint64_t i = 0; i < n; ++i) bucket[a + cur[modules[a + i]]++] = (uint32_t)i;
    });

    // 2: per item, the clusters (kept in item order) and the labels
    std::vector<std::vector<Cluster>> found(EM);
    std::vector<Scratch> scratch(pool.size());
    auto one_item = [&](uint64_t item, unsigned w) {
        const uint32_t e = (uint32_t)(item / M), m = (uint32_t)(item % M);
        if (status[e].load()) return;
        const uint64_t a = offsets[e];
        const uint32_t *st = item_start.get() + (uint64_t)e * (M + 1);
        const uint32_t *list = bucket.get() + a + st[m];
        const uint32_t n = st[m + 1] - st[m];
        if (n == 0) return;
        Scratch &s = scratch[w];
        if (s.grid.size() != (size_t)R * C) s.grid.assign((size_t)R * C, -1);
        s.lin.resize(n);
        s.q.resize(n);
        s.kpos.assign(n, ~0u);
        s.keys.clear();
        bool dup = false;
        for (uint32_t k = 0; k < n; ++k) {
            const Decoded d = decode(words[a + list[k]], R, C);
            const uint32_t lin = d.row * C + d.col;
            s.lin[k] = lin;
            if (s.grid[lin] >= 0) dup = true;
            else s.grid[lin] = (int32_t)k;
            s.q[k] = (int32_t)d.adc * g.gain[m] - g.ped[m];
            if (s.q[k] >= g.pixel_thr) s.keys.push_back((uint64_t)lin << 32 | k);
        }
        if (dup) {
            status[e].store(kStatusDup);
        } else {
            std::sort(s.keys.begin(), s.keys.end()); // raster order
            const uint32_t P = (uint32_t)s.keys.size();
            s.parent.resize(P);
            for (uint32_t i = 0; i < P; ++i) {
                s.parent[i] = i;
                s.kpos[(uint32_t)s.keys[i]] = i;
            }
            // raster pass: join each kept pixel with its kept neighbours already visited
            for (uint32_t i = 0; i < P; ++i) {
                const uint32_t lin = (uint32_t)(s.keys[i] >> 32), r = lin / C, c = lin - r * C;
                const int dr[4] = {0, -1, -1, -1}, dc[4] = {-1, -1, 0, 1};
                for (int t = 0; t < 4; ++t) {
                    const int rr = (int)r + dr[t], cc = (int)c + dc[t];
                    if (rr < 0 || cc < 0 || cc >= (int)C) continue;
                    const int32_t k = s.grid[(uint32_t)rr * C + (uint32_t)cc];
                    if (k < 0 || s.kpos[k] == ~0u) continue;
                    uint32_t x = find(s.parent, i), y = find(s.parent, s.kpos[k]);
                    if (x == y) continue;
                    if (x < y) std::swap(x, y);
                    s.parent[x] = y; // the smaller position (smaller linear index) represents the set
                }
            }
            s.sq.assign(P, 0);
            s.sr.assign(P, 0);
            s.sc.assign(P, 0);
            s.np.assign(P, 0);
            s.rank.assign(P, -1);
            for (uint32_t i = 0; i < P; ++i) {
                const uint32_t root = find(s.parent, i), lin = (uint32_t)(s.keys[i] >> 32);
                const long long qi = s.q[(uint32_t)s.keys[i]];
                s.sq[root] += qi;
                s.sr[root] += qi * (long long)(lin / C);
                s.sc[root] += qi * (long long)(lin % C);
                s.np[root] += 1;
            }
            std::vector<Cluster> &out = found[item];
            for (uint32_t i = 0; i < P; ++i) {
                if (s.parent[i] != i || s.sq[i] < g.cluster_thr) continue;
                s.rank[i] = (int32_t)out.size();
                out.push_back({(int32_t)(s.keys[i] >> 32), (int32_t)s.sq[i], s.np[i], ratio(s.sr[i], s.sq[i]),
                               ratio(s.sc[i], s.sq[i])});
            }
            for (uint32_t k = 0; k < n; ++k) {
                const uint64_t at = a + list[k];
                int32_t lab = -1;
                uint16_t lab16 = 0xFFFFu;
                if (s.kpos[k] != ~0u) {
                    const uint32_t root = find(s.parent, s.kpos[k]);
                    if (s.rank[root] >= 0) {
                        lab = (int32_t)(s.keys[root] >> 32);
                        lab16 = (uint16_t)s.rank[root];
                    } else {
                        lab = -2;
                        lab16 = 0xFFFEu;
                    }
                }
                if (o.label) o.label[at] = lab;
                if (o.label16) o.label16[at] = lab16;
            }
        }
        for (uint32_t k = 0; k < n; ++k) s.grid[s.lin[k]] = -1;
    };
    // An event's labels interleave its modules' digis, so with enough events
    // a worker takes whole events (no two workers write the same label
    // lines); a few large events spread their modules over the workers.
    if (E >= 2 * pool.size())
        pool.parallel_for(E, [&](uint64_t e, unsigned w) {
            for (uint32_t m = 0; m < M; ++m) one_item(e * M + m, w);
        });
    else
        pool.parallel_for(EM, one_item);

    // 3: ordered output (a prefix over the items' cluster counts), statuses,
    // and an invalid event's labels
    std::vector<uint64_t> first(EM + 1, 0);
    uint64_t total = 0;
    for (uint32_t e = 0; e < E; ++e) {
        const bool ok = status[e].load() == 0;
        o.cluster_offsets[e] = total;
        for (uint32_t m = 0; m < M; ++m) {
            const uint64_t item = (uint64_t)e * M + m;
            first[item] = total;
            if (o.item_first) o.item_first[item] = (uint32_t)(total - o.cluster_offsets[e]);
            if (ok) total += found[item].size();
        }
        o.event_status[e] = status[e].load();
    }
    o.cluster_offsets[E] = total;
    pool.parallel_for(EM, [&](uint64_t item, unsigned) {
        const uint32_t e = (uint32_t)(item / M), m = (uint32_t)(item % M);
        if (status[e].load()) {
            if (m == 0)
                for (uint64_t i = offsets[e]; i < offsets[e + 1]; ++i) {
                    if (o.label) o.label[i] = -1;
                    if (o.label16) o.label16[i] = 0xFFFFu;
                }
            return;
        }
        uint64_t at = first[item];
        for (const Cluster &c : found[item]) {
            o.module[at] = m;
            o.id[at] = c.id;
            o.charge[at] = c.q;
            o.npix[at] = c.np;
            o.x[at] = c.x;
            o.y[at] = c.y;
            ++at;
        }
    });
}

} // namespace cpu
} // namespace hp
