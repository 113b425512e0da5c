// sm_103a kernels of libhp: silicon-pixel local reconstruction.
//
// One launch reconstructs a batch of E independent events (a single event is
// E = 1).  The unit of clustering work is an item = (event, module); there
// are E * M items, in (event, module) order.
//
//   hist_kernel     module histogram: count[item] (shared-memory bins per
//                   block of 4096 digis, flushed with global atomics);
//                   validates module ids
//   scan_kernel     one block per event: exclusive prefix sum of the event's
//                   M counts -> bucket start of every item (the event's digi
//                   offset is the base, so events scan independently)
//   scatter_kernel  bucket scatter: each digi's word and in-event index go to
//                   its item's bucket (block-local ranks in shared memory,
//                   one global atomic per non-empty bin to reserve a range)
//   cc_kernel       persistent clustering: blocks take tickets of up to
//                   kGroup consecutive items (the count is a tuning
//                   parameter); small items (up to 32 or 64 digis) are
//                   clustered by one warp in registers, larger items by the
//                   whole block on a shared-memory pixel bitmap with
//                   rank-addressed union-find (items beyond the tile keep
//                   their slot arrays in global scratch), or, with the hash
//                   label store (a tuning choice), by groups of 128-512
//                   threads on a hash table of the item's pixels; kept clusters are
//                   staged per item and written in (event, module, id) order
//                   once their ticket's prefix is known (a cooperative
//                   frontier over the tickets' cluster counts)
//   offsets_kernel  each item's first output position (prefix over the items'
//                   kept-cluster counts, chained across chunks)
//   copy_kernel     staged clusters to their ordered output positions; per-event
//                   status codes
//
// Clustering of one module (block tier): set a bit per digi in an occupancy
// bitmap (a bit already set is a duplicate) and a bit per surviving pixel in
// a survivor bitmap; an exclusive prefix popcount over the survivor bitmap
// gives every surviving pixel a dense slot = its rank in row-major order, so
// slot order is linear-pixel order.  Every pixel starts linked to the first
// pixel of its horizontal run; runs of adjacent rows that touch (8-adjacency)
// are joined by atomicMin linking of roots (smaller slot wins), so every root
// is the smallest slot, i.e. the smallest linear index, of its cluster.
// Charge, pixel count and the two moments sum(q * row), sum(q * col)
// accumulate per root with 32-bit shared-memory atomics (the charge always
// fits, the configuration bounds every cluster's charge; an item with a
// cluster heavy enough to overflow the moments is re-summed exactly in 64
// bits; 64-bit shared atomics measured slower); the ordinal of a
// kept cluster is the rank of its root among kept roots in slot order, so the
// per-module output is already sorted by id.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "hp_internal.h"

namespace hp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Programmatic dependent launch between the pass's kernels: each kernel lets
// the next one launch as soon as all its own blocks are running (the next
// kernel's blocks then take free SM slots and wait), and each dependent
// kernel waits, before its first access to memory, until the previous grid
// has completed and its writes are visible.  The waits are the hardware's,
// not spins.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
constexpr uint32_t kSpinLimit = 1u << 24;          // iterations of a blocking wait, at most
constexpr unsigned long long kWaitNs = 1000000000ull; // and at most one second of it

struct ItemCtx {
    uint32_t e, m, b, n;
    int32_t gain, ped;
    int32_t *label_e;    // label of the event's first digi, or null
    uint16_t *label16_e; // compact label of the event's first digi, or null (then label_e is null)
    uint32_t *err_e;     // the event's error bits
};

// Compact labels: the rank of the digi's cluster among the kept clusters of
// its item (= its staging ordinal), or these two markers.
constexpr uint16_t kLab16Below = 0xFFFFu;   // pixel below threshold (label -1)
constexpr uint16_t kLab16Dropped = 0xFFFEu; // cluster below threshold (label -2)

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive scan of one value per thread over a block of T threads with a
// single barrier: warp scans, then every warp scans the warp totals in
// registers.  tmp must not be rewritten before the caller's next barrier.
template <int T>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *tmp, uint32_t *total)
{
    static_assert(T / 32 <= 32, "one warp scans the warp totals");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    const uint32_t wt = lane < T / 32 ? tmp[lane] : 0u;
    uint32_t ws = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, ws, o);
        if (lane >= o) ws += y;
    }
    *total = __shfl_sync(kFull, ws, T / 32 - 1);
    return __shfl_sync(kFull, ws - wt, warp) + x - v;
}

// s / Q as a float offset, with s an exact integer moment: exact operands and
// one rounding when they fit the float mantissa, else integer quotient plus a
// rounded remainder fraction.
__device__ __forceinline__ float centroid(int32_t origin, long long s, int32_t Q)
{
    if (s > -16777216LL && s < 16777216LL && Q < 16777216)
        return (float)origin + (float)s / (float)Q;
    const long long qt = s / Q;
    const long long rem = s - qt * Q;
    return (float)(origin + qt) + (float)rem / (float)Q;
}

// Event and module of work item `item` (one division, by the thread that
// sets up the item's record).
__device__ __forceinline__ void item_coords(uint64_t item, uint32_t M, uint32_t *e, uint32_t *m)
{
    if (item <= 0xFFFFFFFFull) {
        const uint32_t i32 = (uint32_t)item;
        *e = i32 / M;
        *m = i32 - *e * M;
    } else {
        *e = (uint32_t)(item / M);
        *m = (uint32_t)(item - (uint64_t)*e * M);
    }
}

// Per-item record of a ticket, set up once in shared memory by one thread
// (the division by the module count and the calibration loads happen there,
// not in every thread of the block).
struct ItemRec {
    uint32_t e, m;
    int32_t gain, ped;
    uint64_t label_off; // the event's first digi
};

__device__ __forceinline__ ItemRec make_rec(const Launch &L, uint64_t item)
{
    ItemRec r;
    item_coords(item, L.g.M, &r.e, &r.m);
    r.gain = L.g.gain[r.m];
    r.ped = L.g.ped[r.m];
    r.label_off = L.offsets[r.e];
    return r;
}

__device__ __forceinline__ ItemCtx make_item(const Launch &L, const ItemRec &rec, uint32_t b, uint32_t n)
{
    ItemCtx it;
    it.e = rec.e;
    it.m = rec.m;
    it.b = b;
    it.n = n;
    it.gain = rec.gain;
    it.ped = rec.ped;
    it.label_e = L.out.label ? L.out.label + rec.label_off : nullptr;
    it.label16_e = L.out.label16 ? L.out.label16 + rec.label_off : nullptr;
    it.err_e = L.ws.event_err + rec.e;
    return it;
}

// ---------------------------------------------------------------- histogram / scatter

// Thread t of a histogram/scatter block owns the kPerThread consecutive digis
// [c0 + kPerThread * t, ...) of the block's chunk; module ids and words are
// read with 16-byte vector loads when the arrays are 16-byte aligned.
constexpr int kPerThread = kChunk / kHistThreads;
static_assert(kPerThread == 8, "vector loads below assume 8 digis per thread");

__device__ __forceinline__ void load_modules(const Launch &L, uint64_t k0, uint64_t c1, uint32_t m[kPerThread])
{
    if (((reinterpret_cast<uintptr_t>(L.modules) & 15) == 0) && k0 + kPerThread <= c1) {
        const uint4 a = *reinterpret_cast<const uint4 *>(L.modules + k0);
        m[0] = a.x & 0xFFFFu, m[1] = a.x >> 16, m[2] = a.y & 0xFFFFu, m[3] = a.y >> 16;
        m[4] = a.z & 0xFFFFu, m[5] = a.z >> 16, m[6] = a.w & 0xFFFFu, m[7] = a.w >> 16;
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) m[j] = k0 + j < c1 ? (uint32_t)L.modules[k0 + j] : 0xFFFFFFFFu;
    }
}

__device__ __forceinline__ void load_words(const Launch &L, uint64_t k0, uint64_t c1, uint32_t w[kPerThread])
{
    if (((reinterpret_cast<uintptr_t>(L.words) & 15) == 0) && k0 + kPerThread <= c1) {
        const uint4 a = *reinterpret_cast<const uint4 *>(L.words + k0);
        const uint4 b = *reinterpret_cast<const uint4 *>(L.words + k0 + 4);
        w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w, w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) w[j] = k0 + j < c1 ? L.words[k0 + j] : 0u;
    }
}

// Asynchronous 16-byte copies global -> shared (cp.async), committed as one
// group and waited for by the issuing thread only.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Prefetch of the thread's next kPerThread digis (starting at k0, all before
// c1 and 16-byte aligned) into its own slots of pf_m / pf_w; false (nothing
// issued) for a partial or unaligned group, which is then loaded directly.
__device__ __forceinline__ bool prefetch_digis(const Launch &L, uint64_t k0, uint64_t c1, uint16_t *pf_m, uint32_t *pf_w)
{
    if (k0 + kPerThread > c1 || (reinterpret_cast<uintptr_t>(L.modules) & 15) ||
        (pf_w && (reinterpret_cast<uintptr_t>(L.words) & 15)))
        return false;
    const uint32_t t = threadIdx.x * kPerThread;
    cp_async16(pf_m + t, L.modules + k0);
    if (pf_w) {
        cp_async16(pf_w + t, L.words + k0);
        cp_async16(pf_w + t + 4, L.words + k0 + 4);
    }
    cp_async_commit();
    return true;
}

__device__ __forceinline__ void take_prefetched(const uint16_t *pf_m, const uint32_t *pf_w, uint32_t m[kPerThread],
                                                uint32_t w[kPerThread])
{
    cp_async_wait_all();
    const uint32_t t = threadIdx.x * kPerThread;
    const uint4 a = *reinterpret_cast<const uint4 *>(pf_m + t);
    m[0] = a.x & 0xFFFFu, m[1] = a.x >> 16, m[2] = a.y & 0xFFFFu, m[3] = a.y >> 16;
    m[4] = a.z & 0xFFFFu, m[5] = a.z >> 16, m[6] = a.w & 0xFFFFu, m[7] = a.w >> 16;
    if (pf_w) {
        const uint4 b = *reinterpret_cast<const uint4 *>(pf_w + t);
        const uint4 c = *reinterpret_cast<const uint4 *>(pf_w + t + 4);
        w[0] = b.x, w[1] = b.y, w[2] = b.z, w[3] = b.w, w[4] = c.x, w[5] = c.y, w[6] = c.z, w[7] = c.w;
    }
}

// Event of each of the thread's digis: a binary search over the block's
// event offsets (in shared memory when they fit), then a forward walk.
constexpr uint32_t kChunkEvents = 512; // event offsets a block keeps in shared memory

__device__ __forceinline__ void digi_events(const Launch &L, const uint64_t *s_off, uint32_t ef, uint32_t el,
                                            uint64_t k0, uint32_t e_of[kPerThread])
{
    uint32_t e = ef;
    if (ef != el) {
        const bool in_sh = el - ef + 1 < kChunkEvents;
        uint32_t lo = ef, hi = el;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            const uint64_t o = in_sh ? s_off[mid - ef] : L.offsets[mid];
            if (o <= k0)
                lo = mid;
            else
                hi = mid - 1;
        }
        e = lo;
    }
    uint64_t next = e < el ? (el - ef + 1 < kChunkEvents ? s_off[e + 1 - ef] : L.offsets[e + 1]) : ~0ull;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        while (k0 + j >= next) {
            ++e;
            next = e < el ? L.offsets[e + 1] : ~0ull;
        }
        e_of[j] = e;
    }
}

// Largest e in [lo, hi] with off[e] <= k (requires off[lo] <= k), by one
// full warp: 32 probes per round shrink the interval 32-fold.
__device__ __forceinline__ uint32_t find_event_warp(const uint64_t *off, uint32_t lo, uint32_t hi, uint64_t k)
{
    const uint32_t lane = threadIdx.x & 31;
    while (lo < hi) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t p = min(hi, lo + (lane + 1) * step);
        const uint32_t le = __ballot_sync(kFull, off[p] <= k);
        if (le == 0) {
            hi = lo + step - 1;
        } else {
            const uint32_t t = 31 - __clz(le);
            const uint32_t pt = min(hi, lo + (t + 1) * step);
            if (t < 31) hi = min(hi, lo + (t + 2) * step) - 1;
            lo = pt;
            if (hi < lo) hi = lo;
        }
    }
    return lo;
}

struct ChunkInfo {
    uint64_t c0, c1, keybase;
    uint32_t ef, el, nkeys;
    bool use_sh;
};

// Digis [c0, c1) of block b of nb: contiguous ranges cut at multiples of
// kPerThread digis (so every thread's group of digis is 16-byte aligned).
__device__ __forceinline__ void block_range(uint64_t N, uint32_t b, uint32_t nb, uint64_t *c0, uint64_t *c1)
{
    const uint64_t ng = (N + kPerThread - 1) / kPerThread;
    *c0 = min(N, (uint64_t)b * ng / nb * kPerThread);
    *c1 = min(N, (uint64_t)(b + 1) * ng / nb * kPerThread);
}

// Events and (event, module) keys of the digis [c0, c1) (c0 < c1): the first
// and last event by a warp search, the events' offsets in shared memory when
// they fit, and whether the keys fit a shared-memory histogram.
__device__ __forceinline__ ChunkInfo chunk_info(const Launch &L, uint64_t c0, uint64_t c1, uint32_t *s_ev,
                                                uint64_t *s_off)
{
    ChunkInfo ci;
    ci.c0 = c0;
    ci.c1 = c1;
    if (threadIdx.x < 32) {
        const uint32_t ef = find_event_warp(L.offsets, 0, L.E - 1, ci.c0);
        const uint32_t el = find_event_warp(L.offsets, ef, L.E - 1, ci.c1 - 1);
        if (threadIdx.x == 0) {
            s_ev[0] = ef;
            s_ev[1] = el;
        }
    }
    __syncthreads();
    ci.ef = s_ev[0];
    ci.el = s_ev[1];
    if (ci.el - ci.ef + 1 < kChunkEvents)
        for (uint32_t i = threadIdx.x; i <= ci.el - ci.ef + 1; i += kHistThreads) s_off[i] = L.offsets[ci.ef + i];
    const uint64_t nk = (uint64_t)(ci.el - ci.ef + 1) * L.g.M;
    ci.use_sh = nk <= (uint64_t)kHistCap;
    ci.nkeys = ci.use_sh ? (uint32_t)nk : 0u;
    ci.keybase = (uint64_t)ci.ef * L.g.M;
    return ci;
}

// Shared-memory histogram of a block: with few (event, module) keys every
// warp counts into its own sub-histogram (atomics collide only inside a
// warp), else one shared histogram.
constexpr uint32_t kHistWarps = kHistThreads / 32;
constexpr uint32_t kSubKeys = kHistCap / kHistWarps; // keys per warp sub-histogram

// Histogram, persistent: block b counts the digis of its contiguous range
// (one event search a block), 8 module ids a thread per step with the next
// step's ids loaded ahead (cp.async), into a shared histogram over the
// range's keys, flushed once with one global atomic per non-empty key; the
// atomic's return value (the block's offset inside the key's bucket) is
// kept in blk_off for the scatter kernel.
__global__ void __launch_bounds__(kHistThreads, 3) hist_kernel(const Launch L)
{
    extern __shared__ uint32_t sh[];
    __shared__ uint32_t s_ev[2];
    pdl_trigger();
    __shared__ uint64_t s_off[kChunkEvents + 1];
    __shared__ __align__(16) uint16_t pf_m[kChunk];
    // the event offsets must run 0 = o[0] <= o[1] <= ... <= o[E] = N (the
    // device entry points take them from the caller); each block checks a
    // slice, and a violation makes every later kernel skip its writes and
    // every event report HP_EINVAL
    {
        const uint64_t e0 = (uint64_t)blockIdx.x * L.E / gridDim.x, e1 = (uint64_t)(blockIdx.x + 1) * L.E / gridDim.x;
        bool bad = false;
        for (uint64_t e = e0 + threadIdx.x; e < e1; e += kHistThreads) bad |= L.offsets[e] > L.offsets[e + 1];
        if (threadIdx.x == 0 && blockIdx.x == 0) bad |= L.offsets[0] != 0 || L.offsets[L.E] != L.N;
        if (bad) atomicOr(&L.ws.ctl[1], kErrBadOffsets);
    }
    uint64_t c0, c1;
    block_range(L.N, blockIdx.x, gridDim.x, &c0, &c1);
    if (c0 >= c1) return;
    // the first module ids are loaded before the event search, so that the
    // two latencies overlap
    uint64_t k0 = c0 + (uint64_t)threadIdx.x * kPerThread;
    uint32_t m[kPerThread], e_of[kPerThread];
    load_modules(L, k0, c1, m);
    const ChunkInfo ci = chunk_info(L, c0, c1, s_ev, s_off);
    const uint32_t M = L.g.M, warp = threadIdx.x >> 5;
    const bool sub = ci.use_sh && ci.nkeys <= kSubKeys;
    const uint32_t nbins = sub ? ci.nkeys * kHistWarps : ci.nkeys;
    for (uint32_t i = threadIdx.x; i < nbins; i += kHistThreads) sh[i] = 0;
    __syncthreads();
    uint32_t *bins = sub ? sh + warp * ci.nkeys : sh;
    for (; k0 < c1; k0 += kChunk) {
        const bool pf = prefetch_digis(L, k0 + kChunk, c1, pf_m, nullptr);
        digi_events(L, s_off, ci.ef, ci.el, k0, e_of);
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const bool present = k0 + j < c1;
            const bool ok = present && m[j] < M;
            if (present && !ok) atomicOr(&L.ws.event_err[e_of[j]], kErrBadDigi);
            if (!ok) continue;
            const uint64_t key = (uint64_t)e_of[j] * M + m[j];
            if (ci.use_sh)
                atomicAdd(&bins[key - ci.keybase], 1u);
            else
                atomicAdd(&L.ws.count2[key], 1u);
        }
        if (pf)
            take_prefetched(pf_m, nullptr, m, nullptr);
        else if (k0 + kChunk < c1)
            load_modules(L, k0 + kChunk, c1, m);
    }
    __syncthreads();
    // With few keys (long runs per key) the flush's atomic returns this
    // block's offset inside each key's bucket, and the scatter kernel (over
    // the same ranges) places its digis from there; with many keys the
    // counts go to count2 and the scatter hands out positions step by step,
    // so that blocks running at the same time fill neighbouring positions.
    uint32_t *boffs = L.ws.blk_off + (size_t)blockIdx.x * kHistCap;
    for (uint32_t i = threadIdx.x; i < ci.nkeys; i += kHistThreads) {
        if (sub) {
            uint32_t v = 0;
            for (uint32_t w = 0; w < kHistWarps; ++w) v += sh[w * ci.nkeys + i];
            boffs[i] = v ? atomicAdd(&L.ws.count[ci.keybase + i], v) : 0u;
        } else if (sh[i]) {
            atomicAdd(&L.ws.count2[ci.keybase + i], sh[i]);
        }
    }
}

// ---------------------------------------------------------------- scan

// Per item, count[] holds the digis of histogram blocks with few keys
// (their runs are reserved, by offset, in blk_off) and count2[] those of
// blocks with many keys (placed step by step by the scatter); the scan sets
// boff = the item's bucket start, cursor = the start of the step-by-step
// part (after every reserved run) and count = the item's total.
__global__ void __launch_bounds__(256) scan_kernel(const Launch L)
{
    __shared__ uint32_t tmp[256 / 32 + 1];
    pdl_wait();
    pdl_trigger();
    if (L.ws.ctl[1] & kErrBadOffsets) return;
    const uint32_t e = blockIdx.x, M = L.g.M;
    const uint64_t kb = (uint64_t)e * M;
    const uint32_t per = (M + 255) / 256;
    const uint32_t m0 = min(M, threadIdx.x * per), m1 = min(M, m0 + per);
    uint32_t local = 0;
    for (uint32_t m = m0; m < m1; ++m) local += L.ws.count[kb + m] + L.ws.count2[kb + m];
    uint32_t total;
    uint32_t run = block_exclusive_scan<256>(local, tmp, &total) + (uint32_t)L.offsets[e];
    for (uint32_t m = m0; m < m1; ++m) {
        const uint32_t c1 = L.ws.count[kb + m], n = c1 + L.ws.count2[kb + m];
        L.ws.boff[kb + m] = run;
        L.ws.cursor[kb + m] = run + c1;
        L.ws.count[kb + m] = n;
        run += n;
    }
}

// Shared memory of the scatter kernel (bytes).
constexpr size_t kScatterSmem = kHistCap * 4 + kChunk * (4 + 4 + 2) + (2 * kSubKeys + 2) * 4 + 16 + kChunk * (2 + 4);
static_assert(kChunk * (4 + 4 + 2) >= kHistCap * 4, "the staging area also holds the single-histogram bases");

// Scatter, persistent, over the histogram kernel's ranges: block b walks its
// range in steps of kChunk digis (one event search a block; the next step's
// words and module ids are loaded while the current step is written out,
// cp.async).  Each step ranks its digis per key in shared memory.  With few
// keys it sorts them by key in shared memory and writes each key's run with
// consecutive threads, from the block's offset inside the bucket (reserved
// by the histogram's flush), so no step needs a global atomic.  With many
// keys one global atomic per key and step hands out the positions (after
// the reserved runs), and each digi goes straight to its place; a range
// with more keys than a shared histogram holds takes one atomic per digi.
__global__ void __launch_bounds__(kHistThreads, 2) scatter_kernel(const Launch L)
{
    extern __shared__ __align__(16) uint32_t sh[];
    pdl_wait();
    pdl_trigger();
    uint32_t *cnt = sh;             // counts: per warp sub-histograms, or one histogram
    uint32_t *bas = sh + kHistCap;  // single-histogram mode: base of each key
    uint32_t *stage_w = sh + kHistCap;                                      // sub mode: block-local sorted words
    uint32_t *stage_i = stage_w + kChunk;                                   // and in-event indices
    uint16_t *stage_k = reinterpret_cast<uint16_t *>(stage_i + kChunk);     // and local keys
    uint32_t *lk = reinterpret_cast<uint32_t *>(stage_k + kChunk);          // block-local start of each key
    uint32_t *gb = lk + kSubKeys + 1;                                       // bucket position of each key's run
    __shared__ uint32_t s_ev[2];
    __shared__ uint64_t s_off[kChunkEvents + 1];
    __shared__ uint32_t s_scan[kHistThreads / 32 + 1];
    // next step's module ids and words (16-byte aligned for cp.async)
    uint16_t *pf_m = reinterpret_cast<uint16_t *>((reinterpret_cast<uintptr_t>(gb + kSubKeys + 1) + 15) & ~(uintptr_t)15);
    uint32_t *pf_w = reinterpret_cast<uint32_t *>(pf_m + kChunk);
    if (L.ws.ctl[1] & kErrBadOffsets) return;
    uint64_t c0, c1;
    block_range(L.N, blockIdx.x, gridDim.x, &c0, &c1);
    if (c0 >= c1) return;
    // the first digis are loaded before the event search, so that the two
    // latencies overlap
    uint64_t k0 = c0 + (uint64_t)threadIdx.x * kPerThread;
    uint32_t m[kPerThread], e_of[kPerThread], w[kPerThread], rank[kPerThread];
    load_modules(L, k0, c1, m);
    load_words(L, k0, c1, w);
    const ChunkInfo ci = chunk_info(L, c0, c1, s_ev, s_off);
    const uint32_t M = L.g.M, warp = threadIdx.x >> 5;
    const bool sub = ci.use_sh && ci.nkeys <= kSubKeys;
    const uint32_t nbins = sub ? ci.nkeys * kHistWarps : ci.nkeys;
    const bool off_sh = ci.el - ci.ef + 1 < kChunkEvents;
    auto event_start = [&](uint32_t e) -> uint64_t { return off_sh ? s_off[e - ci.ef] : L.offsets[e]; };
    uint32_t *bins = sub ? cnt + warp * ci.nkeys : cnt;
    // each key's next bucket position for this block: the bucket start, plus
    // the block's offset inside the bucket (from the histogram's flush),
    // advanced step by step
    if (sub) {
        const uint32_t *boffs = L.ws.blk_off + (size_t)blockIdx.x * kHistCap;
        for (uint32_t i = threadIdx.x; i < ci.nkeys; i += kHistThreads) gb[i] = L.ws.boff[ci.keybase + i] + boffs[i];
    }
    for (uint64_t s0 = c0;; s0 += kChunk, k0 += kChunk) {
        for (uint32_t i = threadIdx.x; i < nbins; i += kHistThreads) cnt[i] = 0;
        __syncthreads();
        const bool more = s0 + kChunk < c1; // another step follows
        const bool pf = more && prefetch_digis(L, k0 + kChunk, c1, pf_m, pf_w);
        digi_events(L, s_off, ci.ef, ci.el, k0, e_of);
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const bool ok = k0 + j < ci.c1 && m[j] < M;
            if (!ok) {
                m[j] = 0xFFFFFFFFu;
                continue;
            }
            const uint64_t key = (uint64_t)e_of[j] * M + m[j];
            rank[j] = ci.use_sh ? atomicAdd(&bins[key - ci.keybase], 1u) : atomicAdd(&L.ws.cursor[key], 1u);
        }
        __syncthreads();
        if (sub) {
            // Per key: per-warp counts become offsets within the key, the
            // key's block start comes from a scan over keys, and one atomic
            // reserves its run in the bucket.
            uint32_t tot = 0;
            if (threadIdx.x < ci.nkeys) {
                for (uint32_t wi = 0; wi < kHistWarps; ++wi) {
                    const uint32_t c = cnt[wi * ci.nkeys + threadIdx.x];
                    cnt[wi * ci.nkeys + threadIdx.x] = tot;
                    tot += c;
                }
            }
            uint32_t total;
            const uint32_t start = block_exclusive_scan<kHistThreads>(tot, s_scan, &total);
            uint32_t kg = 0;
            if (threadIdx.x < ci.nkeys) {
                lk[threadIdx.x] = start;
                kg = gb[threadIdx.x];
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                if (m[j] == 0xFFFFFFFFu) continue;
                const uint32_t key = (uint32_t)((uint64_t)e_of[j] * M + m[j] - ci.keybase);
                const uint32_t p = lk[key] + cnt[warp * ci.nkeys + key] + rank[j];
                stage_w[p] = w[j];
                stage_i[p] = (uint32_t)(k0 + j - event_start(e_of[j]));
                stage_k[p] = (uint16_t)key;
            }
            __syncthreads();
            for (uint32_t p = threadIdx.x; p < total; p += kHistThreads) {
                const uint32_t key = stage_k[p];
                const uint32_t g = gb[key] + (p - lk[key]);
                L.ws.bucket_w[g] = stage_w[p];
                L.ws.bucket_i[g] = stage_i[p];
            }
            __syncthreads();
            if (threadIdx.x < ci.nkeys) gb[threadIdx.x] = kg + tot; // the key's cursor after this step
        } else {
            for (uint32_t i = threadIdx.x; i < ci.nkeys; i += kHistThreads) {
                const uint32_t v = cnt[i];
                if (v) bas[i] = atomicAdd(&L.ws.cursor[ci.keybase + i], v);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                if (m[j] == 0xFFFFFFFFu) continue;
                const uint64_t key = (uint64_t)e_of[j] * M + m[j];
                const uint32_t p = ci.use_sh ? bas[key - ci.keybase] + rank[j] : rank[j];
                L.ws.bucket_w[p] = w[j];
                L.ws.bucket_i[p] = (uint32_t)(k0 + j - event_start(e_of[j]));
            }
        }
        __syncthreads();
        if (!more) break;
        if (pf) {
            take_prefetched(pf_m, pf_w, m, w);
        } else {
            load_modules(L, k0 + kChunk, c1, m);
            load_words(L, k0 + kChunk, c1, w);
        }
    }
}

// ---------------------------------------------------------------- clustering

// After the unions, a root's parent entry holds kMark | its linear pixel index.
constexpr uint32_t kMark = 0x80000000u;
// Moments accumulate in 32 bits relative to the root pixel (|drow| < 256,
// |dcol| < 512): they cannot overflow while Q <= INT32_MAX / 512.  Items with
// a heavier cluster recompute the moments in 64 bits.
constexpr int32_t kQSafe32 = 0x7FFFFFFF / 512;

// Per-item arrays of the block tier: shared memory, or global scratch for
// items beyond the shared-memory capacity.
struct Tile {
    uint32_t *parent;          // union-find parent of a slot; kMark | lin for roots after marking
    int32_t *q;                // root: charge Q
    uint32_t *np;              // root: pixel count
    int2 *m;                   // root: sum q*row, sum q*col
    unsigned long long *exact; // root: the same two moments in 64 bits (heavy clusters only)
};

struct BlockShared {
    uint32_t flag;
    uint32_t heavy;
    uint32_t big_off;
    uint32_t scan_tmp[kCCThreads / 32 + 1];
};

// Find with path splitting (each visited node is re-pointed to its
// grandparent).  Parent entries only ever point to a smaller slot of the same
// tree, so a plain store that races with a link elsewhere leaves a valid
// ancestor behind; a link that loses such a race is retried by its union.
__device__ __forceinline__ uint32_t uf_find_halving(uint32_t *parent, uint32_t x)
{
    volatile uint32_t *p = parent;
    uint32_t y = p[x];
    while (y != x) {
        const uint32_t z = p[y];
        if (z != y) p[x] = z;
        x = y;
        y = z;
    }
    return x;
}

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// Lock-free union of the trees of a and b, for all 32 lanes of a warp in
// lockstep (lanes with b == kNoSlot idle; the whole warp must call it): the
// larger root is linked under the smaller with atomicMin, and a lost race
// re-runs with the new parent.
__device__ __forceinline__ void warp_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    bool done = b == kNoSlot;
    while (__any_sync(kFull, !done)) {
        if (!done) {
            a = uf_find_halving(parent, a);
            b = uf_find_halving(parent, b);
            if (a == b) {
                done = true;
            } else {
                if (a < b) {
                    const uint32_t t = a;
                    a = b;
                    b = t;
                }
                const uint32_t old = atomicMin(&parent[a], b);
                if (old == a)
                    done = true;
                else
                    a = old;
            }
        }
    }
}

__device__ __forceinline__ uint32_t rank_of(const uint32_t *sbits, const uint32_t *spre, uint32_t lin)
{
    return spre[lin >> 5] + __popc(sbits[lin >> 5] & ((1u << (lin & 31)) - 1u));
}

__device__ __forceinline__ bool has_bit(const uint32_t *bits, uint32_t lin)
{
    return (bits[lin >> 5] >> (lin & 31)) & 1u;
}

// Number of surviving pixels immediately to the left of pixel lin in its row
// (the pixel's offset in its horizontal run), read from the survivor bitmap
// 32 bits at a time.
__device__ __forceinline__ uint32_t run_offset(const uint32_t *sbits, uint32_t lin, uint32_t row0)
{
    uint32_t off = 0, pos = lin;
    while (pos > row0) {
        const uint32_t bt = (pos - 1) & 31;
        const uint32_t x = ~sbits[(pos - 1) >> 5] << (31 - bt); // bit pos-1 moved to the top
        const uint32_t ones = x ? (uint32_t)__clz(x) : bt + 1;  // set bits from pos-1 downwards
        const uint32_t take = min(ones, pos - row0);
        off += take;
        pos -= take;
        if (take < bt + 1) break;
    }
    return off;
}

// One item of at most 32 * K digis, clustered by one warp in registers:
// digi j is held by lane j % 32 in register slot j / 32.  Adjacency is a bit
// mask over the item's digis per held digi; the cluster id (the smallest
// linear index) spreads over the adjacency by min-propagation; cluster sums
// run over the digis sharing an id.  Returns the number of kept clusters
// (all lanes).
template <int K>
__device__ uint32_t warp_item(const Launch &L, const ItemCtx &it)
{
    using Mask = typename std::conditional<K == 1, uint32_t, unsigned long long>::type;
    const uint32_t lane = threadIdx.x & 31;
    const int R = (int)L.g.R, C = (int)L.g.C;
    const uint32_t n = it.n;
    int r[K], c[K], q[K], lin[K], lab[K];
    uint32_t idx[K];
    bool have[K], surv[K];
    Mask adj[K];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t j = lane + 32 * k;
        have[k] = j < n;
        const uint32_t w = have[k] ? L.ws.bucket_w[it.b + j] : 0u;
        idx[k] = have[k] ? L.ws.bucket_i[it.b + j] : 0u;
        r[k] = (int)(w & 0xFFu);
        c[k] = (int)((w >> 8) & 0x1FFu);
        const int adc = (int)((w >> 17) & 0xFFu);
        if (have[k] && (r[k] >= R || c[k] >= C || adc == 0 || (w >> 25) != 0)) bad = true;
        lin[k] = have[k] ? r[k] * C + c[k] : -1 - (int)j;
        q[k] = adc * it.gain - it.ped;
        surv[k] = have[k] && q[k] >= L.g.pixel_thr;
        adj[k] = 0;
    }
    if (__any_sync(kFull, bad)) {
        if (lane == 0) atomicOr(it.err_e, kErrBadDigi);
        return 0;
    }
    Mask smask = (Mask)__ballot_sync(kFull, surv[0]);
    if constexpr (K == 2) smask |= (Mask)__ballot_sync(kFull, surv[1]) << 32;
    bool dup = false;
    for (uint32_t j = 0; j < n; ++j) {
        const uint32_t sl = j & 31, sk = j >> 5;
        const int lj = __shfl_sync(kFull, (K == 2 && sk) ? lin[K - 1] : lin[0], sl);
        const int rj = __shfl_sync(kFull, (K == 2 && sk) ? r[K - 1] : r[0], sl);
        const int cj = __shfl_sync(kFull, (K == 2 && sk) ? c[K - 1] : c[0], sl);
        const bool sj = (smask >> j) & 1u;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t me = lane + 32 * k;
            if (me == j) continue;
            if (have[k] && lj == lin[k]) dup = true;
            if (surv[k] && sj && abs(rj - r[k]) <= 1 && abs(cj - c[k]) <= 1) adj[k] |= (Mask)1 << j;
        }
    }
    if (__any_sync(kFull, dup)) {
        if (lane == 0) atomicOr(it.err_e, kErrDup);
        return 0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) lab[k] = surv[k] ? lin[k] : INT_MAX;
    for (uint32_t round = 0; round < n; ++round) {
        int nl[K];
#pragma unroll
        for (int k = 0; k < K; ++k) nl[k] = lab[k];
        for (uint32_t j = 0; j < n; ++j) {
            const int lj = __shfl_sync(kFull, (K == 2 && (j >> 5)) ? lab[K - 1] : lab[0], j & 31);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if ((adj[k] >> j) & 1u) nl[k] = min(nl[k], lj);
        }
        bool changed = false;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            changed |= nl[k] != lab[k];
            lab[k] = nl[k];
        }
        if (!__any_sync(kFull, changed)) break;
    }
    // sums over the digis of each held digi's cluster, about the cluster's id pixel
    // (|sums| < 64 * 32263 * 63 < 2^31)
    int Q[K], np[K], Sr[K], Sc[K], rr[K], rc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        Q[k] = np[k] = Sr[k] = Sc[k] = 0;
        rr[k] = surv[k] ? lab[k] / C : 0;
        rc[k] = surv[k] ? lab[k] - rr[k] * C : 0;
    }
    for (uint32_t j = 0; j < n; ++j) {
        const uint32_t sl = j & 31;
        const bool hi = K == 2 && (j >> 5);
        const int labj = __shfl_sync(kFull, hi ? lab[K - 1] : lab[0], sl);
        const int qj = __shfl_sync(kFull, hi ? q[K - 1] : q[0], sl);
        const int rj = __shfl_sync(kFull, hi ? r[K - 1] : r[0], sl);
        const int cj = __shfl_sync(kFull, hi ? c[K - 1] : c[0], sl);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (surv[k] && labj == lab[k]) {
                Q[k] += qj;
                ++np[k];
                Sr[k] += qj * (rj - rr[k]);
                Sc[k] += qj * (cj - rc[k]);
            }
        }
    }
    bool kept[K], lead[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        lead[k] = surv[k] && lin[k] == lab[k];
        kept[k] = surv[k] && Q[k] >= L.g.cluster_thr;
    }
    Mask kl = (Mask)__ballot_sync(kFull, lead[0] && kept[0]);
    if constexpr (K == 2) kl |= (Mask)__ballot_sync(kFull, lead[K - 1] && kept[K - 1]) << 32;
    uint32_t ord[K];
#pragma unroll
    for (int k = 0; k < K; ++k) ord[k] = 0;
    for (uint32_t j = 0; j < n; ++j) {
        const int lj = __shfl_sync(kFull, (K == 2 && (j >> 5)) ? lin[K - 1] : lin[0], j & 31);
        if ((kl >> j) & 1u) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (lj < lab[k]) ++ord[k]; // the rank of the digi's cluster (lab = lin for its lead)
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (lead[k] && kept[k]) {
            L.ws.staging.put(it.b + ord[k], lab[k], Q[k], np[k], centroid(rr[k], Sr[k], Q[k]),
                             centroid(rc[k], Sc[k], Q[k]));
        }
        if (it.label_e && have[k]) it.label_e[idx[k]] = !surv[k] ? -1 : (kept[k] ? lab[k] : -2);
        if (it.label16_e && have[k])
            it.label16_e[idx[k]] = !surv[k] ? kLab16Below : (kept[k] ? (uint16_t)ord[k] : kLab16Dropped);
    }
    if constexpr (K == 1)
        return __popc(kl);
    else
        return __popcll(kl);
}

// Apply f(k, word) to every digi of the item owned by this thread.  The
// loop is kept rolled so that the block tier stays small in the instruction
// cache; the item's bucket (read-only here) is re-read through L1.
template <class F>
__device__ __forceinline__ void for_digis(const uint32_t *bw, uint32_t n, F &&f)
{
#pragma unroll 1
    for (uint32_t k = threadIdx.x; k < n; k += kCCThreads) f(k, __ldg(bw + k));
}

// Centroid coordinate sum / Q from an exact, non-negative moment: one float
// division when both are exact in float (the correctly rounded quotient),
// else integer quotient plus the remainder fraction, so the float result is
// within a few ulps whatever the magnitude.
__device__ __forceinline__ float centroid_abs(long long sum, int32_t Q)
{
    if (sum < 16777216LL && Q < 16777216) return (float)sum / (float)Q;
    if (sum < 0x80000000LL) {
        const uint32_t su = (uint32_t)sum, qu = (uint32_t)Q;
        const uint32_t qt = su / qu;
        return (float)qt + (float)(su - qt * qu) / (float)Q;
    }
    const long long qt = sum / Q;
    return (float)qt + (float)(sum - qt * Q) / (float)Q;
}

// One item clustered by the whole block (see the file comment).  kBig: the
// tile lives in global scratch instead of shared memory.  Returns the number
// of kept clusters (uniform over the block).
template <bool kBig>
__device__ uint32_t block_item(const Launch &L, const ItemCtx &it, uint32_t *abits, uint32_t *sbits, uint32_t *spre,
                               const Tile &t, BlockShared &bs)
{
    const uint32_t R = L.g.R, C = L.g.C, nwords = (R * C + 31) >> 5;
    const int32_t thr = L.g.pixel_thr, cthr = L.g.cluster_thr;
    const uint32_t tid = threadIdx.x, n = it.n, lane = tid & 31, warp = tid >> 5;
    const uint32_t *bw = L.ws.bucket_w + it.b;
    const uint32_t *bi = L.ws.bucket_i + it.b;
    const int32_t gain = it.gain, ped = it.ped;
    auto lin_of = [C](uint32_t w) { return (w & 0xFFu) * C + ((w >> 8) & 0x1FFu); };
    auto charge = [gain, ped](uint32_t w) { return (int32_t)((w >> 17) & 0xFFu) * gain - ped; };

    for (uint32_t i = tid; i < nwords; i += kCCThreads) {
        abits[i] = 0;
        sbits[i] = 0;
    }
    if (tid == 0) {
        bs.flag = 0;
        bs.heavy = 0;
    }
    __syncthreads();

    // occupancy and survivor bitmaps; validation and duplicate detection
    {   // the item's words are loaded four per thread at a time, so that
        // their latencies overlap instead of adding up
        auto body = [&](uint32_t w) {
            const uint32_t r = w & 0xFFu, c = (w >> 8) & 0x1FFu, adc = (w >> 17) & 0xFFu;
            if (r >= R || c >= C || adc == 0 || (w >> 25) != 0) {
                atomicOr(&bs.flag, kErrBadDigi);
                return;
            }
            const uint32_t lin = r * C + c, bit = 1u << (lin & 31);
            if (atomicOr(&abits[lin >> 5], bit) & bit) atomicOr(&bs.flag, kErrDup);
            if (charge(w) >= thr) atomicOr(&sbits[lin >> 5], bit);
        };
#pragma unroll 1
        for (uint32_t k0 = tid; k0 < n; k0 += 4 * kCCThreads) {
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + u * kCCThreads;
                wv[u] = k < n ? __ldg(bw + k) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u * kCCThreads < n) body(wv[u]);
        }
    }
    __syncthreads();
    const uint32_t flag = bs.flag;
    if (flag) {
        if (tid == 0) atomicOr(it.err_e, flag);
        __syncthreads();
        return 0;
    }

    // exclusive prefix popcount of the survivor bitmap -> dense slots
    const uint32_t per = (nwords + kCCThreads - 1) / kCCThreads;
    const uint32_t w0 = min(nwords, tid * per), w1 = min(nwords, w0 + per);
    uint32_t local = 0;
    for (uint32_t i = w0; i < w1; ++i) local += __popc(sbits[i]);
    uint32_t S;
    uint32_t run = block_exclusive_scan<kCCThreads>(local, bs.scan_tmp, &S);
    for (uint32_t i = w0; i < w1; ++i) {
        spre[i] = run;
        run += __popc(sbits[i]);
    }
    // the per-root accumulators of every slot, cleared in slot order
    for (uint32_t s = tid; s < S; s += kCCThreads) {
        t.q[s] = 0;
        t.np[s] = 0;
        t.m[s] = make_int2(0, 0);
    }
    __syncthreads();
    // every surviving pixel starts in its horizontal run: parent = the run's
    // first pixel, whose slot is the pixel's slot minus its run offset
    for_digis(bw, n, [&](uint32_t, uint32_t w) {
        const uint32_t r = w & 0xFFu, lin = lin_of(w);
        if (!has_bit(sbits, lin)) return;
        const uint32_t s = rank_of(sbits, spre, lin);
        t.parent[s] = s - run_offset(sbits, lin, r * C);
    });
    __syncthreads();

    // Join runs of adjacent rows.  For a pixel p whose upper neighbour U
    // survives, one union per maximal stretch of such pixels (at p = the run
    // head, or where the upper-left pixel does not survive) joins p's run to
    // U's run; a run head whose U is empty checks its upper-left pixel, a run
    // tail whose U is empty its upper-right one.  Every 8-adjacency between
    // two runs passes through one of these.  The lanes of a warp walk the
    // item in step, two digis a lane (64 consecutive digis a warp), and union
    // the pairs of both in one lockstep round.
    for (uint32_t k0 = 2 * (tid - lane); k0 < n; k0 += 2 * kCCThreads) {
        uint32_t s[2] = {0u, 0u}, nb0[2] = {kNoSlot, kNoSlot}, nb1[2] = {kNoSlot, kNoSlot};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t k = k0 + 32 * h + lane;
            if (k < n) {
                const uint32_t w = __ldg(bw + k);
                const uint32_t r = w & 0xFFu, c = (w >> 8) & 0x1FFu, lin = r * C + c;
                if (r > 0 && has_bit(sbits, lin)) {
                    s[h] = rank_of(sbits, spre, lin);
                    const uint32_t up = lin - C;
                    const bool head = c == 0 || !has_bit(sbits, lin - 1);
                    const bool tail = c + 1 == C || !has_bit(sbits, lin + 1);
                    const bool ul = c > 0 && has_bit(sbits, up - 1);
                    if (has_bit(sbits, up)) {
                        if (head || !ul) nb0[h] = rank_of(sbits, spre, up);
                    } else {
                        if (head && ul) nb0[h] = rank_of(sbits, spre, up - 1);
                        if (tail && c + 1 < C && has_bit(sbits, up + 1)) nb1[h] = rank_of(sbits, spre, up + 1);
                    }
                }
            }
        }
        // gather the warp's union pairs onto consecutive lanes, then union them
        const uint32_t m00 = __ballot_sync(kFull, nb0[0] != kNoSlot), m01 = __ballot_sync(kFull, nb1[0] != kNoSlot);
        const uint32_t m10 = __ballot_sync(kFull, nb0[1] != kNoSlot), m11 = __ballot_sync(kFull, nb1[1] != kNoSlot);
        const uint32_t e0 = __popc(m00), e1 = e0 + __popc(m01), e2 = e1 + __popc(m10), total = e2 + __popc(m11);
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t p = base + lane;
            const uint32_t seg = p < e0 ? 0u : p < e1 ? 1u : p < e2 ? 2u : 3u;
            const uint32_t mask = seg == 0 ? m00 : seg == 1 ? m01 : seg == 2 ? m10 : m11;
            const uint32_t first = seg == 0 ? 0u : seg == 1 ? e0 : seg == 2 ? e1 : e2;
            const uint32_t src = p < total ? __fns(mask, 0, (int)(p - first) + 1) : 0u;
            const uint32_t a0 = __shfl_sync(kFull, s[0], src), a1 = __shfl_sync(kFull, s[1], src);
            const uint32_t b00 = __shfl_sync(kFull, nb0[0], src), b01 = __shfl_sync(kFull, nb1[0], src);
            const uint32_t b10 = __shfl_sync(kFull, nb0[1], src), b11 = __shfl_sync(kFull, nb1[1], src);
            const uint32_t a = seg < 2 ? a0 : a1;
            const uint32_t bb = seg == 0 ? b00 : seg == 1 ? b01 : seg == 2 ? b10 : b11;
            warp_union(t.parent, a, p < total ? bb : kNoSlot);
        }
    }
    __syncthreads();

    // Charge, size and absolute moments per root.  Each pixel walks to its
    // root (the smallest slot); a root's own pixel marks it with kMark | its
    // linear index (the cluster id), the others compress to it.  Moments
    // accumulate in 32 bits; a cluster heavier than kQSafe32 (possible
    // overflow) sends the item through the exact 64-bit pass below.
    for_digis(bw, n, [&](uint32_t, uint32_t w) {
        const uint32_t r = w & 0xFFu, c = (w >> 8) & 0x1FFu, lin = r * C + c;
        if (!has_bit(sbits, lin)) return;
        const uint32_t s = rank_of(sbits, spre, lin);
        const volatile uint32_t *vp = t.parent;
        uint32_t x = s, p = vp[s];
        while (p != x && !(p & kMark)) {
            x = p;
            p = vp[x];
        }
        t.parent[s] = x == s ? (kMark | lin) : x;
        const int32_t q = charge(w);
        const int32_t old = atomicAdd(&t.q[x], q);
        if (old + q > kQSafe32) bs.heavy = 1;
        atomicAdd(&t.np[x], 1u);
        atomicAdd(&t.m[x].x, q * (int32_t)r);
        atomicAdd(&t.m[x].y, q * (int32_t)c);
    });
    __syncthreads();
    const bool heavy = bs.heavy != 0;
    if (heavy) {
        for (uint32_t s = tid; s < S; s += kCCThreads) {
            t.exact[2 * s] = 0;
            t.exact[2 * s + 1] = 0;
        }
        __syncthreads();
        for_digis(bw, n, [&](uint32_t, uint32_t w) {
            const uint32_t r = w & 0xFFu, c = (w >> 8) & 0x1FFu, lin = r * C + c;
            if (!has_bit(sbits, lin)) return;
            const uint32_t s = rank_of(sbits, spre, lin);
            const uint32_t p = t.parent[s];
            const uint32_t x = (p & kMark) ? s : p;
            const long long q = charge(w);
            atomicAdd(&t.exact[2 * x], (unsigned long long)(q * (long long)r));
            atomicAdd(&t.exact[2 * x + 1], (unsigned long long)(q * (long long)c));
        });
        __syncthreads();
    }

    if (it.label_e) { // loads of four digis (word and index) issued together, as for the bitmaps
        auto label_of = [&](uint32_t w) -> int32_t {
            const uint32_t lin = lin_of(w);
            int32_t lab = -1;
            if (has_bit(sbits, lin)) {
                const uint32_t s = rank_of(sbits, spre, lin);
                const uint32_t p = t.parent[s];
                const uint32_t x = (p & kMark) ? s : p;
                const uint32_t px = (p & kMark) ? p : t.parent[x];
                lab = t.q[x] >= cthr ? (int32_t)(px & ~kMark) : -2;
            }
            return lab;
        };
#pragma unroll 1
        for (uint32_t k0 = tid; k0 < n; k0 += 4 * kCCThreads) {
            uint32_t wv[4], iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + u * kCCThreads;
                const bool in = k < n;
                wv[u] = in ? __ldg(bw + k) : 0u;
                iv[u] = in ? __ldg(bi + k) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u * kCCThreads < n) it.label_e[iv[u]] = label_of(wv[u]);
        }
    }

    // Kept roots in slot order (= id order): every warp takes a contiguous
    // range of 32-slot chunks and ballots them (into abits, free since the
    // bitmaps were built), one scan of the warp totals gives each warp's
    // first ordinal, and the warp walks its chunks again in order.
    const uint32_t chunks = (S + 31) >> 5;
    constexpr uint32_t kWarps = kCCThreads / 32;
    const uint32_t cpw = (chunks + kWarps - 1) / kWarps;
    const uint32_t wc0 = min(chunks, warp * cpw), wc1 = min(chunks, wc0 + cpw);
    uint32_t wrun = 0;
    for (uint32_t ch = wc0; ch < wc1; ++ch) {
        const uint32_t s = (ch << 5) + lane;
        const bool kept = s < S && (t.parent[s] & kMark) && t.q[s] >= cthr;
        const uint32_t bal = __ballot_sync(kFull, kept);
        if (lane == 0) abits[ch] = bal;
        wrun += __popc(bal);
    }
    if (lane == 0) bs.scan_tmp[warp] = wrun;
    __syncthreads();
    uint32_t K, woff;
    {
        const uint32_t wt = lane < kWarps ? bs.scan_tmp[lane] : 0u;
        uint32_t ws = wt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, ws, o);
            if ((int)lane >= o) ws += y;
        }
        K = __shfl_sync(kFull, ws, kWarps - 1);
        woff = __shfl_sync(kFull, ws - wt, warp);
    }
    auto stage = [&](uint32_t s, uint32_t ord) {
        const int32_t Q = t.q[s];
        long long mr, mc;
        if (heavy) {
            mr = (long long)t.exact[2 * s];
            mc = (long long)t.exact[2 * s + 1];
        } else {
            const int2 mm = t.m[s];
            mr = mm.x;
            mc = mm.y;
        }
        L.ws.staging.put(it.b + ord, (int32_t)(t.parent[s] & ~kMark), Q, (int32_t)t.np[s], centroid_abs(mr, Q),
                         centroid_abs(mc, Q));
        if (it.label16_e) t.np[s] = ord; // read back by the compact labels
    };
    // (the compact labels look digis up in the survivor bitmap afterwards, so
    // with them the kept roots are not compacted into its space)
    if (S <= 2 * nwords && !it.label16_e) {
        // compact the kept roots (their slots, by ordinal, into the survivor
        // bitmap's space, free now) so that every lane stages a cluster
        uint16_t *kslot = reinterpret_cast<uint16_t *>(sbits);
        uint32_t run = woff;
        for (uint32_t ch = wc0; ch < wc1; ++ch) {
            const uint32_t bal = abits[ch];
            if ((bal >> lane) & 1u) kslot[run + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)((ch << 5) + lane);
            run += __popc(bal);
        }
        __syncthreads();
        for (uint32_t o = tid; o < K; o += kCCThreads) stage(kslot[o], o);
    } else {
        uint32_t run = woff;
        for (uint32_t ch = wc0; ch < wc1; ++ch) {
            const uint32_t bal = abits[ch];
            if ((bal >> lane) & 1u) stage((ch << 5) + lane, run + __popc(bal & ((1u << lane) - 1u)));
            run += __popc(bal);
        }
    }
    if (it.label16_e) { // compact labels: the ordinal of the digi's root, kept in t.np by the staging
        __syncthreads();
#pragma unroll 1
        for (uint32_t k0 = tid; k0 < n; k0 += 4 * kCCThreads) {
            uint32_t wv[4], iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t k = k0 + u * kCCThreads;
                const bool in = k < n;
                wv[u] = in ? __ldg(bw + k) : 0u;
                iv[u] = in ? __ldg(bi + k) : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k0 + u * kCCThreads >= n) continue;
                const uint32_t lin = lin_of(wv[u]);
                uint16_t v = kLab16Below;
                if (has_bit(sbits, lin)) {
                    const uint32_t sl = rank_of(sbits, spre, lin);
                    const uint32_t p = t.parent[sl];
                    const uint32_t x = (p & kMark) ? sl : p;
                    v = t.q[x] >= cthr ? (uint16_t)t.np[x] : kLab16Dropped;
                }
                it.label16_e[iv[u]] = v;
            }
        }
    }
    return K;
}

// Zero nw words at p (16-byte stores where p is 16-byte aligned).
__device__ __forceinline__ void clear_words(uint32_t *p, uint32_t nw)
{
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        uint4 *v = reinterpret_cast<uint4 *>(p);
        for (uint32_t i = threadIdx.x; i < nw / 4; i += kCCThreads) v[i] = make_uint4(0, 0, 0, 0);
        done = nw & ~3u;
    }
    for (uint32_t i = done + threadIdx.x; i < nw; i += kCCThreads) p[i] = 0;
}

// Slot of the first pixel of the horizontal run holding surviving pixel lin,
// whose row starts at linear index row0; word = sbits[lin >> 5] and base =
// spre[lin >> 5] are passed in (already loaded by the caller).  The run
// starts one past the nearest non-surviving pixel to the left of lin, or at
// the row start.
__device__ __noinline__ uint32_t run_head_slot_far(const uint32_t *sbits, const uint32_t *spre, uint32_t wi,
                                                   uint32_t row0);
__device__ __forceinline__ uint32_t run_head_slot(const uint32_t *sbits, const uint32_t *spre, uint32_t lin,
                                                  uint32_t row0, uint32_t word, uint32_t base)
{
    uint32_t wi = lin >> 5;
    const uint32_t b = lin & 31;
    uint32_t lo = row0 > (wi << 5) ? row0 - (wi << 5) : 0u; // first bit of the row in this word
    uint32_t z = ~word & ((1u << b) - 1u) & ~((1u << lo) - 1u);
    if (z) return base + __popc(word & ((1u << (32 - __clz(z))) - 1u));
    if ((wi << 5) + lo == row0) return base + __popc(word & ((1u << lo) - 1u));
    return run_head_slot_far(sbits, spre, wi, row0);
}

__device__ __noinline__ uint32_t run_head_slot_far(const uint32_t *sbits, const uint32_t *spre, uint32_t wi,
                                                   uint32_t row0)
{
    uint32_t word, lo, z;
    for (;;) { // the run continues into the previous word (rare)
        --wi;
        word = sbits[wi];
        lo = row0 > (wi << 5) ? row0 - (wi << 5) : 0u;
        z = ~word & ~((1u << lo) - 1u);
        if (z) {
            const uint32_t hb = 32 - __clz(z);
            return hb == 32 ? spre[wi + 1] : spre[wi] + __popc(word & ((1u << hb) - 1u));
        }
        if ((wi << 5) + lo == row0) return spre[wi] + __popc(word & ((1u << lo) - 1u));
    }
}

// Lock-free union of the trees of a and b by one thread: the larger root is
// linked under the smaller with atomicMin; a link that finds its root already
// linked elsewhere retries from the new parent.
__device__ __noinline__ void uf_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    for (;;) {
        a = uf_find_halving(parent, a);
        b = uf_find_halving(parent, b);
        if (a == b) return;
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicMin(&parent[a], b);
        if (old == a) return;
        a = old;
    }
}

// Root reached from slot y (its parent not yet known to be the root).
__device__ __noinline__ uint32_t root_walk_far(const uint32_t *parent, uint32_t y)
{
    const volatile uint32_t *vp = parent;
    uint32_t p = vp[y];
    while (p != y && !(p & kMark)) {
        y = p;
        p = vp[y];
    }
    return y;
}

// Write kept cluster s (a root of tile t) to the item's staging slot ord.
__device__ __forceinline__ void stage_cluster(const Launch &L, const ItemCtx &it, const Tile &t, bool heavy,
                                              uint32_t s, uint32_t ord)
{
    const int32_t Q = t.q[s];
    long long mr, mc;
    if (heavy) {
        mr = (long long)t.exact[2 * s];
        mc = (long long)t.exact[2 * s + 1];
    } else {
        const int2 mm = t.m[s];
        mr = mm.x;
        mc = mm.y;
    }
    L.ws.staging.put(it.b + ord, (int32_t)(t.parent[s] & ~kMark), Q, (int32_t)t.np[s], centroid_abs(mr, Q),
                     centroid_abs(mc, Q));
    if (it.label16_e) t.np[s] = ord; // read back by the compact labels
}

// Register tier of the block: items of at most kD * kCCThreads digis (and at
// most the shared-memory tile).  Thread t holds digis t, t + kCCThreads, ...
// of the item in registers from the first load to the labels, with its
// slot (then its root) beside each word, so the bucket is read once per
// digi (words) plus once (in-event indices, for the labels).
//
// Union-find runs on run heads only: every surviving pixel points at the
// first pixel of its horizontal run (found from the survivor bitmap word by
// a leading-zero count), and only heads are linked across rows, so finds
// never visit another run's inner pixels.  Phases, one barrier each:
//   1 occupancy + survivor bits (duplicates and invalid words flagged)
//   2 prefix popcount -> slots; parent[s] = s; occupancy bitmap cleared
//   3 slot and run head of every survivor; accumulators cleared at heads;
//     one union per stretch of contact with the row above
//   4 root of every survivor (roots marked with their linear index);
//     charge, size and moments accumulated per root; survivor bitmap cleared
//   5 labels; kept roots balloted per 32-slot chunk
//   6 kept roots compacted in slot (= id) order, then staged
// Both bitmaps are left zeroed for the next item.
template <int kD, bool kCompact>
__device__ uint32_t block_item_reg(const Launch &L, const ItemCtx &it, uint32_t *abits, uint32_t *sbits,
                                   uint32_t *spre, const Tile &t, BlockShared &bs)
{
    const uint32_t R = L.g.R, C = L.g.C, nwords = (R * C + 31) >> 5;
    const int32_t thr = L.g.pixel_thr, cthr = L.g.cluster_thr;
    const uint32_t tid = threadIdx.x, n = it.n, lane = tid & 31, warp = tid >> 5;
    const uint32_t *bw = L.ws.bucket_w + it.b;
    const int32_t gain = it.gain, ped = it.ped;

    // 1: the thread's words, then their bits
    uint32_t w[kD], s[kD];
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        const uint32_t j = tid + k * kCCThreads;
        w[k] = j < n ? __ldg(bw + j) : 0u;
    }
    uint32_t err = 0;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        s[k] = kNoSlot;
        if (tid + k * kCCThreads < n) {
            const uint32_t x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu, adc = (x >> 17) & 0xFFu;
            if (r >= R || c >= C || adc == 0 || (x >> 25) != 0) {
                err |= kErrBadDigi;
            } else {
                const uint32_t lin = r * C + c, bit = 1u << (lin & 31);
                if (atomicOr(&abits[lin >> 5], bit) & bit) err |= kErrDup;
                if ((int32_t)adc * gain - ped >= thr) {
                    atomicOr(&sbits[lin >> 5], bit);
                    s[k] = 0;
                }
            }
        }
    }
    err = __reduce_or_sync(kFull, err);
    if (err && lane == 0) atomicOr(&bs.flag, err);
    __syncthreads();
    const uint32_t flag = bs.flag;
    if (flag) {
        if (tid == 0) atomicOr(it.err_e, flag);
        clear_words(abits, nwords);
        clear_words(sbits, nwords);
        __syncthreads();
        if (tid == 0) bs.flag = 0;
        return 0;
    }

    // 2: exclusive prefix popcount of the survivor bitmap -> dense slots
    const uint32_t per = (nwords + kCCThreads - 1) / kCCThreads;
    const uint32_t w0 = min(nwords, tid * per), w1 = min(nwords, w0 + per);
    uint32_t local = 0;
    for (uint32_t i = w0; i < w1; ++i) local += __popc(sbits[i]);
    uint32_t S;
    uint32_t run = block_exclusive_scan<kCCThreads>(local, bs.scan_tmp, &S);
    for (uint32_t i = w0; i < w1; ++i) {
        spre[i] = run;
        run += __popc(sbits[i]);
    }
    for (uint32_t i = tid; i < S; i += kCCThreads) t.parent[i] = i;
    __syncthreads();

    // 3: slots, run heads, and the unions with the row above.  For a pixel p
    // whose upper neighbour U survives, one union per maximal stretch of such
    // pixels (at the run head, or where the upper-left pixel does not
    // survive) joins p's run to U's run; a run head whose U is empty checks
    // its upper-left pixel, a run tail whose U is empty its upper-right one.
    // Every 8-adjacency between two runs passes through one of these.
    // union pairs (head slot | target head slot << 16) go to a per-warp list in
    // the occupancy bitmap (free since phase 2); a full list unions in place
    const uint32_t seg = nwords / (kCCThreads / 32);
    uint32_t *plist = abits + warp * seg;
    uint32_t pcount = 0;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if (k * kCCThreads >= n) break;
        uint32_t h = 0, th1 = kNoSlot, th2 = kNoSlot;
        if (s[k] != kNoSlot) {
            const uint32_t x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu, lin = r * C + c;
            const uint32_t wi = lin >> 5, b = lin & 31;
            const uint32_t word = sbits[wi], base = spre[wi];
            const uint32_t slot = base + __popc(word & ((1u << b) - 1u));
            h = run_head_slot(sbits, spre, lin, r * C, word, base);
            s[k] = slot;
            if (h != slot) {
                t.parent[slot] = h;
            } else {
                t.q[slot] = 0;
                t.np[slot] = 0;
                t.m[slot] = make_int2(0, 0);
            }
            if (r > 0) {
                const uint32_t up = lin - C, wu = up >> 5, bu = up & 31;
                const uint32_t uword = sbits[wu];
                const bool U = (uword >> bu) & 1u;
                const bool UL = c > 0 && (bu > 0 ? ((uword >> (bu - 1)) & 1u) : (sbits[wu - 1] >> 31));
                const bool UR = c + 1 < C && (bu < 31 ? ((uword >> (bu + 1)) & 1u) : (sbits[wu + 1] & 1u));
                const bool head = h == slot;
                const bool tail = c + 1 == C || !(b < 31 ? ((word >> (b + 1)) & 1u) : (sbits[wi + 1] & 1u));
                uint32_t t1 = kNoSlot, t2 = kNoSlot;
                if (U) {
                    if (head || !UL) t1 = up;
                } else {
                    if (head && UL) t1 = up - 1;
                    if (tail && UR) t2 = up + 1;
                }
                const uint32_t row0u = (r - 1) * C;
                if (t1 != kNoSlot) {
                    const uint32_t tw = t1 >> 5;
                    th1 = run_head_slot(sbits, spre, t1, row0u, sbits[tw], spre[tw]);
                }
                if (t2 != kNoSlot) {
                    const uint32_t tw = t2 >> 5;
                    th2 = run_head_slot(sbits, spre, t2, row0u, sbits[tw], spre[tw]);
                }
            }
        }
        const uint32_t m1 = __ballot_sync(kFull, th1 != kNoSlot), m2 = __ballot_sync(kFull, th2 != kNoSlot);
        const uint32_t p1 = pcount + __popc(m1 & lt), p2 = pcount + __popc(m1) + __popc(m2 & lt);
        if (th1 != kNoSlot) {
            if (p1 < seg) plist[p1] = h | (th1 << 16);
            else uf_union(t.parent, h, th1);
        }
        if (th2 != kNoSlot) {
            if (p2 < seg) plist[p2] = h | (th2 << 16);
            else uf_union(t.parent, h, th2);
        }
        pcount += __popc(m1) + __popc(m2);
    }
    __syncwarp();
    for (uint32_t i = lane; i < min(pcount, seg); i += 32) {
        const uint32_t pr = plist[i];
        uf_union(t.parent, pr & 0xFFFFu, pr >> 16);
    }
    __syncthreads();

    // 4: roots and per-root sums.  Each pixel walks to its root (the smallest
    // slot); a root's own pixel marks it with kMark | its linear index (the
    // cluster id), the others point straight at it.  Moments accumulate in
    // 32 bits; a cluster heavier than kQSafe32 sends the item through the
    // exact 64-bit pass.
    clear_words(sbits, nwords);
    clear_words(abits, nwords);
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if (s[k] == kNoSlot) continue;
        const uint32_t slot = s[k];
        const volatile uint32_t *vp = t.parent;
        uint32_t y = slot, p = vp[slot];
        if (p != y && !(p & kMark)) {
            y = p;
            p = vp[y];
            if (p != y && !(p & kMark)) y = root_walk_far(t.parent, p);
        }
        const uint32_t x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu;
        t.parent[slot] = y == slot ? (kMark | (r * C + c)) : y;
        s[k] = y;
        const int32_t q = (int32_t)((x >> 17) & 0xFFu) * gain - ped;
        const int32_t old = atomicAdd(&t.q[y], q);
        if (old + q > kQSafe32) bs.heavy = 1;
        atomicAdd(&t.np[y], 1u);
        atomicAdd(&t.m[y].x, q * (int32_t)r);
        atomicAdd(&t.m[y].y, q * (int32_t)c);
    }
    __syncthreads();
    const bool heavy = bs.heavy != 0;
    if (heavy) {
        for (uint32_t i = tid; i < S; i += kCCThreads) {
            t.exact[2 * i] = 0;
            t.exact[2 * i + 1] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            if (s[k] == kNoSlot) continue;
            const uint32_t x = w[k], y = s[k];
            const long long q = (long long)((int32_t)((x >> 17) & 0xFFu) * gain - ped);
            atomicAdd(&t.exact[2 * y], (unsigned long long)(q * (long long)(x & 0xFFu)));
            atomicAdd(&t.exact[2 * y + 1], (unsigned long long)(q * (long long)((x >> 8) & 0x1FFu)));
        }
        __syncthreads();
    }

    // 5: labels, and the kept roots of every 32-slot chunk (a warp ballots a
    // contiguous range of chunks into spre, free since phase 3)
    if (it.label_e) {
        const uint32_t *bi = L.ws.bucket_i + it.b;
        uint32_t iv[kD];
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const uint32_t j = tid + k * kCCThreads;
            iv[k] = j < n ? __ldg(bi + j) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            if (tid + k * kCCThreads >= n) continue;
            int32_t lab = -1;
            if (s[k] != kNoSlot) {
                const uint32_t y = s[k];
                lab = t.q[y] >= cthr ? (int32_t)(t.parent[y] & ~kMark) : -2;
            }
            it.label_e[iv[k]] = lab;
        }
    }
    constexpr uint32_t kWarps = kCCThreads / 32;
    const uint32_t chunks = (S + 31) >> 5;
    const uint32_t cpw = (chunks + kWarps - 1) / kWarps;
    const uint32_t wc0 = min(chunks, warp * cpw), wc1 = min(chunks, wc0 + cpw);
    uint32_t *ball = spre;
    uint32_t wrun = 0;
    for (uint32_t ch = wc0; ch < wc1; ++ch) {
        const uint32_t sl = (ch << 5) + lane;
        const bool kept = sl < S && (t.parent[sl] & kMark) && t.q[sl] >= cthr;
        const uint32_t bal = __ballot_sync(kFull, kept);
        if (lane == 0) ball[ch] = bal;
        wrun += __popc(bal);
    }
    if (lane == 0) bs.scan_tmp[warp] = wrun;
    __syncthreads();

    // 6: ordinals of the kept roots, compaction, staging
    uint32_t K, woff;
    {
        const uint32_t wt = lane < kWarps ? bs.scan_tmp[lane] : 0u;
        uint32_t ws = wt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, ws, o);
            if ((int)lane >= o) ws += y;
        }
        K = __shfl_sync(kFull, ws, kWarps - 1);
        woff = __shfl_sync(kFull, ws - wt, warp);
    }
    if (tid == 0) bs.heavy = 0;
    const uint32_t kslot_off = (chunks + 1) & ~1u; // words of ballots, rounded to keep kslot 4-byte aligned
    if (K <= 2 * (nwords - min(nwords, kslot_off))) {
        // compact the kept roots (their slots, by ordinal, after the ballot
        // words) so that every lane stages a cluster
        uint16_t *kslot = reinterpret_cast<uint16_t *>(spre + kslot_off);
        uint32_t o = woff;
        for (uint32_t ch = wc0; ch < wc1; ++ch) {
            const uint32_t bal = ball[ch];
            if ((bal >> lane) & 1u) kslot[o + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)((ch << 5) + lane);
            o += __popc(bal);
        }
        __syncthreads();
        for (uint32_t i = tid; i < K; i += kCCThreads) stage_cluster(L, it, t, heavy, kslot[i], i);
    } else {
        uint32_t o = woff;
        for (uint32_t ch = wc0; ch < wc1; ++ch) {
            const uint32_t bal = ball[ch];
            if ((bal >> lane) & 1u) stage_cluster(L, it, t, heavy, (ch << 5) + lane, o + __popc(bal & ((1u << lane) - 1u)));
            o += __popc(bal);
        }
    }
    // 7: compact labels, once every kept root's ordinal is in t.np
    if (kCompact) {
        __syncthreads();
        const uint32_t *bi = L.ws.bucket_i + it.b;
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const uint32_t j = tid + k * kCCThreads;
            if (j >= n) continue;
            uint16_t v = kLab16Below;
            if (s[k] != kNoSlot) v = t.q[s[k]] >= cthr ? (uint16_t)t.np[s[k]] : kLab16Dropped;
            it.label16_e[__ldg(bi + j)] = v;
        }
    }
    return K;
}

// ---------------------------------------------------------------- hash label store

// The hash store (tuning label_store = kStoreHash) clusters an item with a
// group of item_threads threads, one of the block's kCCThreads / item_threads
// groups, each with its own slice of shared memory and its own named
// barrier, so that several items of a ticket run side by side.  Pixel
// lookup goes through an open-addressing table keyed by linear pixel index
// (2n slots for n digis, linear probing) instead of module-sized bitmaps, so
// the memory an item needs follows its digi count.  Digi j of the item (in
// bucket order) owns entry j of the accumulator and parent arrays; the
// union-find links packed keys (lin << kHashIdxBits | j) with atomicMin, so
// the root of every cluster is its pixel of smallest linear index (the
// cluster id) with no sort.  Ids are put in order at the end: kept roots are
// counted per row, the row counts scanned, and each root ranked by column
// among the kept roots of its own row.
struct HashMem {
    int2 *m;           // [cap] root: sum q*row, sum q*col (32-bit, as in the block tiers)
    int32_t *q;        // [cap] root: charge
    uint32_t *np;      // [cap] root: pixel count; then its ordinal (compact labels)
    uint32_t *par;     // [cap] packed parent key; then a kept root's row base
    uint32_t *rowcnt;  // [256] kept roots per row
    uint32_t *table;   // [2 cap] (lin + 1) << 13 | surviving << 12 | j, 0 empty; then the row lists
    unsigned long long *exact; // [2 cap] (global) 64-bit moments of an item with a heavy cluster
};

__device__ __forceinline__ HashMem hash_mem(unsigned char *dsm, size_t smem, uint32_t groups, uint32_t gid,
                                            uint32_t cap, unsigned long long *exact)
{
    const size_t slice = (smem / groups) & ~(size_t)15;
    HashMem h;
    h.m = reinterpret_cast<int2 *>(dsm + slice * gid);
    h.q = reinterpret_cast<int32_t *>(h.m + cap);
    h.np = reinterpret_cast<uint32_t *>(h.q + cap);
    h.par = h.np + cap;
    h.rowcnt = h.par + cap;
    h.table = h.rowcnt + 256;
    h.exact = exact + (size_t)2 * cap * gid;
    return h;
}

// Barrier of the `threads` threads of one group (named barrier `id` >= 1;
// barrier 0 is the block's __syncthreads).  The compiler's own builtin, not
// inline assembly: like __syncthreads it is convergent, so the compiler
// never duplicates it into paths that a warp's threads take apart.
__device__ __forceinline__ void group_sync(uint32_t id, uint32_t threads)
{
    __syncwarp();
    __barrier_sync_count(id, threads);
}

// Home slot of pixel `lin` in a table of H slots (multiplicative hashing:
// the high bits of lin times the 32-bit golden ratio, scaled to [0, H)).
__device__ __forceinline__ uint32_t hash_home(uint32_t lin, uint32_t H) { return __umulhi(lin * 0x9E3779B1u, H); }

// Table entry of pixel `lin` if it is there and survives the pixel
// threshold, else 0.  The table holds at most H / 2 entries, so a probe
// always ends at an empty slot.
__device__ __forceinline__ uint32_t hash_survivor(const uint32_t *table, uint32_t H, uint32_t lin)
{
    uint32_t s = hash_home(lin, H);
    for (uint32_t i = 0; i < H; ++i) {
        const uint32_t e = table[s];
        if (e == 0) return 0u;
        if ((e >> 13) == lin + 1) return (e >> 12) & 1u ? e : 0u;
        s = s + 1 == H ? 0u : s + 1;
    }
    return 0u;
}

// Packed union-find key of a table entry.
__device__ __forceinline__ uint32_t hash_key(uint32_t e)
{
    return (((e >> 13) - 1u) << kHashIdxBits) | (e & ((1u << kHashIdxBits) - 1u));
}

// Find on packed keys with path halving (the index of a key is its low
// kHashIdxBits bits); parents only ever decrease, as in uf_find_halving.
__device__ __forceinline__ uint32_t hash_find(uint32_t *par, uint32_t x)
{
    constexpr uint32_t kIdx = (1u << kHashIdxBits) - 1u;
    volatile uint32_t *p = par;
    uint32_t y = p[x & kIdx];
    while (y != x) {
        const uint32_t z = p[y & kIdx];
        if (z != y) p[x & kIdx] = z;
        x = y;
        y = z;
    }
    return x;
}

// Lock-free union of the trees of packed keys a and b (the root with the
// larger key is linked under the smaller with atomicMin; a lost race retries
// from the new parent), as uf_union on slots.
__device__ __noinline__ void hash_union(uint32_t *par, uint32_t a, uint32_t b)
{
    for (;;) {
        a = hash_find(par, a);
        b = hash_find(par, b);
        if (a == b) return;
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicMin(&par[a & ((1u << kHashIdxBits) - 1u)], b);
        if (old == a) return;
        a = old;
    }
}

// One item of at most hash_capacity digis clustered by the calling group
// (gt = thread index in the group, GT = its size, bar = its barrier id);
// gflag and gheavy are the group's shared flag words (zero on entry, left
// zero).  Thread gt holds digis gt, gt + GT, ... in registers throughout.
// Phases, one group barrier each:
//   0 table and row counters emptied (the words load meanwhile)
//   1 every valid digi into the table (a pixel already there is a
//     duplicate); parent and accumulators of the survivors
//   2 unions with the surviving neighbours before the pixel in row-major
//     order: left L and up U; without U, upper-left UL (unless L, which
//     reaches UL through its own U) and upper-right UR.  With U, UL and UR
//     are U's own left and right neighbours, so every 8-adjacency is
//     covered with at most two unions a pixel.
//   3 roots, and charge, size and moments per root (32-bit shared atomics;
//     a cluster heavier than kQSafe32 sends the item through the exact
//     64-bit pass, as in the block tiers)
//   4 labels; kept roots counted per row
//   5 row bases by a scan of the row counts (each warp scans all 256, eight
//     a lane); every kept root's column into its row's list
//   6 ordinal = row base + kept roots of the row with a smaller column;
//     staging; (compact labels) the ordinals read back per digi
// Returns the number of kept clusters (uniform over the group).
template <int kD>
__device__ uint32_t hash_item(const Launch &L, const ItemCtx &it, const HashMem &h, uint32_t gt, uint32_t GT,
                              uint32_t bar, uint32_t *gflag, uint32_t *gheavy)
{
    constexpr uint32_t kIdx = (1u << kHashIdxBits) - 1u;
    const uint32_t R = L.g.R, C = L.g.C;
    const int32_t thr = L.g.pixel_thr, cthr = L.g.cluster_thr;
    const uint32_t n = it.n, lane = threadIdx.x & 31, H = 2 * n;
    const uint32_t *bw = L.ws.bucket_w + it.b;
    const uint32_t *bi = L.ws.bucket_i + it.b;
    const int32_t gain = it.gain, ped = it.ped;

    // 0
    for (uint32_t i = gt; i < H; i += GT) h.table[i] = 0;
    for (uint32_t i = gt; i < 256; i += GT) h.rowcnt[i] = 0;
    uint32_t w[kD], rt[kD];
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        const uint32_t j = gt + k * GT;
        w[k] = j < n ? __ldg(bw + j) : 0u;
    }
    group_sync(bar, GT);

    // 1
    uint32_t err = 0;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        rt[k] = kNoSlot;
        const uint32_t j = gt + k * GT;
        if (j >= n) continue;
        const uint32_t x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu, adc = (x >> 17) & 0xFFu;
        if (r >= R || c >= C || adc == 0 || (x >> 25) != 0) {
            err |= kErrBadDigi;
            continue;
        }
        const uint32_t lin = r * C + c;
        const bool surv = (int32_t)adc * gain - ped >= thr;
        const uint32_t e = ((lin + 1) << 13) | ((uint32_t)surv << 12) | j;
        uint32_t s = hash_home(lin, H), i = 0;
        for (; i < H; ++i) {
            const uint32_t old = atomicCAS(&h.table[s], 0u, e);
            if (old == 0) break;
            if ((old >> 13) == lin + 1) {
                err |= kErrDup;
                break;
            }
            s = s + 1 == H ? 0u : s + 1;
        }
        if (i == H) err |= kErrCapacity; // not reached: at most n entries in 2n slots
        if (surv) {
            const uint32_t key = (lin << kHashIdxBits) | j;
            h.par[j] = key;
            h.q[j] = 0;
            h.np[j] = 0;
            h.m[j] = make_int2(0, 0);
            rt[k] = key;
        }
    }
    err = __reduce_or_sync(kFull, err);
    if (err && lane == 0) atomicOr(gflag, err);
    group_sync(bar, GT);
    const uint32_t flag = *(volatile uint32_t *)gflag;
    if (flag) {
        group_sync(bar, GT); // every thread of the group has read the flag
        if (gt == 0) {
            if (flag & (kErrBadDigi | kErrDup)) atomicOr(it.err_e, flag & (kErrBadDigi | kErrDup));
            if (flag & kErrCapacity) atomicOr(&L.ws.ctl[1], kErrCapacity);
            *gflag = 0;
        }
        return 0;
    }

    // 2
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if (rt[k] == kNoSlot) continue;
        const uint32_t x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu, lin = r * C + c;
        const uint32_t eL = c > 0 ? hash_survivor(h.table, H, lin - 1) : 0u;
        uint32_t e1 = eL, e2 = 0;
        if (r > 0) {
            const uint32_t eU = hash_survivor(h.table, H, lin - C);
            if (eU) {
                e2 = eU;
            } else {
                if (!eL && c > 0) e1 = hash_survivor(h.table, H, lin - C - 1);
                if (c + 1 < C) e2 = hash_survivor(h.table, H, lin - C + 1);
            }
        }
        if (e1) hash_union(h.par, rt[k], hash_key(e1));
        if (e2) hash_union(h.par, rt[k], hash_key(e2));
    }
    group_sync(bar, GT);

    // 3
    bool heavy_here = false;
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if (rt[k] == kNoSlot) continue;
        const uint32_t root = hash_find(h.par, rt[k]), y = root & kIdx;
        const uint32_t x = w[k];
        const int32_t q = (int32_t)((x >> 17) & 0xFFu) * gain - ped;
        const int32_t old = atomicAdd(&h.q[y], q);
        if (old + q > kQSafe32) heavy_here = true;
        atomicAdd(&h.np[y], 1u);
        atomicAdd(&h.m[y].x, q * (int32_t)(x & 0xFFu));
        atomicAdd(&h.m[y].y, q * (int32_t)((x >> 8) & 0x1FFu));
        rt[k] = root;
    }
    if (heavy_here) *gheavy = 1;
    group_sync(bar, GT);
    const bool heavy = *(volatile uint32_t *)gheavy != 0;
    if (heavy) {
        for (uint32_t i = gt; i < 2 * n; i += GT) h.exact[i] = 0;
        group_sync(bar, GT);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            if (rt[k] == kNoSlot) continue;
            const uint32_t x = w[k], y = rt[k] & kIdx;
            const long long q = (long long)((int32_t)((x >> 17) & 0xFFu) * gain - ped);
            atomicAdd(&h.exact[2 * y], (unsigned long long)(q * (long long)(x & 0xFFu)));
            atomicAdd(&h.exact[2 * y + 1], (unsigned long long)(q * (long long)((x >> 8) & 0x1FFu)));
        }
        group_sync(bar, GT);
    }

    // 4
    uint32_t kr = 0; // bit k: digi k of this thread is a kept root
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        const uint32_t j = gt + k * GT;
        if (j >= n) continue;
        int32_t lab = -1;
        if (rt[k] != kNoSlot) {
            const bool kept = h.q[rt[k] & kIdx] >= cthr;
            lab = kept ? (int32_t)(rt[k] >> kHashIdxBits) : -2;
            const uint32_t x = w[k], r = x & 0xFFu;
            if (kept && rt[k] == (((r * C + ((x >> 8) & 0x1FFu)) << kHashIdxBits) | j)) {
                h.par[j] = atomicAdd(&h.rowcnt[r], 1u); // arrival in the row
                kr |= 1u << k;
            }
        }
        if (it.label_e) it.label_e[__ldg(bi + j)] = lab;
    }
    group_sync(bar, GT);
    if (gt == 0) *gheavy = 0; // read by every thread before the barrier above

    // 5
    uint32_t K, base8;
    {
        uint32_t s8 = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s8 += h.rowcnt[lane * 8 + i];
        uint32_t incl = s8;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        K = __shfl_sync(kFull, incl, 31);
        base8 = incl - s8; // kept roots in the rows before this lane's eight
    }
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if ((uint32_t)k * GT >= n) break; // uniform over the warp
        const uint32_t r = w[k] & 0xFFu;
        uint32_t pre = __shfl_sync(kFull, base8, r >> 3);
        if ((kr >> k) & 1u) {
            const uint32_t j = gt + k * GT;
            for (uint32_t i = r & ~7u; i < r; ++i) pre += h.rowcnt[i];
            h.table[pre + h.par[j]] = (w[k] >> 8) & 0x1FFu;
            h.par[j] = pre;
        }
    }
    group_sync(bar, GT);

    // 6
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        if (!((kr >> k) & 1u)) continue;
        const uint32_t j = gt + k * GT, x = w[k], r = x & 0xFFu, c = (x >> 8) & 0x1FFu;
        const uint32_t pre = h.par[j], end = pre + h.rowcnt[r];
        uint32_t ord = pre;
        for (uint32_t i = pre; i < end; ++i) ord += h.table[i] < c ? 1u : 0u;
        const int32_t Q = h.q[j];
        long long mr, mc;
        if (heavy) {
            mr = (long long)h.exact[2 * j];
            mc = (long long)h.exact[2 * j + 1];
        } else {
            const int2 mm = h.m[j];
            mr = mm.x;
            mc = mm.y;
        }
        L.ws.staging.put(it.b + ord, (int32_t)(rt[k] >> kHashIdxBits), Q, (int32_t)h.np[j], centroid_abs(mr, Q),
                         centroid_abs(mc, Q));
        if (it.label16_e) h.np[j] = ord; // read back by the compact labels
    }
    if (it.label16_e) {
        group_sync(bar, GT);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const uint32_t j = gt + k * GT;
            if (j >= n) continue;
            uint16_t v = kLab16Below;
            if (rt[k] != kNoSlot) {
                const uint32_t y = rt[k] & kIdx;
                v = h.q[y] >= cthr ? (uint16_t)h.np[y] : kLab16Dropped;
            }
            it.label16_e[__ldg(bi + j)] = v;
        }
    }
    group_sync(bar, GT); // the slice is free for the group's next item
    return K;
}

// Ordered output across tickets.  chain[g] holds ticket g's aggregate (the
// number of clusters it staged, flag bit 62), published by its owner as soon
// as it is staged, without waiting; chain[ngroups + g] receives its inclusive
// prefix (flag bit 63).  The prefix spreads by a cooperative frontier:
// ctl[3] = F means tickets below F carry their inclusive prefix.  Any warp may
// push F forward: it reads the aggregates of the 32 tickets from F on, scans
// the run of consecutive published ones on top of the inclusive prefix of
// F - 1, publishes those prefixes and raises F.  Racing warps compute and
// write identical values.
__device__ void advance_frontier(unsigned long long *chain, uint32_t *frontier, uint64_t ngroups)
{
    const unsigned long long kFlagInc = 1ull << 63, kMask = (1ull << 62) - 1;
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long *inc = chain + ngroups;
    for (int rounds = 0; rounds < 64; ++rounds) {
        uint32_t F = 0;
        if (lane == 0) F = *(volatile uint32_t *)frontier;
        F = __shfl_sync(kFull, F, 0);
        if (F >= ngroups) return;
        unsigned long long prev = 0;
        if (F > 0) {
            const unsigned long long pv = ld_acquire(&inc[F - 1]);
            if (!(pv & kFlagInc)) return; // the prefix below F is not visible yet
            prev = pv & kMask;
        }
        const uint64_t j = (uint64_t)F + lane;
        const unsigned long long a = j < ngroups ? ld_acquire(&chain[j]) : 0ull;
        const uint32_t avail = __ballot_sync(kFull, (a >> 62) != 0);
        const uint32_t u = (~avail) ? (uint32_t)(__ffs(~avail) - 1) : 32u; // leading run of published tickets
        if (u == 0) return;
        unsigned long long x = lane < u ? (a & kMask) : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane < u) st_release(&inc[j], kFlagInc | (prev + x));
        __syncwarp();
        __threadfence();
        if (lane == 0) atomicMax(frontier, F + u);
        if (u < 32) return;
    }
}

// Resolve ticket g (one full warp): its exclusive prefix once the frontier
// has passed it.  Non-blocking mode returns false if it has not; blocking
// mode keeps pushing the frontier, for at most kSpinLimit iterations and
// kWaitNs of wall time, then reports kErrTimeout (and every later blocking
// wait of the launch gives up at once).  Every aggregate is published
// without waiting, so a blocking wait only expires if one never is.
__device__ bool chain_resolve(unsigned long long *chain, uint32_t *frontier, uint64_t ngroups, uint64_t g,
                              unsigned long long agg, bool blocking, unsigned long long *excl_out,
                              uint32_t *launch_err)
{
    const unsigned long long kFlagInc = 1ull << 63, kMask = (1ull << 62) - 1;
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long *inc = chain + ngroups;
    unsigned long long t0 = 0;
    for (uint32_t spins = 0;; ++spins) {
        unsigned long long v = 0;
        uint32_t failed = 0;
        if (lane == 0) {
            v = ld_acquire(&inc[g]);
            failed = *(volatile uint32_t *)launch_err & kErrTimeout;
        }
        v = __shfl_sync(kFull, v, 0);
        failed = __shfl_sync(kFull, failed, 0);
        if (blocking && failed && !(v & kFlagInc)) {
            *excl_out = 0;
            return true;
        }
        if (!(v & kFlagInc)) {
            advance_frontier(chain, frontier, ngroups);
            if (lane == 0) v = ld_acquire(&inc[g]);
            v = __shfl_sync(kFull, v, 0);
        }
        if (v & kFlagInc) {
            *excl_out = (v & kMask) - agg;
            return true;
        }
        if (!blocking) return false;
        unsigned long long now = 0;
        if (lane == 0) now = global_ns();
        now = __shfl_sync(kFull, now, 0);
        if (spins == 0) t0 = now;
        if (spins > kSpinLimit || now - t0 > kWaitNs) {
            if (lane == 0) atomicOr(launch_err, kErrTimeout);
            *excl_out = 0;
            return true;
        }
        __nanosleep(64);
    }
}

template <int kMinBlocks, bool kHash>
__global__ void __launch_bounds__(kCCThreads, kMinBlocks) cc_kernel(const Launch L)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ BlockShared bs;
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_n[kGroup], s_b[kGroup];
    __shared__ ItemRec s_rec[kGroup];
    __shared__ uint32_t s_ticket;

    const uint32_t R = L.g.R, C = L.g.C, M = L.g.M;
    const uint32_t nwords = (R * C + 31) >> 5;
    const uint32_t tid = threadIdx.x;
    const uint32_t T = L.tune.tile_slots, warp_max = L.tune.warp_max;
    Tile sm;
    sm.q = reinterpret_cast<int32_t *>(dsm);
    sm.np = reinterpret_cast<uint32_t *>(sm.q + T);
    sm.m = reinterpret_cast<int2 *>(sm.np + T);
    sm.parent = reinterpret_cast<uint32_t *>(sm.m + T);
    sm.exact = L.ws.exact + (size_t)blockIdx.x * 2 * T;
    uint32_t *abits = sm.parent + T;
    uint32_t *sbits = abits + nwords;
    uint32_t *spre = sbits + nwords;

    const uint64_t EM = (uint64_t)L.E * M;
    const uint32_t G = ticket_items(EM, gridDim.x, L.tune.ticket_max, L.N);
    const uint64_t ngroups = (EM + G - 1) / G;
    // items of the register tier and the hash store: kD digis a thread
    constexpr int kD = cc_digis_per_thread(kMinBlocks);
    // hash store: items of warp_max < n <= hash_max go to groups of GT
    // threads (0 with the bitmap store)
    const uint32_t GT = L.tune.item_threads, hgroups = (uint32_t)kCCThreads / GT;
    const uint32_t hash_max = kHash ? hash_capacity(cc_smem_bytes(R, C, T), T, GT, (uint32_t)kD) : 0u;
    const uint32_t gid = tid / GT, gtid = tid - gid * GT;
    const HashMem hm = hash_mem(dsm, cc_smem_bytes(R, C, T), hgroups, gid, hash_max, sm.exact);
    __shared__ uint32_t s_gflag[kCCThreads / 128], s_gheavy[kCCThreads / 128];
    if (kHash && tid < (uint32_t)(kCCThreads / 128)) {
        s_gflag[tid] = 0;
        s_gheavy[tid] = 0;
    }
    if (tid == 0) {
        bs.flag = 0;
        bs.heavy = 0;
    }
    // block-tier items start from zeroed bitmaps and leave them zeroed
    clear_words(abits, nwords);
    clear_words(sbits, nwords);
    if (L.ws.ctl[1] & kErrBadOffsets) return;
    // each item's count of kept clusters goes to kcount[item]; the ordered
    // output is written by offsets_kernel and copy_kernel
    uint32_t *kcount = L.ws.cursor;
    for (;;) {
        {
            if (tid == 0) s_ticket = atomicAdd(&L.ws.ctl[0], 1u);
            __syncthreads();
            const uint64_t g = s_ticket;
            if (g >= ngroups) break;
            {
                const uint64_t item0 = g * G;
                if (tid < (uint32_t)kGroup) {
                    const uint64_t item = item0 + tid;
                    const bool ok = tid < G && item < EM;
                    s_n[tid] = ok ? L.ws.count[item] : 0u;
                    s_b[tid] = ok ? L.ws.boff[item] : 0u;
                    if (ok) {
                        s_rec[tid] = make_rec(L, item);
                        if (s_n[tid] == 0) kcount[item] = 0;
                    }
                }
                __syncthreads();
                {   // pull the ticket's buckets (words and digi indices, contiguous
                    // over its items) into L2, one 128-byte line per thread, so
                    // that the items after the first do not wait on DRAM
                    uint32_t last = 0;
                    for (uint32_t i = 0; i < G; ++i)
                        if (s_n[i]) last = i;
                    const uint64_t b0 = s_b[0], b1 = (uint64_t)s_b[last] + s_n[last];
                    const uint32_t lines = b1 > b0 ? (uint32_t)(((b1 - b0) * 4 + 127) / 128) : 0u;
                    for (uint32_t li = tid; li < 2 * lines; li += kCCThreads) {
                        const bool second = li >= lines;
                        const uint32_t *base = second ? L.ws.bucket_i : L.ws.bucket_w;
                        const uint64_t off = b0 * 4 + (uint64_t)(second ? li - lines : li) * 128; // inside the array
                        if (off < b1 * 4)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(base) + off));
                    }
                }
                {   // warp tier: one warp per small item
                    const uint32_t wi = tid >> 5;
                    const uint32_t n = s_n[wi];
                    if (n > 0 && n <= warp_max) {
                        const ItemCtx it = make_item(L, s_rec[wi], s_b[wi], n);
                        const uint32_t K = n <= 32 ? warp_item<1>(L, it) : warp_item<2>(L, it);
                        if ((tid & 31) == 0) kcount[item0 + wi] = K;
                    }
                }
                __syncthreads();
                if (kHash && hash_max > warp_max) {
                    // hash store: the items above the warp tier and within
                    // its capacity, dealt round-robin to the block's groups
                    uint32_t nh = 0;
                    for (int i = 0; i < kGroup; ++i) {
                        const uint32_t n = s_n[i];
                        if (n <= warp_max || n > hash_max) continue;
                        if (nh++ % hgroups != gid) continue;
                        const ItemCtx it = make_item(L, s_rec[i], s_b[i], n);
                        const uint32_t K = hash_item<kD>(L, it, hm, gtid, GT, 1 + gid, &s_gflag[gid], &s_gheavy[gid]);
                        if (gtid == 0) kcount[item0 + i] = K;
                    }
                    if (nh) { // block-uniform: the slices covered the bitmaps, which the block tier wants zeroed
                        __syncthreads();
                        clear_words(abits, nwords);
                        clear_words(sbits, nwords);
                        __syncthreads();
                    }
                }
                for (int i = 0; i < kGroup; ++i) { // block tier: larger items one at a time
                    const uint32_t n = s_n[i];
                    if (n <= warp_max || n <= hash_max) continue;
                    const ItemCtx it = make_item(L, s_rec[i], s_b[i], n);
                    uint32_t K;
                    if (n <= (uint32_t)kD * kCCThreads && n <= T) {
                        // (compact labels keep each digi's root slot live through the
                        // staging: a separate instance, so the other keeps its registers)
                        K = it.label16_e ? block_item_reg<kD, true>(L, it, abits, sbits, spre, sm, bs)
                                         : block_item_reg<kD, false>(L, it, abits, sbits, spre, sm, bs);
                    } else if (n <= T) {
                        K = block_item<false>(L, it, abits, sbits, spre, sm, bs);
                    } else {
                        if (tid == 0) {
                            bs.big_off = 0;
                            if (L.ws.big_arena) bs.big_off = atomicAdd(&L.ws.ctl[2], n);
                        }
                        __syncthreads();
                        const uint64_t cap = L.ws.big_arena ? (uint64_t)n : L.ws.big_slots;
                        unsigned char *base =
                            L.ws.big + (L.ws.big_arena ? (uint64_t)bs.big_off : (uint64_t)blockIdx.x * L.ws.big_slots) *
                                           kBigSlotBytes;
                        const bool fits = L.ws.big_arena ? (uint64_t)bs.big_off + n <= L.ws.big_slots
                                                         : (uint64_t)min(n, R * C) <= L.ws.big_slots;
                        Tile gt;
                        gt.q = reinterpret_cast<int32_t *>(base);
                        gt.np = reinterpret_cast<uint32_t *>(gt.q + cap);
                        gt.exact = reinterpret_cast<unsigned long long *>(gt.np + cap);
                        gt.m = reinterpret_cast<int2 *>(gt.exact + 2 * cap);
                        gt.parent = reinterpret_cast<uint32_t *>(gt.m + cap);
                        K = fits ? block_item<true>(L, it, abits, sbits, spre, gt, bs) : 0u;
                        if (!fits && tid == 0) atomicOr(&L.ws.ctl[1], kErrCapacity);
                    }
                    if (n > (uint32_t)kD * kCCThreads || n > T) {
                        // the general tier leaves its bitmaps (and scratch in them) behind
                        __syncthreads();
                        clear_words(abits, nwords);
                        clear_words(sbits, nwords);
                        if (tid == 0) {
                            bs.flag = 0;
                            bs.heavy = 0;
                        }
                    }
                    if (tid == 0) kcount[item0 + i] = K;
                    __syncthreads();
                }
            }
        }
    }
}


// Ordered output, in two kernels.
//
// offsets_kernel: block c takes chunk c of kOffItems consecutive items (in
// the order blocks start, so the chunks below it are running or done), scans
// the items' kept-cluster counts (cursor[], from cc_kernel), publishes the
// chunk's total in chain[c] and resolves its exclusive prefix with the
// cooperative frontier (a bounded wait; few, large chunks keep the frontier
// short); it writes every item's first output position to count[] (free
// since cc_kernel read it), the cluster offsets of the events that start in
// the chunk, and the capacity check.
constexpr int kOffThreads = 1024;
constexpr uint32_t kOffItems = kOffThreads;

__global__ void __launch_bounds__(kOffThreads) offsets_kernel(const Launch L)
{
    __shared__ uint32_t s_tmp[kOffThreads / 32 + 1];
    __shared__ uint32_t s_chunk;
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_prefix;
    const uint32_t tid = threadIdx.x, M = L.g.M;
    const uint64_t EM = (uint64_t)L.E * M;
    const uint64_t nchunks = (EM + kOffItems - 1) / kOffItems;
    if (L.ws.ctl[1] & kErrBadOffsets) return;
    if (tid == 0) s_chunk = atomicAdd(&L.ws.ctl[4], 1u);
    __syncthreads();
    const uint64_t c = s_chunk;
    if (c >= nchunks) return;
    const uint64_t item = c * kOffItems + tid;
    const bool in = item < EM;
    const uint32_t k = in ? L.ws.cursor[item] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<kOffThreads>(k, s_tmp, &total);
    if (tid < 32) {
        // The chunk's total is all that other blocks read of it, so a relaxed
        // store suffices.  (The test hook kDebugWithholdTicket0 keeps chunk
        // 0's total back, so that the waits on it expire.)
        const unsigned long long kAgg = 1ull << 62;
        if (tid == 0 && (c != 0 || !(L.debug & kDebugWithholdTicket0))) st_relaxed(&L.ws.chain[c], kAgg | total);
        __syncwarp();
        unsigned long long P = 0;
        chain_resolve(L.ws.chain, &L.ws.ctl[3], nchunks, c, total, true, &P, &L.ws.ctl[1]);
        if (tid == 0) s_prefix = P;
    }
    __syncthreads();
    const unsigned long long P = s_prefix;
    if (in) {
        const unsigned long long o = P + ex;
        L.ws.count[item] = (uint32_t)o;
        uint32_t e, m;
        item_coords(item, M, &e, &m);
        if (m == 0) L.out.cluster_offsets[e] = o;
        // the output chunks whose first position falls in this item's range
        if (k > 0)
            for (unsigned long long q = (o + kOutChunk - 1) / kOutChunk; q * kOutChunk < o + k; ++q)
                L.ws.chunk_item[q] = (uint32_t)item;
    }
    if (tid == 0 && c == nchunks - 1) {
        L.out.cluster_offsets[L.E] = P + total;
        L.ws.ctl[6] = (uint32_t)(P + total);
    }
    if (tid == 0 && P + total > L.out.capacity) atomicOr(&L.ws.ctl[1], kErrCapacity);
}

// copy_kernel: the staged clusters (SoA, at each item's bucket start) to
// their ordered output positions, driven by the output: a warp takes a chunk
// of kOutChunk consecutive positions, four a lane, finds the item of its
// first position by a binary search between the items that hold the first
// positions of this chunk and the next (chunk_item[], from offsets_kernel),
// and walks on from there.  Every warp store is then a whole, aligned 512-byte
// run of one output array, which matters most when the outputs are mapped
// host memory written over the chip-to-chip link (partial lines cost there).
// The first E threads write the per-event status codes from the error bits.
constexpr int kCopyThreads = 256;

__global__ void __launch_bounds__(kCopyThreads) copy_kernel(const Launch L)
{
    pdl_wait();
    const uint32_t lane = threadIdx.x & 31, M = L.g.M;
    const uint64_t gt = (uint64_t)blockIdx.x * kCopyThreads + threadIdx.x;
    const bool bad_offsets = (L.ws.ctl[1] & kErrBadOffsets) != 0;
    if (bad_offsets && gt <= L.E) L.out.cluster_offsets[gt] = 0; // no clusters
    if (gt < L.E) {
        const uint32_t bits = L.ws.event_err[gt] | L.ws.ctl[1];
        int32_t st = 0;                          // HP_OK
        if (bits & kErrBadOffsets) st = 3;       // HP_EINVAL
        else if (bits & kErrTimeout) st = 8;     // HP_ETIMEOUT
        else if (bits & kErrCapacity) st = 6;    // HP_ECAPACITY
        else if (bits & kErrBadDigi) st = 4;     // HP_EBADDIGI
        else if (bits & kErrDup) st = 5;         // HP_EDUP
        L.out.event_status[gt] = st;
    }
    if (bad_offsets) return;
    const Staging sg = L.ws.staging;
    const uint32_t total = L.ws.ctl[6];
    const uint32_t T = (uint32_t)min((unsigned long long)total, (unsigned long long)L.out.capacity);
    const uint32_t nchunks = (uint32_t)(((uint64_t)total + kOutChunk - 1) / kOutChunk);
    const uint32_t last_item = (uint32_t)((uint64_t)L.E * M - 1);
    const bool vec = ((reinterpret_cast<uintptr_t>(L.out.module) | reinterpret_cast<uintptr_t>(L.out.id) |
                       reinterpret_cast<uintptr_t>(L.out.charge) | reinterpret_cast<uintptr_t>(L.out.npix) |
                       reinterpret_cast<uintptr_t>(L.out.x) | reinterpret_cast<uintptr_t>(L.out.y)) & 15) == 0;
    const uint64_t warps = (uint64_t)gridDim.x * (kCopyThreads / 32);
    for (uint64_t ch = gt >> 5; ch < nchunks; ch += warps) {
        const uint32_t p0 = (uint32_t)ch * kOutChunk + 4 * lane;
        if (p0 >= T) continue;
        // the item of p0: the last one in [lo, hi] whose range starts at or
        // before p0 (empty items share their start with the next item)
        uint32_t lo = L.ws.chunk_item[ch];
        uint32_t hi = ch + 1 < nchunks ? L.ws.chunk_item[ch + 1] : last_item;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (L.ws.count[mid] <= p0) lo = mid;
            else hi = mid - 1;
        }
        uint32_t it = lo, start = L.ws.count[it], K = L.ws.cursor[it];
        const uint32_t nv = min(4u, T - p0);
        uint32_t mo[4];
        int32_t id[4], q[4], np[4];
        float x[4], y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mo[j] = 0;
            id[j] = q[j] = np[j] = 0;
            x[j] = y[j] = 0.f;
            if ((uint32_t)j >= nv) continue;
            const uint32_t p = p0 + j;
            while (p - start >= K) { // on to the item holding p (count[it + 1] = start + K)
                ++it;
                start = L.ws.count[it];
                K = L.ws.cursor[it];
            }
            const uint64_t a = (uint64_t)L.ws.boff[it] + (p - start);
            uint32_t e, m;
            item_coords(it, M, &e, &m);
            mo[j] = m;
            id[j] = sg.id[a];
            q[j] = sg.charge[a];
            np[j] = sg.npix[a];
            x[j] = sg.x[a];
            y[j] = sg.y[a];
        }
        const ClusterCols host = {L.out.module, L.out.id, L.out.charge, L.out.npix, L.out.x, L.out.y};
        const bool in_head = p0 + nv <= L.out.head_n, past_head = p0 >= L.out.head_n;
        if (nv == 4 && (in_head || (past_head && vec))) {
            const ClusterCols &d = in_head ? L.out.head : host;
            *reinterpret_cast<uint4 *>(d.module + p0) = make_uint4(mo[0], mo[1], mo[2], mo[3]);
            *reinterpret_cast<int4 *>(d.id + p0) = make_int4(id[0], id[1], id[2], id[3]);
            *reinterpret_cast<int4 *>(d.charge + p0) = make_int4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<int4 *>(d.npix + p0) = make_int4(np[0], np[1], np[2], np[3]);
            *reinterpret_cast<float4 *>(d.x + p0) = make_float4(x[0], x[1], x[2], x[3]);
            *reinterpret_cast<float4 *>(d.y + p0) = make_float4(y[0], y[1], y[2], y[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((uint32_t)j >= nv) continue;
                const ClusterCols &d = p0 + j < L.out.head_n ? L.out.head : host;
                d.module[p0 + j] = mo[j];
                d.id[p0 + j] = id[j];
                d.charge[p0 + j] = q[j];
                d.npix[p0 + j] = np[j];
                d.x[p0 + j] = x[j];
                d.y[p0 + j] = y[j];
            }
        }
    }
    // with compact labels: every item's first cluster counted from its event's first
    if (L.out.item_first) {
        const uint64_t EM = (uint64_t)L.E * M;
        for (uint64_t item = gt; item < EM; item += (uint64_t)gridDim.x * kCopyThreads)
            L.out.item_first[item] = L.ws.count[item] - L.ws.count[item - item % M];
    }
}

// Serving batches: block (x, e) copies a slice of request e's digis.
// Four digis a thread, read with one 16-byte (words) and one 8-byte
// (module ids) load where the source allows it: the sources are host memory
// read over the chip-to-chip link, where wide loads carry more per request.
__global__ void __launch_bounds__(256) gather_kernel(const GatherEntry *table, uint32_t *words, uint16_t *modules)
{
    const GatherEntry g = table[blockIdx.y];
    const bool wv = (reinterpret_cast<uintptr_t>(g.words) & 15) == 0;
    const bool mv = (reinterpret_cast<uintptr_t>(g.modules) & 7) == 0;
    const uint64_t n4 = g.n / 4, stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t *dw = words + g.off;
    uint16_t *dm = modules + g.off;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        uint32_t w[4];
        uint16_t m[4];
        if (wv) {
            const uint4 v = reinterpret_cast<const uint4 *>(g.words)[q];
            w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = g.words[4 * q + j];
        }
        if (mv) {
            const ushort4 v = reinterpret_cast<const ushort4 *>(g.modules)[q];
            m[0] = v.x, m[1] = v.y, m[2] = v.z, m[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) m[j] = g.modules[4 * q + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            dw[4 * q + j] = w[j];
            dm[4 * q + j] = m[j];
        }
    }
    for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
        dw[i] = g.words[i];
        dm[i] = g.modules[i];
    }
}

} // namespace

cudaError_t launch_gather(const GatherEntry *table, uint32_t n_requests, uint64_t max_n, uint32_t *words,
                          uint16_t *modules, cudaStream_t stream)
{
    if (n_requests == 0 || max_n == 0) return cudaSuccess;
    const uint64_t bx = std::min<uint64_t>(32, (max_n + 4095) / 4096);
    gather_kernel<<<dim3((unsigned)bx, n_requests), 256, 0, stream>>>(table, words, modules);
    return cudaGetLastError();
}

size_t carve_workspace(void *base, uint32_t E, uint32_t M, uint64_t N, uint32_t R, uint32_t C, int cc_grid,
                       const Tuning &tune, Workspace *ws, int sm_count)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char * {
        off = (off + 255) & ~(size_t)255;
        const size_t o = off;
        off += bytes;
        return base ? static_cast<unsigned char *>(base) + o : nullptr;
    };
    const uint64_t EM = (uint64_t)E * M;
    const uint64_t nchunks = (EM + kOffItems - 1) / kOffItems;
    Workspace w{};
    w.ctl = reinterpret_cast<uint32_t *>(take(64));
    w.event_err = reinterpret_cast<uint32_t *>(take(4ull * E));
    w.count = reinterpret_cast<uint32_t *>(take(4ull * EM));
    w.count2 = reinterpret_cast<uint32_t *>(take(4ull * EM));
    w.chain = reinterpret_cast<unsigned long long *>(take(16ull * nchunks)); // aggregates, then inclusive prefixes
    off = (off + 255) & ~(size_t)255;
    w.zero_bytes = off;
    w.boff = reinterpret_cast<uint32_t *>(take(4ull * EM));
    w.blk_off = reinterpret_cast<uint32_t *>(take(4ull * kHistCap * bucket_grid(N, sm_count)));
    w.cursor = reinterpret_cast<uint32_t *>(take(4ull * EM));
    w.bucket_w = reinterpret_cast<uint32_t *>(take(4ull * N));
    w.bucket_i = reinterpret_cast<uint32_t *>(take(4ull * N));
    w.chunk_item = reinterpret_cast<uint32_t *>(take(4ull * (N / kOutChunk + 2)));
    w.staging.id = reinterpret_cast<int32_t *>(take(4ull * N));
    w.staging.charge = reinterpret_cast<int32_t *>(take(4ull * N));
    w.staging.npix = reinterpret_cast<int32_t *>(take(4ull * N));
    w.staging.x = reinterpret_cast<float *>(take(4ull * N));
    w.staging.y = reinterpret_cast<float *>(take(4ull * N));
    w.exact = reinterpret_cast<unsigned long long *>(take(16ull * tune.tile_slots * (cc_grid > 0 ? cc_grid : 1)));
    const uint64_t slab_slots = std::min<uint64_t>((uint64_t)R * C, N);
    const uint64_t slab_total = slab_slots * (uint64_t)(cc_grid > 0 ? cc_grid : 1);
    w.big_arena = N <= slab_total ? 1 : 0;
    w.big_slots = w.big_arena ? N : slab_slots;
    w.big = take(kBigSlotBytes * (w.big_arena ? N : slab_total));
    off = (off + 255) & ~(size_t)255;
    if (ws) *ws = w;
    return off;
}

namespace {

// Largest tile (a multiple of 256 slots, at most max_slots) with which
// `blocks` blocks of `kern` stay resident on one SM; 0 if none does.  Also
// raises the kernel's dynamic shared memory limit to what that tile needs.
template <class K>
cudaError_t fit_tile(K kern, int device, int blocks, uint32_t R, uint32_t C, uint32_t max_slots, uint32_t *tile)
{
    *tile = 0;
    int optin = 0;
    cudaError_t err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (err != cudaSuccess) return err;
    cudaFuncAttributes fa;
    err = cudaFuncGetAttributes(&fa, kern);
    if (err != cudaSuccess) return err;
    const size_t limit = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    uint32_t t = max_slots;
    while (t >= 256 && cc_smem_bytes(R, C, t) > limit) t -= 256;
    if (t < 256) return cudaSuccess;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cc_smem_bytes(R, C, t));
    if (err != cudaSuccess) return err;
    for (; t >= 256; t -= 256) {
        int nb = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kCCThreads, cc_smem_bytes(R, C, t));
        if (err != cudaSuccess) return err;
        if (nb >= blocks) {
            *tile = t;
            break;
        }
    }
    return cudaSuccess;
}

} // namespace

cudaError_t init_kernels(int device, uint32_t R, uint32_t C, uint32_t max_tile[4], uint32_t hash_tile[4])
{
    cudaError_t err = cudaSetDevice(device);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    if (err != cudaSuccess) return err;
    max_tile[0] = hash_tile[0] = 0;
    // the bitmap and hash label stores are separate instances of the kernel
    err = fit_tile(cc_kernel<1, false>, device, 1, R, C, kMaxTileSlots, &max_tile[1]);
    if (err == cudaSuccess) err = fit_tile(cc_kernel<1, true>, device, 1, R, C, kMaxTileSlots, &hash_tile[1]);
    if (err == cudaSuccess) err = fit_tile(cc_kernel<2, false>, device, 2, R, C, kSmemSlots, &max_tile[2]);
    if (err == cudaSuccess) err = fit_tile(cc_kernel<2, true>, device, 2, R, C, kSmemSlots, &hash_tile[2]);
    if (err == cudaSuccess) err = fit_tile(cc_kernel<3, false>, device, 3, R, C, kSmemSlots, &max_tile[3]);
    if (err == cudaSuccess) err = fit_tile(cc_kernel<3, true>, device, 3, R, C, kSmemSlots, &hash_tile[3]);
    return err;
}

const char *const kKernelNames[kNumKernels] = {"hist_kernel", "scan_kernel",    "scatter_kernel",
                                                "cc_kernel",   "offsets_kernel", "copy_kernel"};

// Launch `kern` on `stream` as a programmatic dependent of the kernel before it.
template <typename K>
cudaError_t launch_dependent(K kern, unsigned grid, unsigned block, size_t smem, cudaStream_t stream, const Launch &L)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, L);
}

cudaError_t launch_reconstruct(const Launch &L, cudaStream_t stream, uint64_t *kernel_count, cudaEvent_t *marks)
{
    NvtxRange range("hp_launch_reconstruct");
    cudaError_t err = cudaMemsetAsync(L.ws.ctl, 0, L.ws.zero_bytes, stream);
    if (err != cudaSuccess) return err;
    auto mark = [&](int i) {
        if (marks && err == cudaSuccess) err = cudaEventRecord(marks[i], stream);
    };
    uint64_t nk = 0;
    const uint64_t nchunks = (L.N + kChunk - 1) / kChunk;
    // persistent histogram and scatter over the same contiguous ranges
    const unsigned hist_grid = bucket_grid(L.N, L.sm_count), scat_grid = hist_grid; // the same ranges
    mark(0);
    if (L.N > 0) {
        hist_kernel<<<hist_grid, kHistThreads, kHistCap * sizeof(uint32_t), stream>>>(L);
        ++nk;
    }
    mark(1);
    if (err == cudaSuccess) err = launch_dependent(scan_kernel, L.E, 256, 0, stream, L);
    ++nk;
    mark(2);
    if (L.N > 0) {
        if (err == cudaSuccess) err = launch_dependent(scatter_kernel, scat_grid, kHistThreads, kScatterSmem, stream, L);
        ++nk;
    }
    mark(3);
    const size_t cc_smem = cc_smem_bytes(L.g.R, L.g.C, L.tune.tile_slots);
    if (err == cudaSuccess) {
        const bool hash = L.tune.label_store == kStoreHash;
        if (L.tune.blocks_per_sm >= 3)
            err = launch_dependent(hash ? cc_kernel<3, true> : cc_kernel<3, false>, L.cc_grid, kCCThreads, cc_smem,
                                   stream, L);
        else if (L.tune.blocks_per_sm == 1)
            err = launch_dependent(hash ? cc_kernel<1, true> : cc_kernel<1, false>, L.cc_grid, kCCThreads, cc_smem,
                                   stream, L);
        else
            err = launch_dependent(hash ? cc_kernel<2, true> : cc_kernel<2, false>, L.cc_grid, kCCThreads, cc_smem,
                                   stream, L);
    }
    ++nk;
    mark(4);
    const uint64_t EM = (uint64_t)L.E * L.g.M;
    if (err == cudaSuccess)
        err = launch_dependent(offsets_kernel, (unsigned)((EM + kOffItems - 1) / kOffItems), kOffThreads, 0, stream, L);
    ++nk;
    mark(5);
    {   // a warp per output chunk (at most copy_grid blocks, looping), and a thread per event status and offset
        const uint64_t by_items = (L.N / kOutChunk + 1 + kCopyThreads / 32 - 1) / (kCopyThreads / 32);
        const uint64_t by_events = ((uint64_t)L.E + kCopyThreads) / kCopyThreads; // E + 1 offsets
        const uint64_t blocks =
            std::max<uint64_t>(1, std::max<uint64_t>(by_events, std::min<uint64_t>(by_items, (uint64_t)L.copy_grid)));
        if (err == cudaSuccess) err = launch_dependent(copy_kernel, (unsigned)blocks, kCopyThreads, 0, stream, L);
    }
    ++nk;
    mark(6);
    if (kernel_count) *kernel_count += nk;
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

} // namespace hp
