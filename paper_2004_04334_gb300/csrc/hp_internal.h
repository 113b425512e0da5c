// Internal interface between the libhp host runtime and its sm_103a kernels.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

struct hp_ctx;

namespace hp {

// NVTX range around a host-side stage (visible to Nsight tools, e.g.
// `ncu --nvtx`; costs nothing measurable when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Error bits accumulated on the device (per event, and per launch).
constexpr uint32_t kErrBadDigi = 1u;
constexpr uint32_t kErrDup = 2u;
constexpr uint32_t kErrCapacity = 4u;
constexpr uint32_t kErrTimeout = 8u;
constexpr uint32_t kErrBadOffsets = 16u; // event offsets not 0 = o[0] <= o[1] <= ... <= o[E] = N (launch-wide)

// Tuning constants of the kernels.
constexpr int kChunk = 4096;         // digis per histogram / scatter block
constexpr int kHistThreads = 512;
constexpr int kHistCap = 4096;       // (event, module) bins a block can histogram in shared memory
constexpr int kCCThreads = 512;      // threads of a clustering block
constexpr int kGroup = kCCThreads / 32; // most (event, module) items per work-queue ticket, one per warp
constexpr int kWarpMax = 64;         // items with at most this many digis are clustered by one warp
constexpr int kSmemSlots = 4096;     // digis of an item a block clusters in shared memory (default tile)
constexpr int kMaxTileSlots = 16384; // largest tile considered (one block per SM)

// Launch parameters of the clustering kernel, chosen per launch shape by the
// autotuner (defaults: the values above, two resident blocks per SM).
struct Tuning {
    uint32_t tile_slots = kSmemSlots; // block-tier capacity in shared memory; larger items use global scratch
    uint32_t blocks_per_sm = 2;       // 1 (largest tile), 2 (up to 64 registers a thread) or 3 (up to 40, smaller tile)
    uint32_t ticket_max = kGroup;     // items per ticket before halving for small launches (<= kGroup)
    uint32_t warp_max = kWarpMax;     // 32 or 64: largest item of the warp tier
    uint32_t label_store = 0;         // kStoreBitmap or kStoreHash: pixel lookup of the items above the warp tier
    uint32_t item_threads = kCCThreads; // threads clustering one item of the hash store: 128, 256 or 512
};

// Pixel lookup of the clustering items above the warp tier: module-sized
// occupancy and survivor bitmaps (one block an item), or an open-addressing
// hash table keyed by linear pixel index, sized by the item's digi count
// (item_threads threads an item, several items of a block side by side).
constexpr uint32_t kStoreBitmap = 0;
constexpr uint32_t kStoreHash = 1;
// Digi index bits of the hash store's packed keys (items of at most 4096 digis).
constexpr uint32_t kHashIdxBits = 12;

// Digis a clustering thread holds in registers in the register tier and
// the hash store: fewer at three resident blocks per SM (40 registers).
__host__ __device__ constexpr int cc_digis_per_thread(int blocks_per_sm) { return blocks_per_sm >= 3 ? 5 : 8; }

// Largest item (digis) of the hash store: each of the block's
// kCCThreads / item_threads groups takes an equal 16-byte-aligned slice of
// the clustering kernel's dynamic shared memory (`smem` bytes) for 28 bytes
// a digi (accumulators, parent, two table slots) plus 256 row counters, and
// a slice of the block's 64-bit moment scratch (2 * tile_slots entries);
// each thread holds at most `per_thread` digis in registers.
__host__ __device__ inline uint32_t hash_capacity(size_t smem, uint32_t tile_slots, uint32_t item_threads,
                                                  uint32_t per_thread)
{
    const uint32_t groups = (uint32_t)kCCThreads / item_threads;
    const size_t slice = (smem / groups) & ~(size_t)15;
    size_t cap = slice > 1024 ? (slice - 1024) / 28 : 0;
    if (cap > tile_slots / groups) cap = tile_slots / groups;
    if (cap > (size_t)per_thread * item_threads) cap = (size_t)per_thread * item_threads;
    if (cap > (1u << kHashIdxBits)) cap = 1u << kHashIdxBits;
    return (uint32_t)cap;
}

// Whether a launch of N digis in EM items has block-tier items on average
// (64 digis or more an item) rather than warp-tier ones.
__host__ __device__ inline bool large_items(uint64_t N, uint64_t EM) { return N >= 64ull * EM; }

// Items per work-queue ticket of a launch of EM items on `grid` clustering
// blocks: `gmax`, halved while a launch would have too few tickets per
// block.  Warp-tier items (small on average) keep at least four a ticket, so
// that a block's warps work on several at once, and want two tickets a
// block; block-tier items go down to one a ticket and want four a block, so
// that a small launch's large items spread over blocks instead of queueing
// in one ticket (one per block: the grid is sized to match, see the runtime).
__host__ __device__ inline uint32_t ticket_items(uint64_t EM, unsigned grid, uint32_t gmax, uint64_t N)
{
    const bool large = large_items(N, EM);
    const uint32_t least = large ? 1u : 4u;
    const uint64_t want = (large ? 4ull : 2ull) * grid;
    uint32_t g = gmax;
    while (g > least && (EM + g - 1) / g < want) g >>= 1;
    return g;
}

// Clusters parked between the clustering kernel and the ordered write, as
// structure-of-arrays indexed by bucket position: item i's k-th kept cluster
// (in id order) sits at boff[i] + k.
struct Staging {
    int32_t *id, *charge, *npix;
    float *x, *y;
    __device__ __forceinline__ void put(uint64_t at, int32_t id_, int32_t q, int32_t np_, float x_, float y_) const
    {
        id[at] = id_;
        charge[at] = q;
        npix[at] = np_;
        x[at] = x_;
        y[at] = y_;
    }
};

struct Geometry {
    uint32_t M, R, C;
    int32_t pixel_thr, cluster_thr;
    const int32_t *gain; // device [M]
    const int32_t *ped;  // device [M]
};

// The six per-cluster output columns.
struct ClusterCols {
    uint32_t *module;
    int32_t *id, *charge, *npix;
    float *x, *y;
};

struct Outputs {
    uint64_t capacity;
    uint32_t *module;
    int32_t *id, *charge, *npix;
    float *x, *y;
    uint64_t *cluster_offsets; // [E+1]
    int32_t *label;            // [N] or null
    int32_t *event_status;     // [E] written by copy_kernel
    // compact labels, instead of `label` (cc_kernel): each digi's cluster as
    // its rank among the kept clusters of its (event, module) item, 0xFFFF
    // below the pixel threshold, 0xFFFE in a cluster below the cluster
    // threshold; and (copy_kernel) each item's first cluster counted from its
    // event's first
    uint16_t *label16 = nullptr;    // [N] or null
    uint32_t *item_first = nullptr; // [E*M] (with label16)
    // Outputs in mapped host memory: positions below head_n go to these
    // device columns instead (16-byte aligned), which the launch then copies
    // to the host columns by DMA, so that the copy engine, not the SMs,
    // carries them over the host link; the positions from head_n on (the
    // launch cannot know the cluster count in advance) go straight to host.
    ClusterCols head{};
    uint32_t head_n = 0;
};

// Output positions a copy_kernel warp writes per step (four a lane).
constexpr uint32_t kOutChunk = 128;

// Scratch of one launch.  The first `zero_bytes` bytes must be zero before
// the first kernel (one memset): control words, per-event error bits,
// per-item counts and the chained-scan state.
struct Workspace {
    uint32_t *ctl;        // [16]: 0 item ticket, 1 launch error bits, 2 arena bump, 3 prefix frontier,
                          //       4 offsets chunk ticket, 6 clusters of the launch (offsets_kernel)
    uint32_t *event_err;  // [E]
    uint32_t *count;      // [E*M] digis of each item (reserved part, then the total: scan_kernel);
                          //       then each item's first output position (offsets_kernel)
    uint32_t *count2;     // [E*M] digis of histogram ranges with many keys (placed step by step)
    unsigned long long *chain; // [2 * n_chunks]: offsets_kernel chunk totals, then inclusive prefixes
    size_t zero_bytes;
    uint32_t *boff;       // [E*M] bucket start of each item
    uint32_t *blk_off;    // [bucket_grid * kHistCap] each histogram block's offset inside each key's bucket
    uint32_t *cursor;     // [E*M] scatter cursor of the step-by-step part; then each item's count of kept
                          //       clusters (cc_kernel)
    uint32_t *bucket_w;   // [N]
    uint32_t *bucket_i;   // [N] index of the digi within its event
    Staging staging;      // [N] each array
    uint32_t *chunk_item; // [N / kOutChunk + 2] item holding the first position of each output chunk
    unsigned long long *exact; // [cc_grid * 2 * tile_slots] 64-bit moments of heavy clusters
    unsigned char *big;   // scratch of items too large for shared memory
    uint64_t big_slots;   // slots per block (slab mode) or in total (arena mode)
    int big_arena;        // 1: bump-allocated arena, 0: one slab per block
};

struct Launch {
    Geometry g;
    uint32_t E;
    uint64_t N;
    const uint64_t *offsets; // device [E+1]
    const uint32_t *words;   // device [N]
    const uint16_t *modules; // device [N]
    Outputs out;
    Workspace ws;
    int cc_grid;             // blocks of the clustering kernel
    int copy_grid = 1216;    // most blocks of the output copy (8 an SM of a 152-SM GPU)
    int sm_count = 152;      // SMs of the device (grids of the persistent histogram and scatter)
    Tuning tune;
    uint32_t debug = 0;      // test hooks (kDebug*)
};

// Test hook: offsets_kernel never publishes chunk 0's cluster count,
// so the bounded waits of the ordered output expire and the launch reports
// HP_ETIMEOUT (the wait's limit is one second).
constexpr uint32_t kDebugWithholdTicket0 = 1u;

// Blocks of the persistent histogram and scatter kernels (the same
// contiguous digi ranges in both): two an SM, at least one kChunk a block.
__host__ __device__ inline unsigned bucket_grid(uint64_t N, int sm_count)
{
    const uint64_t chunks = (N + kChunk - 1) / kChunk;
    const uint64_t cap = 2ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    return (unsigned)(chunks < 1 ? 1 : (chunks < cap ? chunks : cap));
}

// Bytes of one global-tier slot: (Q, npix), two 64-bit and two 32-bit moments,
// parent, padded to 8-byte multiples so every slot range stays 8-byte aligned.
constexpr size_t kBigSlotBytes = 8 + 16 + 8 + 4 + 4;

// Dynamic shared memory of a clustering block: the tile's slot arrays (charge,
// count, 32-bit moments, parent: 20 bytes a slot), then the occupancy and
// survivor bitmaps and the survivor prefix (a word each per 32 pixels).
__host__ __device__ inline size_t cc_smem_bytes(uint32_t R, uint32_t C, uint32_t tile_slots)
{
    const size_t nwords = ((size_t)R * C + 31) / 32;
    return (size_t)tile_slots * (8 + 8 + 4) + nwords * 4 * 3;
}
// Lay out the workspace for (E, M, N) in `base` (nullptr: only compute size).
size_t carve_workspace(void *base, uint32_t E, uint32_t M, uint64_t N, uint32_t R, uint32_t C, int cc_grid,
                       const Tuning &tune, Workspace *ws, int sm_count);
// Configure kernel attributes once per device.  max_tile[b] receives the
// largest tile (slots) with which b clustering blocks stay resident per SM
// (0 if b blocks cannot be resident), for b = 1, 2 and 3 (at most
// kMaxTileSlots for one block, kSmemSlots otherwise); max_tile[0] unused.
// hash_tile[b] receives the same for the kernel's hash-store instance.
cudaError_t init_kernels(int device, uint32_t R, uint32_t C, uint32_t max_tile[4], uint32_t hash_tile[4]);
// Kernels of one launch, in order; marks[i] (if given) is recorded before
// kernel i and marks[kNumKernels] after the last one.
constexpr int kNumKernels = 6;
extern const char *const kKernelNames[kNumKernels];
// Queue the whole reconstruction of one launch on `stream` (memset + kernels).
cudaError_t launch_reconstruct(const Launch &L, cudaStream_t stream, uint64_t *kernel_count,
                               cudaEvent_t *marks = nullptr);

// One request of a serving batch: its inputs in (mapped) pinned host memory
// and where they go in the batch's device arrays.
struct GatherEntry {
    const uint32_t *words;
    const uint16_t *modules;
    uint64_t n;
    uint64_t off;
};
// Copy every request's inputs into the batch's device arrays (reads the host
// buffers over the C2C link; `table` must be device-accessible).
cudaError_t launch_gather(const GatherEntry *table, uint32_t n_requests, uint64_t max_n, uint32_t *words,
                          uint16_t *modules, cudaStream_t stream);

// Module placement for the clusters -> hits step, as the device holds it:
// per module three affine rows (r_i0, r_i1, o_i, 0), i = x, y, z, so that
// a hit is row_i . (u, v, 1).  Only the first two rotation columns matter
// because the local point has w = 0.
struct Placement {
    const float4 *rows;  // [3 * M]
    uint32_t M;
    float pitch_row, pitch_col;
    float half_rows, half_cols; // (rows - 1) / 2 and (cols - 1) / 2: the module centre in pixel units
};

// One hits launch: clusters in, hits out (all device-accessible pointers).
struct HitsLaunch {
    Placement p;
    uint32_t E;
    uint64_t capacity;                 // room in the cluster and hit arrays
    const uint64_t *cluster_offsets;   // [E + 1]
    const int32_t *event_status;       // [E] or null
    const uint32_t *module;            // [capacity]
    const float *x, *y;                // [capacity] centroids (pixel units)
    uint64_t *hit_offsets;             // [E + 1] or null: copy of cluster_offsets
    int32_t *hit_status;               // [E] or null: copy of event_status
    uint32_t *hit_module;              // [capacity] or null: copy of module
    float *hx, *hy, *hz;               // [capacity] global position
};
// Queue the hits kernel on `stream` (grid-stride; the cluster count is read
// on the device, so nothing waits for the clusters to exist).
cudaError_t launch_hits(const HitsLaunch &h, int max_blocks, cudaStream_t stream);

// Transfer on demand: copy a product's outputs (`src`, device memory) to
// `dst` (mapped pinned host memory): cluster offsets and event statuses
// always, and, if `clusters`, the cluster arrays of the clusters that exist
// (their count is read on the device, so only those bytes cross the link).
cudaError_t launch_copy_out(const Outputs &src, const Outputs &dst, uint32_t E, bool clusters, int max_blocks,
                            cudaStream_t stream);

// Launch parameters of a context (implemented by the runtime): geometry with
// device calibration pointers, device ordinal, clustering grid size and SM
// count; false if the context has failed.
bool context_launch_params(hp_ctx *ctx, Geometry *g, int *device, int *cc_grid, int *sm_count);
// Argument checks shared by the device-resident entry points: 0 (HP_OK) or
// the hp_status to return.
int check_device_call(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                      const uint32_t *d_words, const uint16_t *d_module_ids, const struct hp_device_clusters *out);
// Mark the context failed after a CUDA error (every later call reports
// HP_ECUDA); returns HP_ECUDA.
int context_fail(hp_ctx *ctx);

} // namespace hp
