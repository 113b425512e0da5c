// Clusters -> hits (the step after the clusters in the paper's Fig. 1): each
// cluster centroid becomes a global position through its module's placement.
//
// HBM-bound and tiny next to the clustering: per hit it reads module, x and
// y (12 B) and writes three floats (12 B, 16 B with the module copy); the
// placement table (48 B per module, 89 KB for 1856 modules) stays in L1/L2.
// Clusters arrive sorted by module, so neighbouring threads read the same
// placement rows.
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kHitsThreads = 256;

__global__ void __launch_bounds__(kHitsThreads) hits_kernel(HitsLaunch h)
{
    uint64_t n = h.cluster_offsets[h.E];
    if (n > h.capacity) n = h.capacity;
    const uint64_t span = n > (uint64_t)h.E + 1 ? n : (uint64_t)h.E + 1;
    const uint64_t stride = (uint64_t)gridDim.x * kHitsThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kHitsThreads + threadIdx.x; i < span; i += stride) {
        if (h.hit_offsets && i <= h.E) h.hit_offsets[i] = h.cluster_offsets[i];
        if (h.hit_status && h.event_status && i < h.E) h.hit_status[i] = h.event_status[i];
        if (i >= n) continue;
        const uint32_t m = h.module[i];
        float gx = __int_as_float(0x7fc00000), gy = gx, gz = gx; // NaN for a module outside the table
        if (m < h.p.M) {
            const float u = (h.x[i] - h.p.half_rows) * h.p.pitch_row;
            const float v = (h.y[i] - h.p.half_cols) * h.p.pitch_col;
            const float4 rx = __ldg(h.p.rows + 3 * (size_t)m);
            const float4 ry = __ldg(h.p.rows + 3 * (size_t)m + 1);
            const float4 rz = __ldg(h.p.rows + 3 * (size_t)m + 2);
            gx = fmaf(rx.y, v, fmaf(rx.x, u, rx.z));
            gy = fmaf(ry.y, v, fmaf(ry.x, u, ry.z));
            gz = fmaf(rz.y, v, fmaf(rz.x, u, rz.z));
        }
        h.hx[i] = gx;
        h.hy[i] = gy;
        h.hz[i] = gz;
        if (h.hit_module) h.hit_module[i] = m;
    }
}

} // namespace

cudaError_t launch_hits(const HitsLaunch &h, int max_blocks, cudaStream_t stream)
{
    const uint64_t span = (h.capacity > (uint64_t)h.E + 1 ? h.capacity : (uint64_t)h.E + 1);
    uint64_t blocks = (span + kHitsThreads - 1) / kHitsThreads;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    if (blocks < 1) blocks = 1;
    hits_kernel<<<(unsigned)blocks, kHitsThreads, 0, stream>>>(h);
    return cudaGetLastError();
}

} // namespace hp
