// Transfer on demand (Sec. 4.3): results kept in device memory reach the
// host only when a transfer consumer asks for them, and then only the
// clusters that exist.  The copy runs as a kernel writing mapped pinned host
// memory over NVLink-C2C, because the number of clusters is known only on
// the device: a cudaMemcpyAsync would have to move the whole capacity.
#include "hp_internal.h"

namespace hp {

namespace {

constexpr int kCopyThreads = 256;

__global__ void __launch_bounds__(kCopyThreads) copy_out_kernel(const Outputs src, const Outputs dst, uint32_t E,
                                                                 bool clusters)
{
    uint64_t n = clusters ? src.cluster_offsets[E] : 0;
    if (n > src.capacity) n = src.capacity;
    const uint64_t span = n > (uint64_t)E + 1 ? n : (uint64_t)E + 1;
    const uint64_t stride = (uint64_t)gridDim.x * kCopyThreads;
    for (uint64_t i = (uint64_t)blockIdx.x * kCopyThreads + threadIdx.x; i < span; i += stride) {
        if (i <= E) dst.cluster_offsets[i] = src.cluster_offsets[i];
        if (i < E) dst.event_status[i] = src.event_status[i];
        if (i < n) {
            dst.module[i] = src.module[i];
            dst.id[i] = src.id[i];
            dst.charge[i] = src.charge[i];
            dst.npix[i] = src.npix[i];
            dst.x[i] = src.x[i];
            dst.y[i] = src.y[i];
        }
    }
}

} // namespace

cudaError_t launch_copy_out(const Outputs &src, const Outputs &dst, uint32_t E, bool clusters, int max_blocks,
                            cudaStream_t stream)
{
    const uint64_t span = (clusters && src.capacity > (uint64_t)E + 1) ? src.capacity : (uint64_t)E + 1;
    uint64_t blocks = (span + kCopyThreads - 1) / kCopyThreads;
    if (blocks > (uint64_t)max_blocks) blocks = (uint64_t)max_blocks;
    if (blocks < 1) blocks = 1;
    copy_out_kernel<<<(unsigned)blocks, kCopyThreads, 0, stream>>>(src, dst, E, clusters);
    return cudaGetLastError();
}

} // namespace hp
