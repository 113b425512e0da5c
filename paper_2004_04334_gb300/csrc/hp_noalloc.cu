// hp_reconstruct_device_noalloc: the device-resident reconstruction for
// callers that cannot allocate device memory.
//
// Its scratch (the workspace that hp_reconstruct_device takes from a
// per-stream cudaMalloc) is a fixed file-scope device array instead, so a
// call allocates nothing: no cudaMalloc, cudaFree or allocating library
// routine.  The array is part of this library's device image: every GPU on
// which the library is used holds kScratchBytes of it until the process
// exits.
#include <mutex>

#include "hp.h"
#include "hp_internal.h"

namespace {

// Largest call the fixed scratch serves.
constexpr uint64_t kMaxDigis = 131072; // digis per call (all events together)
constexpr uint64_t kMaxItems = 16384;  // events * modules per call
constexpr int kMaxGrid = 152;          // clustering blocks (one per SM of a GB300)
constexpr size_t kScratchBytes = 24u << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on `device` (current), looked up once per
// device (and kept for the process: after a cudaDeviceReset the module is
// reloaded elsewhere, so the entry point must not be used after a reset).
// In host code g_scratch names a host-side stand-in, never the device memory
// itself.
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_scratch);
        if (err != cudaSuccess) return err;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

} // namespace

extern "C" hp_status hp_reconstruct_device_noalloc(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis,
                                                   const uint64_t *d_offsets, const uint32_t *d_words,
                                                   const uint16_t *d_module_ids, const hp_device_clusters *out,
                                                   void *stream)
{
    // the same argument checks as hp_reconstruct_device (a failed context
    // reports HP_ECUDA)
    const int chk = hp::check_device_call(ctx, n_events, n_digis, d_offsets, d_words, d_module_ids, out);
    if (chk != HP_OK) return (hp_status)chk;
    hp::Geometry g;
    int device = 0, grid = 0, sms = 0;
    if (!hp::context_launch_params(ctx, &g, &device, &grid, &sms)) return HP_ECUDA;
    if (device < 0 || device >= kMaxDevices) return HP_EINVAL;
    const uint64_t items = (uint64_t)n_events * g.M;
    if (n_digis > kMaxDigis || items > kMaxItems) return HP_ECAPACITY;
    const uint64_t groups = (items + hp::kGroup - 1) / hp::kGroup;
    grid = (int)(groups < (uint64_t)grid ? groups : (uint64_t)grid);
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) grid = 1;
    const hp::Tuning tune; // the default tuning: the scratch limits are sized for it
    if (hp::carve_workspace(nullptr, n_events, g.M, n_digis, g.R, g.C, grid, tune, nullptr, sms) > kScratchBytes)
        return HP_ECAPACITY;
    if (cudaSetDevice(device) != cudaSuccess) return (hp_status)hp::context_fail(ctx);
    void *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) {
        cudaGetLastError();
        return (hp_status)hp::context_fail(ctx);
    }
    hp::Launch L;
    L.g = g;
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
    hp::carve_workspace(base, n_events, g.M, n_digis, g.R, g.C, grid, tune, &L.ws, sms);
    L.cc_grid = grid;
    L.copy_grid = 4 * grid;
    L.sm_count = sms;
    L.tune = tune;
    uint64_t nk = 0;
    if (hp::launch_reconstruct(L, static_cast<cudaStream_t>(stream), &nk, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return (hp_status)hp::context_fail(ctx); // as hp_reconstruct_device: the context is failed
    }
    return HP_OK;
}
