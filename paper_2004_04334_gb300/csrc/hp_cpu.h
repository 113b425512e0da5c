// The CPU case of libhp (Sec. 3): the reconstruction on the host's cores,
// for contexts without a usable GPU.  Shares no code with the CUDA path or
// with the test oracle.
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace hp {
namespace cpu {

struct Geometry {
    uint32_t M, R, C;
    int32_t pixel_thr, cluster_thr;
    const int32_t *gain, *ped; // host [M]
};

// Host output arrays, capacity n_digis for the six cluster columns.
struct Outputs {
    uint32_t *module;
    int32_t *id, *charge, *npix;
    float *x, *y;
    uint64_t *cluster_offsets;     // [E + 1]
    int32_t *event_status;         // [E] hp_status
    int32_t *label = nullptr;      // [N] cluster id, -1, -2 (or null)
    uint16_t *label16 = nullptr;   // [N] rank in the module, 0xFFFF, 0xFFFE (or null)
    uint32_t *item_first = nullptr; // [E * M] with label16
};

// A fixed set of host threads running one parallel loop at a time.
class ThreadPool {
  public:
    explicit ThreadPool(unsigned n = 0); // 0: one per hardware thread
    ~ThreadPool();
    unsigned size() const { return (unsigned)workers_.size(); }
    // fn(i, worker) for every i < n, spread over the workers; returns when all are done
    void parallel_for(uint64_t n, const std::function<void(uint64_t, unsigned)> &fn);

  private:
    void loop(unsigned self);
    void work(unsigned self);
    std::vector<std::thread> workers_;
    std::mutex mu_, call_mu_;
    std::condition_variable cv_, done_;
    const std::function<void(uint64_t, unsigned)> *fn_ = nullptr;
    uint64_t n_ = 0, gen_ = 0;
    std::atomic<uint64_t> next_{0};
    unsigned busy_ = 0;
    bool stop_ = false;
};

// Reconstruct E events (event e owns digis [offsets[e], offsets[e+1]) of
// words/modules) into o.  Blocking; runs its loops on `pool`.
void reconstruct(const Geometry &g, uint32_t E, const uint64_t *offsets, const uint32_t *words,
                 const uint16_t *modules, const Outputs &o, ThreadPool &pool);

} // namespace cpu
} // namespace hp
