// Host-side helpers shared by the launchers (internal).
#pragma once

#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

namespace cgh {

// A setting that CUDA keeps per device (a kernel's shared-memory limit): set() runs once for each device it is
// launched on, with that device current, under a lock, and again after a failure.
class PerDeviceOnce {
  public:
    template <class F>
    cudaError_t run(F set)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(m_);
        if (dev >= 0 && dev < 64 && ((done_ >> dev) & 1ull)) return cudaSuccess;
        e = set();
        if (e == cudaSuccess && dev >= 0 && dev < 64) done_ |= 1ull << dev;
        return e;
    }

  private:
    std::mutex m_;
    uint64_t done_ = 0;
};

}  // namespace cgh
