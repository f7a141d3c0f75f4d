// Device launch of a phased kernel (included by the kernel translation units,
// which instantiate DevRun for every kernel / shape they own).
#pragma once
#include <atomic>
#include <climits>

#include "internal.hpp"
#include "phases.cuh"

namespace fcns {

template <class K>
struct DevRun {
  static fc_status run(const typename K::Args& a, long long grid, cudaStream_t s);
};

template <class K>
fc_status DevRun<K>::run(const typename K::Args& a, long long grid, cudaStream_t s) {
  if constexpr (K::smem_bytes > 227 * 1024) {
    set_error("kernel shape exceeds the shared-memory budget");
    return FC_ERR_UNSUPPORTED;
  } else {
    if (grid <= 0) return FC_OK;
    if (grid > INT_MAX) return FC_ERR_UNSUPPORTED;
    auto kern = phased_kernel<K>;
    // the shared-memory attribute once per device (not inside every launch, so
    // that launches can also be captured into CUDA graphs)
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !(attr_set.load() >> dev & 1ull)) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes);
      if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute");
      if (dev < 64) attr_set.fetch_or(1ull << dev);
    }
    kern<<<(unsigned)grid, K::THREADS, K::smem_bytes, s>>>(a);
    return cuda_status(cudaGetLastError(), "kernel launch");
  }
}

}  // namespace fcns
