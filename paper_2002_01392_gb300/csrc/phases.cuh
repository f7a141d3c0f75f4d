// Kernels are written as a sequence of phase functions separated by block
// barriers.  On the device the phases run inside one __global__ function; the
// host-check library runs the same phase functions sequentially over every
// thread of every block on the CPU (barrier = end of a phase), which lets the
// index arithmetic be verified against the oracle without a GPU.
#pragma once
#include <cuda_runtime.h>
#include <vector>
#include "fft_reg.cuh"

#if defined(__CUDACC__)
#define FC_HD __host__ __device__ __forceinline__
#else
#define FC_HD inline
#endif

namespace fcns {

#ifndef FC_HOSTCHECK
template <class K>
__global__ void __launch_bounds__(K::THREADS, K::MINB) phased_kernel(const typename K::Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename K::Regs r;
  SFor<0, K::NPHASE>::run([&](auto pc) {
    constexpr int p = decltype(pc)::value;
    if constexpr (p > 0) __syncthreads();
    K::template phase<p>(a, smem_raw, (int)threadIdx.x, (long long)blockIdx.x, r);
  });
}
#endif

// CPU execution of the same phases (host-check builds only).
template <class K>
void phased_emulate(const typename K::Args& a, long long grid, size_t smem_bytes) {
  std::vector<unsigned char> smem(smem_bytes + 16);
  std::vector<typename K::Regs> regs(K::THREADS);
  for (long long b = 0; b < grid; ++b) {
    SFor<0, K::NPHASE>::run([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      for (int t = 0; t < K::THREADS; ++t) K::template phase<p>(a, smem.data(), t, b, regs[t]);
    });
  }
}

}  // namespace fcns
