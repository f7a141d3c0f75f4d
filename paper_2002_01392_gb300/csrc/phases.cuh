// Kernels are written as a sequence of phase functions separated by block
// barriers.  On the device the phases run inside one __global__ function; the
// host-check library runs the same phase functions sequentially over every
// thread of every block on the CPU (barrier = end of a phase), which lets the
// index arithmetic be verified against the oracle without a GPU.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <type_traits>
#include <vector>
#include "fft_reg.cuh"

#if defined(__CUDACC__)
#define FC_HD __host__ __device__ __forceinline__
#else
#define FC_HD inline
#endif

namespace fcns {

// Kernels may declare a loop section: phases [LB, LE) are repeated NIT times
// with a runtime iteration index (one copy of their code), between the
// prologue phases [0, LB) and the epilogue phases [LE, NPHASE).  Such kernels
// define phase<P>(a, smem, tid, bid, it, regs).
template <class K, class = void>
struct LoopSpec {
  static constexpr bool on = false;
  static constexpr int LB = K::NPHASE, LE = K::NPHASE, NIT = 0;
};
template <class K>
struct LoopSpec<K, std::void_t<decltype(K::NIT)>> {
  static constexpr bool on = true;
  static constexpr int LB = K::LB, LE = K::LE, NIT = K::NIT;
};

template <class K, int P>
FC_HD void call_phase(const typename K::Args& a, unsigned char* sm, int tid, long long bid, int it,
                      typename K::Regs& r) {
  if constexpr (LoopSpec<K>::on) K::template phase<P>(a, sm, tid, bid, it, r);
  else K::template phase<P>(a, sm, tid, bid, r);
}

#ifndef FC_HOSTCHECK
template <class K>
__global__ void __launch_bounds__(K::THREADS, K::MINB) phased_kernel(const typename K::Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename K::Regs r;
  using LS = LoopSpec<K>;
  if constexpr (!LS::on) {
    SFor<0, K::NPHASE>::run([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      if constexpr (p > 0) __syncthreads();
      K::template phase<p>(a, smem_raw, (int)threadIdx.x, (long long)blockIdx.x, r);
    });
  } else {
    const int tid = (int)threadIdx.x;
    const long long bid = (long long)blockIdx.x;
    SFor<0, LS::LB>::run([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      if constexpr (p > 0) __syncthreads();
      K::template phase<p>(a, smem_raw, tid, bid, 0, r);
    });
#pragma unroll 1
    for (int it = 0; it < LS::NIT; ++it) {
      SFor<LS::LB, LS::LE>::run([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        __syncthreads();
        K::template phase<p>(a, smem_raw, tid, bid, it, r);
      });
    }
    SFor<LS::LE, K::NPHASE>::run([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      __syncthreads();
      K::template phase<p>(a, smem_raw, tid, bid, 0, r);
    });
  }
}
#endif

// CPU execution of the same phases (host-check builds only).
// Race and initialisation checks of the emulation: threads of a phase run in
// ascending (order 0) or descending (order 1) thread index, and with poison
// set, shared memory is filled with 0xFF bytes (NaN as float and double) at
// the start of every block.  A kernel whose threads exchange shared-memory
// data without a barrier in between, or read shared memory that their block
// has not written, gives different results under the two settings.
inline int& emu_order() { static int v = 0; return v; }
inline int& emu_poison() { static int v = 0; return v; }

template <class K>
void phased_emulate(const typename K::Args& a, long long grid, size_t smem_bytes) {
  std::vector<unsigned char> smem(smem_bytes > 16 ? smem_bytes : 16);
  std::vector<typename K::Regs> regs(K::THREADS);
  using LS = LoopSpec<K>;
  const bool rev = emu_order() != 0;
  auto th = [&](int t) { return rev ? K::THREADS - 1 - t : t; };
  for (long long b = 0; b < grid; ++b) {
    if (emu_poison()) std::fill(smem.begin(), smem.end(), (unsigned char)0xFF);
    SFor<0, LS::LB>::run([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      for (int t = 0; t < K::THREADS; ++t) call_phase<K, p>(a, smem.data(), th(t), b, 0, regs[th(t)]);
    });
    if constexpr (LS::on) {
      for (int it = 0; it < LS::NIT; ++it)
        SFor<LS::LB, LS::LE>::run([&](auto pc) {
          constexpr int p = decltype(pc)::value;
          for (int t = 0; t < K::THREADS; ++t) call_phase<K, p>(a, smem.data(), th(t), b, it, regs[th(t)]);
        });
      SFor<LS::LE, K::NPHASE>::run([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        for (int t = 0; t < K::THREADS; ++t) call_phase<K, p>(a, smem.data(), th(t), b, 0, regs[th(t)]);
      });
    }
  }
}

}  // namespace fcns
