// Typed launcher of the fc_deriv_z kernels (one translation unit per
// precision instantiates it: the kernels of all compiled lengths).
#pragma once
#include <atomic>
#include <cstdint>

#include "deriv_kernel.cuh"
#include "internal.hpp"

namespace fcns {


template <class T, int L1, int L2, int LINES, int JN, bool SYM, int JI = 0, bool FULL = false>
fc_status run_deriv(const DerivDevTables& t, const PlanData& p, int batch, long long lines, double Lz,
                    const void* f, void* df, void* d2f, cudaStream_t stream) {
  using K = DerivPair<T, L1, L2, LINES, JN, SYM, JI, FULL>;
  static_assert(K::smem_bytes <= 227 * 1024, "shared memory budget");
  typename K::Args a;
  a.f = static_cast<const T*>(f);
  a.df = static_cast<T*>(df);
  a.d2f = static_cast<T*>(d2f);
  a.Nz = p.Nz; a.Np = p.Np; a.d = p.d; a.Cc = p.C;
  a.lines = lines;
  a.pairs = (lines + 1) / 2;
  a.tiles = (a.pairs + LINES - 1) / LINES;
  a.zstride = lines;
  a.bstride = lines * p.Nz;
  const double dz = Lz / (p.Nz - 1);
  a.s1 = T(1.0 / dz);
  a.s2 = T(1.0 / (dz * dz));
  a.Mr = t.Mr;
  a.Mr2 = t.Mr2;
  a.H1 = static_cast<const cx<T>*>(sizeof(T) == 4 ? t.H1_32 : t.H1_64);
  a.H2 = static_cast<const cx<T>*>(sizeof(T) == 4 ? t.H2_32 : t.H2_64);
  a.tw = static_cast<const cx<T>*>(sizeof(T) == 4 ? t.tw32 : t.tw64);
  auto kern = phased_kernel<K>;
  // the shared-memory attribute once per device (launches may be graph-captured)
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set.load() >> dev & 1ull)) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes);
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(fc_deriv_z)");
    if (dev < 64) attr_set.fetch_or(1ull << dev);
  }
  const long long grid = a.tiles * batch;
  if (grid > 0x7fffffffLL) return FC_ERR_UNSUPPORTED;
  // L2 prefetch of the block one residency ahead: measured +27 % for the
  // length-512 transforms and -7 % for 1080 on GB300, so only below 1000
  static int sms = 0;
  if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
  a.nblocks = grid;
  // pairs start at even lines: with an even line count (and 2-element aligned
  // arrays, as device allocations are) each pair is one aligned vector
  const uintptr_t al = 2 * sizeof(T);
  a.vec = (lines % 2 == 0 && ((uintptr_t)f | (uintptr_t)df | (uintptr_t)d2f) % al == 0) ? 1 : 0;
  a.pf_dist = (L1 * L2 < 1000) ? (long long)sms * K::MINB : 0;
  kern<<<(unsigned)grid, K::THREADS, K::smem_bytes, stream>>>(a);
  return cuda_status(cudaGetLastError(), "fc_deriv_z launch");
}


template <class T>
fc_status launch_deriv_typed(const DerivDevTables& t, const PlanData& p, int batch, long long lines, double Lz,
                             const void* f, void* df, void* d2f, cudaStream_t stream) {
  constexpr bool F = sizeof(T) == 4;
// the padded case (N' <= L2 (L1/2 + 1)) runs the variant whose upper input
// registers are known zeros; with L >= 2 N' - 1 (or L = N') the kernel
// spectra are purely imaginary / real (symmetric placement, host_tables)
  const bool sym = t.L == p.Np || t.L >= 2 * p.Np - 1;
  // float32 at L = 1080 (the length every Nz from 481 to 551 with C <= 64 is
  // given): register rows 0..12 (n <= 467) lie below Nz - 10 whenever
  // Nz >= 481, so they run without bounds checks (DerivPair JI)
  if constexpr (F) {
    if (t.L == 1080 && sym && p.Np <= 36 * 16 && p.Nz >= 481) {
      // whole tiles of aligned pair vectors: no per-element pair checks (FULL)
      const uintptr_t al = 2 * sizeof(T);
      const bool full = lines % 8 == 0 && ((uintptr_t)f | (uintptr_t)df | (uintptr_t)d2f) % al == 0;
      return full ? run_deriv<T, 30, 36, 4, 16, true, 13, true>(t, p, batch, lines, Lz, f, df, d2f, stream)
                  : run_deriv<T, 30, 36, 4, 16, true, 13>(t, p, batch, lines, Lz, f, df, d2f, stream);
    }
  }
#define FC_CASE(LL, A, B, LF, LD)                                                                          \
  case LL:                                                                                                 \
    if (p.Np <= B * (A / 2 + 1))                                                                           \
      return sym ? run_deriv<T, A, B, F ? LF : LD, A / 2 + 1, true>(t, p, batch, lines, Lz, f, df, d2f, stream) \
                 : run_deriv<T, A, B, F ? LF : LD, A / 2 + 1, false>(t, p, batch, lines, Lz, f, df, d2f, stream); \
    return sym ? run_deriv<T, A, B, F ? LF : LD, A, true>(t, p, batch, lines, Lz, f, df, d2f, stream)       \
               : run_deriv<T, A, B, F ? LF : LD, A, false>(t, p, batch, lines, Lz, f, df, d2f, stream);
  switch (t.L) {
    FC_CASE(64, 8, 8, 16, 8)
    FC_CASE(96, 8, 12, 16, 8)
    FC_CASE(128, 8, 16, 16, 8)
    FC_CASE(160, 10, 16, 16, 8)
    FC_CASE(192, 12, 16, 16, 8)
    FC_CASE(256, 16, 16, 16, 8)
    FC_CASE(288, 16, 18, 16, 8)
    FC_CASE(320, 16, 20, 16, 8)
    FC_CASE(512, 16, 32, 8, 4)
    FC_CASE(576, 24, 24, 8, 4)
    FC_CASE(768, 24, 32, 4, 2)
    FC_CASE(1024, 32, 32, 4, 2)
    FC_CASE(1080, 30, 36, 4, 2)
    FC_CASE(1152, 32, 36, 4, 2)
    FC_CASE(1536, 32, 48, 2, 1)
    default:
      return FC_ERR_UNSUPPORTED;
  }
#undef FC_CASE
}

}  // namespace fcns
