// fc_deriv_z: FC-Gram first and second z-derivatives of real fields.
//
// Per z-line (Sec. 3 continuation + Sec. 4.2 spectral derivative): the N'-point
// continued line x = [f; M_r f_last + M_l f_first] is convolved circularly with
// the derivative kernels d1, d2 of the N'-periodic grid.  Only outputs n < Nz
// are needed, so the circular convolution of length N' is computed as a
// circular convolution of length L >= N' + Nz - 1 (forward and inverse FFTs of
// length L, kernel spectra precomputed); when N' itself is a compiled smooth
// length, L = N'.
//
// Thread layout: tid = r * LINES + li, li = line within the tile (lines are
// adjacent in memory, so every global access is coalesced across li).
// FFT of length L = L1 * L2 in two register passes with one shared-memory
// exchange each way (engine.cuh).
#pragma once
#include "phases.cuh"

#if defined(__CUDACC__)
#define DERIV_NOINLINE __host__ __device__ __noinline__
#else
#define DERIV_NOINLINE
#endif

#include "engine.cuh"

namespace fcns {

// float32 input loads cached in L2 only (float64: through L1, measured 11 %
// faster there; the host-check build: a plain load)
template <class X>
FC_HD X ld_stream(const X* p) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same_v<X, float> || std::is_same_v<X, float2>) return __ldcg(p);
  else return *p;
#else
  return *p;
#endif
}

// fc_deriv_z with two adjacent real z-lines packed as one complex line
// x = a + i b.  The derivative kernels d1, d2 of the N'-periodic grid are
// real, so one forward transform X = FFT_L(x) serves both lines and
//   IFFT_L(X H1) = d1*a + i d1*b,   IFFT_L(X H2) = d2*a + i d2*b
// (H1, H2: spectra of d1, d2 placed circularly on L >= N' + Nz - 1, with 1/L):
// three length-L transforms per two lines instead of four.
// JN: registers j >= JN of the input (indices r + L2 j) are known to be zero
// (N' <= L2 JN, the padded case) and no output lies there, so their loads,
// continuation checks and stores are left out at compile time.
// SYM: the kernels sit on the whole window |j| <= N' - 1 (L >= 2 N' - 1, or
// L = N'), so H1 is purely imaginary and H2 purely real: the spectrum
// products are two real multiplies per value instead of a complex multiply.
// JI: register rows j < JI hold only indices n = r + L2 j below Nz - DMAX
// (the launcher picks JI > 0 only when Nz is large enough for that): their
// loads and stores need no bounds check and they hold no continuation or end
// values (row 0 still keeps the first d values).
// FULL: every tile holds LINES whole pairs and every pair is one aligned
// vector (the launcher checks: even line count, a multiple of 2 LINES, aligned
// arrays), so the per-element pair checks are left out.
template <class T, int L1_, int L2_, int LINES_, int JN_ = L1_, bool SYM = false, int JI = 0, bool FULL = false>
struct DerivPair {
  using E = Eng<T, L1_, L2_, LINES_>;
  using C = cx<T>;
  static constexpr int L1 = L1_, L2 = L2_, LINES = LINES_, JN = JN_;
  static_assert(JI <= JN_, "interior rows lie among the loaded rows");
  static constexpr int THREADS = E::THREADS, NPHASE = 4;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  static constexpr int MR_MAX = 640;
  static constexpr int DMAX = 10;

  struct Args {
    const T* f;
    T* df;
    T* d2f;
    int Nz, Np, d, Cc;
    long long lines;      // real lines per field (Nx * Ny)
    long long pairs;      // ceil(lines / 2)
    long long tiles;      // tiles of LINES pairs per field
    long long zstride;    // elements between consecutive z (= lines)
    long long bstride;    // elements between fields
    T s1, s2;             // 1/dz, 1/dz^2
    const double* Mr;
    const float2* Mr2;
    const C* H1;          // spectrum of d1 (natural order, length L)
    const C* H2;          // spectrum of d2
    const C* tw;          // engine twiddles
    long long pf_dist;    // prefetch into L2 the input of block bid + pf_dist (0: off)
    long long nblocks;    // grid size
    int vec;              // 1: every line pair is one aligned 2-element vector (even line count)
  };
  struct Regs { C v[L1]; C u[L2]; };

  // (the continuation matrix is read through the data cache: few threads use it)
  static constexpr size_t off_b1 = sizeof(C) * E::BUF;
  static constexpr size_t off_E = off_b1 + sizeof(C) * E::BUF;
  static constexpr size_t smem_bytes = off_E + sizeof(C) * LINES * 2 * DMAX;

  // continuation value jj of a complex line: M_r f_last + M_l f_first, with
  // compensated sums in both precisions (float-float / double-double)
  static DERIV_NOINLINE C cont_cplx(int jj, const C* first, const C* last, int d, int Cc, const double* Ms,
                                    const float2* Ms2) {
    if constexpr (sizeof(T) == 4) {
      ff re{0.f, 0.f}, im{0.f, 0.f};
      for (int i = 0; i < d; ++i) {
        const float2 m1 = Ms2[jj * d + i];
        const float2 m2 = Ms2[(Cc - 1 - jj) * d + (d - 1 - i)];
        ff_fma(re, m1.x, m1.y, last[i].x);
        ff_fma(im, m1.x, m1.y, last[i].y);
        ff_fma(re, m2.x, m2.y, first[i].x);
        ff_fma(im, m2.x, m2.y, first[i].y);
      }
      return mk<T>(ff_round(re), ff_round(im));
    } else {
      dd re{0.0, 0.0}, im{0.0, 0.0};
      for (int i = 0; i < d; ++i) {
        const double m1 = Ms[jj * d + i], m2 = Ms[(Cc - 1 - jj) * d + (d - 1 - i)];
        dd_fma(re, m1, last[i].x);
        dd_fma(im, m1, last[i].y);
        dd_fma(re, m2, first[i].x);
        dd_fma(im, m2, first[i].y);
      }
      return mk<T>((T)dd_round(re), (T)dd_round(im));
    }
  }

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    C* b1 = reinterpret_cast<C*>(sm + off_b1);
    const double* Ms = a.Mr;
    const float2* Ms2 = a.Mr2;
    const int r = tid / LINES, li = tid % LINES;
    C* Ev = reinterpret_cast<C*>(sm + off_E) + li * 2 * DMAX;
    const long long field = bid / a.tiles;
    const long long pair = (bid % a.tiles) * LINES + li;
    const long long la = 2 * pair;                 // first line of the pair
    const bool va = FULL || la < a.lines, vb = FULL || la + 1 < a.lines;
    const long long base = field * a.bstride + la;

    if constexpr (P == 0) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          if (j >= JN) {
            R.v[j] = mk<T>(0, 0);
            continue;
          }
          const int n = r + L2 * j;
          C x = mk<T>(0, 0);
          if (j < JI || n < a.Nz) {
            // streamed once: cached in L2 only, so that it does not evict the
            // twiddle and spectrum tables from L1
            const T* p = a.f + base + (long long)n * a.zstride;
            if (FULL || a.vec) {
              if (va) x = ld_stream(reinterpret_cast<const C*>(p));
            } else {
              if (va) x.x = ld_stream(p);
              if (vb) x.y = ld_stream(p + 1);
            }
          }
          R.v[j] = x;
          if (j == 0 || j >= JI) {
            if (n < a.d) Ev[n] = x;
            if (j >= JI && n >= a.Nz - a.d && n < a.Nz) Ev[DMAX + n - (a.Nz - a.d)] = x;
          }
        }
      }
    } else if constexpr (P == 1) {
      // the block that will run on this SM about one block-lifetime from now:
      // bring its input rows into L2 while this block computes
      if (a.pf_dist > 0 && bid + a.pf_dist < a.nblocks) {
        const long long b2 = bid + a.pf_dist;
        const long long f2 = b2 / a.tiles, p2 = (b2 % a.tiles) * LINES;
        const T* src = a.f + f2 * a.bstride + 2 * p2;
        for (int n = tid; n < a.Nz; n += THREADS) prefetch_l2(src + (long long)n * a.zstride);
      }
      if (r < L2) {
#pragma unroll
        for (int j = JI; j < JN; ++j) {
          const int n = r + L2 * j;
          if (n >= a.Nz && n < a.Np) R.v[j] = cont_cplx(n - a.Nz, Ev, Ev + DMAX, a.d, a.Cc, Ms, Ms2);
        }
        E::template A<-1>(R.v, b0, a.tw, r, li);
      }
    } else if constexpr (P == 2) {
      if (r < L1) {
        E::template B<-1>(R.u, b0, r, li);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) b1[E::bidx(r, k2, li)] = R.u[k2];
        // the two inverse transforms share one copy of the code (instruction cache)
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          C* bo = o == 0 ? b0 : b1;
          if (o == 1) {
            FC_FENCE();
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) R.u[k2] = b1[E::bidx(r, k2, li)];
          }
          if constexpr (SYM) {
            if (o == 0) E::mulH_imag(R.u, a.H1, r);
            else E::mulH_real(R.u, a.H2, r);
          } else {
            E::mulH(R.u, o == 0 ? a.H1 : a.H2, r);
          }
          E::template Bi<1>(R.u, bo, a.tw, r, li);
        }
      }
    } else if constexpr (P == 3) {
      if (r < L2 && va) {
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          T* out = o == 0 ? a.df : a.d2f;
          if (!out) continue;
          E::template Ai<1>(R.v, o == 0 ? b0 : b1, r, li);
          const T sc = o == 0 ? a.s1 : a.s2;
#pragma unroll
          for (int j = 0; j < JN; ++j) {
            const int n = r + L2 * j;
            if (j < JI || n < a.Nz) {
              T* p = out + base + (long long)n * a.zstride;
              if (FULL || a.vec) {
                *reinterpret_cast<C*>(p) = cscale(R.v[j], sc);
              } else {
                p[0] = R.v[j].x * sc;
                if (vb) p[1] = R.v[j].y * sc;
              }
            }
          }
        }
      }
    }
  }
};

}  // namespace fcns
