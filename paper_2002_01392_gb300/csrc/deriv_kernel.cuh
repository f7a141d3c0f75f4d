// fc_deriv_z: FC-Gram first and second z-derivatives of real fields.
//
// Per z-line (Sec. 3 continuation + Sec. 4.2 spectral derivative): the N'-point
// continued line x = [f; M_r f_last + M_l f_first] is convolved circularly with
// the derivative kernels d1 + i d2 of the N'-periodic grid.  Only outputs
// n < Nz are needed, so the circular convolution of length N' is computed as a
// circular convolution of length L >= N' + Nz - 1 (one forward and one inverse
// FFT of length L, kernel spectrum precomputed), and Re / Im of the result are
// the first / second derivative.
//
// Thread layout: tid = r * LINES + li, li = line within the tile (lines are
// adjacent in memory, so every global access is coalesced across li).
// FFT of length L = L1 * L2 in two register passes with one shared-memory
// exchange each way:  input index n = n2 + L2 n1 lives in thread r = n2;
// frequency k = k1 + L1 k2 lives in thread r = k1.
#pragma once
#include "phases.cuh"

#if defined(__CUDACC__)
#define DERIV_NOINLINE __host__ __device__ __noinline__
#else
#define DERIV_NOINLINE
#endif

namespace fcns {

template <class T, int L1_, int L2_, int LINES_>
struct DerivConv {
  static constexpr int L1 = L1_, L2 = L2_, L = L1 * L2, LINES = LINES_;
  static constexpr int G = L1 > L2 ? L1 : L2;
  static constexpr int THREADS = G * LINES;
  static constexpr int NPHASE = 4;
  static constexpr int MINB = (sizeof(T) == 4 && THREADS <= 512) ? 2 : 1;  // CTAs per SM (register budget)
  static constexpr int MR_MAX = 640;  // C * d <= 64 * 10
  // row padding of the exchange buffer: a warp touches several k1 rows of
  // LINES elements; shifting rows by half a 128-byte bank line keeps those
  // accesses conflict-free when one row chunk is narrower than 128 bytes
  static constexpr int PAD = (LINES * 2 * (int)sizeof(T) < 128) ? LINES : 0;
  static constexpr int ROW = L2 * LINES + PAD;
  static constexpr int DMAX = 10;
  using C = cx<T>;

  struct Args {
    const T* f;
    T* df;
    T* d2f;
    int Nz, Np, d, Cc;
    long long lines;           // lines per field (Nx * Ny)
    long long tiles;           // tiles per field
    long long zstride;         // elements between consecutive z
    long long bstride;         // elements between fields
    T s1, s2;                  // 1/dz, 1/dz^2
    const double* Mr;          // C x d (float64 path)
    const float2* Mr2;         // C x d as (hi, lo) float pairs (float32 path)
    const C* H;                // kernel spectrum, natural order, length L
    const C* tw;               // tw[n2 * L1 + k1] = e^{-2 pi i n2 k1 / L}
  };

  struct Regs {
    C v[L1];
    C u[L2];
  };

  // shared memory layout (the kernel spectrum and twiddles are read through
  // the read-only data cache; every CTA uses the same L entries)
  static constexpr size_t off_buf = 0;
  static constexpr size_t off_M = off_buf + sizeof(C) * ROW * L1;
  static constexpr size_t off_E = off_M + sizeof(double) * MR_MAX;
  static constexpr size_t smem_bytes = off_E + sizeof(T) * LINES * 2 * DMAX;

  static FC_HD int bidx(int k1, int n2, int li) { return k1 * ROW + n2 * LINES + li; }

  // continuation value jj of a real line (Sec. 3): M_r f_last + M_l f_first,
  // float64 (float64 path) or compensated float-float (float32 path); kept out
  // of line so the unrolled loops stay small
  static DERIV_NOINLINE T cont_real(int jj, const T* first, const T* last, int d, int Cc, const double* Ms,
                                    const float2* Ms2) {
    if constexpr (sizeof(T) == 4) {
      ff c{0.f, 0.f};
      for (int i = 0; i < d; ++i) {
        const float2 m1 = Ms2[jj * d + i];
        const float2 m2 = Ms2[(Cc - 1 - jj) * d + (d - 1 - i)];
        ff_fma(c, m1.x, m1.y, (float)last[i]);
        ff_fma(c, m2.x, m2.y, (float)first[i]);
      }
      return (T)ff_round(c);
    } else {
      double c = 0.0;
      for (int i = 0; i < d; ++i) {
        c += Ms[jj * d + i] * (double)last[i];
        c += Ms[(Cc - 1 - jj) * d + (d - 1 - i)] * (double)first[i];
      }
      return (T)c;
    }
  }

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* buf = reinterpret_cast<C*>(sm + off_buf);
    const C* __restrict__ Hs = a.H;
    const C* __restrict__ tws = a.tw;
    double* Ms = reinterpret_cast<double*>(sm + off_M);
    float2* Ms2 = reinterpret_cast<float2*>(sm + off_M);
    T* E = reinterpret_cast<T*>(sm + off_E);
    const int r = tid / LINES, li = tid % LINES;
    const long long field = bid / a.tiles;
    const long long line = (bid % a.tiles) * LINES + li;
    const bool valid = line < a.lines;
    const long long base = field * a.bstride + line;

    if constexpr (P == 0) {
      if constexpr (sizeof(T) == 4) {
        for (int i = tid; i < a.Cc * a.d; i += THREADS) Ms2[i] = a.Mr2[i];
      } else {
        for (int i = tid; i < a.Cc * a.d; i += THREADS) Ms[i] = a.Mr[i];
      }
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int n = r + L2 * j;
          T x = T(0);
          if (valid && n < a.Nz) x = a.f[base + (long long)n * a.zstride];
          R.v[j] = mk<T>(x, T(0));
          if (n < a.d) E[li * 2 * DMAX + n] = x;
          if (n >= a.Nz - a.d && n < a.Nz) E[li * 2 * DMAX + DMAX + (n - (a.Nz - a.d))] = x;
        }
      }
    } else if constexpr (P == 1) {
      if (r < L2) {
        const T* first = E + li * 2 * DMAX;
        const T* last = first + DMAX;
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int n = r + L2 * j;
          if (n >= a.Nz && n < a.Np) R.v[j] = mk<T>(cont_real(n - a.Nz, first, last, a.d, a.Cc, Ms, Ms2), T(0));
        }
        dft_reg<L1, -1, T>(R.v);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) buf[bidx(k1, r, li)] = cmul(R.v[k1], tws[r * L1 + k1]);
      }
    } else if constexpr (P == 2) {
      if (r < L1) {
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) R.u[n2] = buf[bidx(r, n2, li)];
        dft_reg<L2, -1, T>(R.u);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) R.u[k2] = cmul(R.u[k2], Hs[r + L1 * k2]);
        dft_reg<L2, 1, T>(R.u);
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) buf[bidx(r, n2, li)] = cmulc(R.u[n2], tws[n2 * L1 + r]);
      }
    } else if constexpr (P == 3) {
      if (r < L2) {
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) R.v[k1] = buf[bidx(k1, r, li)];
        dft_reg<L1, 1, T>(R.v);
        if (valid) {
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            if (n < a.Nz) {
              const long long o = base + (long long)n * a.zstride;
              if (a.df) a.df[o] = R.v[j].x * a.s1;
              if (a.d2f) a.d2f[o] = R.v[j].y * a.s2;
            }
          }
        }
      }
    }
  }
};

}  // namespace fcns

#include "engine.cuh"

namespace fcns {

// fc_deriv_z with two adjacent real z-lines packed as one complex line
// x = a + i b.  The derivative kernels d1, d2 of the N'-periodic grid are
// real, so one forward transform X = FFT_L(x) serves both lines and
//   IFFT_L(X H1) = d1*a + i d1*b,   IFFT_L(X H2) = d2*a + i d2*b
// (H1, H2: spectra of d1, d2 placed circularly on L >= N' + Nz - 1, with 1/L):
// three length-L transforms per two lines instead of four.
template <class T, int L1_, int L2_, int LINES_>
struct DerivPair {
  using E = Eng<T, L1_, L2_, LINES_>;
  using C = cx<T>;
  static constexpr int L1 = L1_, L2 = L2_, LINES = LINES_;
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
  };
  struct Regs { C v[L1]; C u[L2]; };

  // (the continuation matrix is read through the data cache: few threads use it)
  static constexpr size_t off_b1 = sizeof(C) * E::BUF;
  static constexpr size_t off_E = off_b1 + sizeof(C) * E::BUF;
  static constexpr size_t smem_bytes = off_E + sizeof(C) * LINES * 2 * DMAX;

  // continuation value jj of a complex line: M_r f_last + M_l f_first
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
      double re = 0, im = 0;
      for (int i = 0; i < d; ++i) {
        const double m1 = Ms[jj * d + i], m2 = Ms[(Cc - 1 - jj) * d + (d - 1 - i)];
        re += m1 * last[i].x + m2 * first[i].x;
        im += m1 * last[i].y + m2 * first[i].y;
      }
      return mk<T>((T)re, (T)im);
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
    const bool va = la < a.lines, vb = la + 1 < a.lines;
    const long long base = field * a.bstride + la;

    if constexpr (P == 0) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int n = r + L2 * j;
          C x = mk<T>(0, 0);
          if (n < a.Nz) {
            const T* p = a.f + base + (long long)n * a.zstride;
            if (va) x.x = p[0];
            if (vb) x.y = p[1];
          }
          R.v[j] = x;
          if (n < a.d) Ev[n] = x;
          if (n >= a.Nz - a.d && n < a.Nz) Ev[DMAX + n - (a.Nz - a.d)] = x;
        }
      }
    } else if constexpr (P == 1) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
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
        E::mulH(R.u, a.H1, r);
        E::template Bi<1>(R.u, b0, a.tw, r, li);
        FC_FENCE();
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) R.u[k2] = b1[E::bidx(r, k2, li)];
        E::mulH(R.u, a.H2, r);
        E::template Bi<1>(R.u, b1, a.tw, r, li);
      }
    } else if constexpr (P == 3) {
      if (r < L2 && va) {
        E::template Ai<1>(R.v, b0, r, li);
        if (a.df) {
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            if (n < a.Nz) {
              T* p = a.df + base + (long long)n * a.zstride;
              p[0] = R.v[j].x * a.s1;
              if (vb) p[1] = R.v[j].y * a.s1;
            }
          }
        }
        if (a.d2f) {
          E::template Ai<1>(R.v, b1, r, li);
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            if (n < a.Nz) {
              T* p = a.d2f + base + (long long)n * a.zstride;
              p[0] = R.v[j].x * a.s2;
              if (vb) p[1] = R.v[j].y * a.s2;
            }
          }
        }
      }
    }
  }
};

}  // namespace fcns
