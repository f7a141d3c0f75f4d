// Kernels of the time-splitting FC-Gram Navier-Stokes / Boussinesq step.
//
// State representation: every field is kept in the mixed (kx, ky, z') space
// on the CONTINUED z grid, X[f][s][ky][kx], s = 0..N'-1 (the FC extension of
// the physical values plus the continuation points).  This is the inverse z
// DFT of the paper's continued spectral field (Sec. 3, Sec. 4.2): the two
// representations are related exactly by a length-N' DFT, and every
// spectral-space operation of the method is applied either as a circular
// convolution along z' (z derivatives, the z filter) or through explicit
// Bluestein DFTs (the projection, which mixes the three velocity components
// with k-dependent weights).
//
// Layouts (Kx = Nx/2 + 1, lines = Ny * Kx, line index l = ky * Kx + kx):
//   X      [nf][N'][lines]   complex   state (extended mixed space)
//   M*     [nf][Nz][lines]   complex   mixed-space work arrays
//   rows   [nf][Nz][Ny][Kx]  complex   same memory seen as x-rows
//   walls  [2][2][lines]     complex double  tangential grad p at z = 0, Lz
#pragma once
#include <cmath>

#include "engine.cuh"

namespace fcns {

// ---------------------------------------------------------------------------
// tables and geometry shared by the z kernels
// ---------------------------------------------------------------------------
template <class T>
struct ZTab {
  const double* Mr;     // C x d continuation matrix (float64 path)
  const float2* Mr2;    // C x d as (hi, lo) float pairs (float32 path)
  const cx<T>* tw;      // engine twiddles, L entries
  const cx<T>* H1;      // conv spectrum of d/dz (unit spacing), L entries
  const cx<T>* H2;      // conv spectrum of d2/dz2 (unit spacing)
  const cx<T>* Hf;      // conv spectrum of the z filter
  const cx<T>* chirp;   // Bluestein chirp exp(-i pi n^2 / N'), N' entries
  const cx<T>* Hbf;     // Bluestein kernel spectrum (forward DFT)
  const cx<T>* Hbi;     // Bluestein kernel spectrum (inverse DFT)
  const T* kxo;         // kx with the Nyquist entry zeroed (Kx)
  const T* kyo;         // ky with the Nyquist entry zeroed (Ny)
  const T* kzo;         // kz with the Nyquist entry zeroed (N'), FFT order
  const T* kx;          // kx (Kx)
  const T* ky;          // ky (Ny)
  const T* fx;          // x filter / mask factor (Kx)
  const T* fy;          // y filter / mask factor (Ny)
  const double* kxo_d;  // float64 copies for the homogeneous-pressure coefficients
  const double* kyo_d;
};

struct ZGeom {
  int Nz, Np, d, Cc, Kx, Kxp, Ny, nf;   // Kxp: kx row length padded to a multiple of TL
  long long lines;    // Ny * Kxp (line = ky * Kxp + kx; kx >= Kx are padding)
  long long ntiles;   // lines / TL
  double Lz, dz;
};

// Tiled layout of every [field][z][line] array: lines are grouped in tiles
// of TL, and a tile stores its z rows contiguously, so the z-line kernels
// (few lines per CTA) read short runs that are adjacent in memory, and the
// x / y kernels still read TL contiguous lines per z row.
constexpr int TL = 16;
// element index of (field f, row z, line) in an array of Z rows per tile;
// every array holds fewer than 2^31 elements (checked when the layout is made)
FC_HD int lay(long long f, long long z, long long line, long long Z, long long ntiles) {
  const int l = (int)line;
  return ((((int)f * (int)ntiles + (l >> 4)) * (int)Z + (int)z) << 4) + (l & (TL - 1));
}

// lines of a tile row that share one 32-byte L2 sector
template <class C>
constexpr int sector_lines() { return sizeof(C) >= 32 ? 1 : 32 / (int)sizeof(C); }

// L2 prefetch of rows r, r + R, ... (< nrows) of `line` of field f in a tiled
// array of Z rows per tile, issued by the first thread of each 32-byte sector
template <class C, int JN>
FC_HD void prefetch_line(const C* base, long long f, long long line, int Z, int nrows, long long ntiles, int r,
                         int R, int li) {
  if (li % sector_lines<C>() != 0) return;
  const C* x = base + lay(f, 0, line, Z, ntiles);
#pragma unroll
  for (int j = 0; j < JN; ++j) {
    const int n = r + R * j;
    if (n < nrows) prefetch_l2(x + n * TL);
  }
}

#if defined(__CUDACC__)
#define FC_NOINLINE __host__ __device__ __noinline__
#else
#define FC_NOINLINE
#endif

constexpr int DMAX = 10;
constexpr int MRMAX = 640;


// C continuation value jj (point Nz + jj) of a complex line from its first /
// last d values (Sec. 3 continuation formula; right matrix M_r, left matrix
// its row/column reversal), with compensated sums: float-float products in
// float32, double-double in float64 (the weights reach 4e3 and cancel).
template <class T>
FC_NOINLINE cx<T> continuation_value(int jj, const cx<T>* first, const cx<T>* last, int d, int Cc,
                                     const double* Ms, const float2* Ms2) {
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
      const double m1 = Ms[jj * d + i];
      const double m2 = Ms[(Cc - 1 - jj) * d + (d - 1 - i)];
      dd_fma(re, m1, last[i].x);
      dd_fma(im, m1, last[i].y);
      dd_fma(re, m2, first[i].x);
      dd_fma(im, m2, first[i].y);
    }
    return mk<T>((T)dd_round(re), (T)dd_round(im));
  }
}

template <class T>
FC_HD void load_mr(unsigned char* sm, const ZTab<T>& t, int n, int tid, int threads) {
  if constexpr (sizeof(T) == 4) {
    float2* M2 = reinterpret_cast<float2*>(sm);
    for (int i = tid; i < n; i += threads) M2[i] = t.Mr2[i];
  } else {
    double* M = reinterpret_cast<double*>(sm);
    for (int i = tid; i < n; i += threads) M[i] = t.Mr[i];
  }
}

// ===========================================================================
// K1  zderiv: dz and dzz of the state at the Nz physical points.
// Circular convolution of the extended line with the derivative kernels of
// the N'-periodic grid (= multiplication of the continued spectrum by i kz
// (Nyquist zeroed) and -kz^2, Sec. 4.2), first Nz outputs.
// ===========================================================================
// JN: input registers j >= JN (indices r + L2 j >= L2 JN) are known to be
// zero and hold no output: L2 JN >= N' (padded lengths, L >= 2 N' - 1, give
// JN = L1 / 2; direct lengths JN = L1).
template <class T, int L1, int L2, int LINES, int JN = L1>
struct KZDeriv {
  using E = Eng<T, L1, L2, LINES>;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 3;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  struct Args {
    ZGeom g;
    ZTab<T> t;
    const C* X;
    C* DZ;
    C* DZZ;
    long long tiles;
    long long pf, nblocks;   // prefetch into L2 the input of block bid + pf (0: off)
    T s1, s2;
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t off_b1 = sizeof(C) * E::BUF;
  static constexpr size_t smem_bytes = 2 * sizeof(C) * E::BUF;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    C* b1 = reinterpret_cast<C*>(sm + off_b1);
    const int r = tid / LINES, li = tid % LINES;
    const long long f = bid / a.tiles;
    const long long line = (bid % a.tiles) * LINES + li;
    const bool valid = line < a.g.lines && (line % a.g.Kxp) < a.g.Kx;
    if constexpr (P == 0) {
      if (r < L2) {
        const C* x = a.X + lay(f, 0, line, a.g.Np, a.g.ntiles);
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int n = r + L2 * j;
          R.v[j] = (j < JN && valid && n < a.g.Np) ? x[n * TL] : mk<T>(0, 0);
        }
        if (a.pf > 0 && bid + a.pf < a.nblocks) {
          const long long b2 = bid + a.pf, line2 = (b2 % a.tiles) * LINES + li;
          if (line2 < a.g.lines && (line2 % a.g.Kxp) < a.g.Kx)
            prefetch_line<C, JN>(a.X, b2 / a.tiles, line2, a.g.Np, a.g.Np, a.g.ntiles, r, L2, li);
        }
        E::template A<-1>(R.v, b0, a.t.tw, r, li);
      }
    } else if constexpr (P == 1) {
      if (r < L1) {
        E::template B<-1>(R.u, b0, r, li);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) b1[E::bidx(r, k2, li)] = R.u[k2];
        // the two inverse transforms share one copy of the code (instruction cache)
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          if (o == 1) {
            FC_FENCE();
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) R.u[k2] = b1[E::bidx(r, k2, li)];
          }
          // the NS lengths satisfy L >= 2 N' - 1 (or L = N'): H1 imaginary, H2 real
          if (o == 0) E::mulH_imag(R.u, a.t.H1, r);
          else E::mulH_real(R.u, a.t.H2, r);
          E::template Bi<1>(R.u, o == 0 ? b0 : b1, a.t.tw, r, li);
        }
      }
    } else if constexpr (P == 2) {
      if (r < L2) {
#pragma unroll 1
        for (int o = 0; o < 2; ++o) {
          C* out = (o == 0 ? a.DZ : a.DZZ) + lay(f, 0, line, a.g.Nz, a.g.ntiles);
          const T sc = o == 0 ? a.s1 : a.s2;
          E::template Ai<1>(R.v, o == 0 ? b0 : b1, r, li);
          if (valid) {
#pragma unroll
            for (int j = 0; j < JN; ++j) {
              const int n = r + L2 * j;
              if (n < a.g.Nz) out[n * TL] = cscale(R.v[j], sc);
            }
          }
        }
      }
    }
  }
};

// ===========================================================================
// K5  zcombine: pressureless stage update in mixed space, BC injection and
// re-continuation (Sec. 4.4 steps 1-2 with the state in extended mixed
// space):
//   v*(z) = v^t(z) + dt_j [ F_xy (f_z * FC(N))(z) + nu (dzz v^{j-1} - kperp^2 v^{j-1}) ]
//   tangential v* := dt_j grad_par p^{prev} at z = 0, Lz; theta := 0 there;
//   X_out = [v*; continuation of v*].
// The z filter acts as a circular convolution of the continued N.
// ===========================================================================
template <class T, int L1, int L2, int LINES, int JN = L1>
struct KZCombine {
  using E = Eng<T, L1, L2, LINES>;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 5;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  struct Args {
    ZGeom g;
    ZTab<T> t;
    const C* NL;      // [nf][Nz][lines] nonlinear term (mixed)
    const C* Xt;      // [nf][N'][lines] state at t
    const C* Xj;      // [nf][N'][lines] state of the previous stage
    const C* DZZ;     // [nf][Nz][lines]
    C* Xout;          // [nf][N'][lines]
    const double2* gradp;  // [2][2][lines]
    double dtj;
    double dif[4];
    long long tiles;
    long long pf, nblocks;  // prefetch into L2 the input of block bid + pf (0: off)
    int inject;            // 1: wall injection (RK stage); 0: plain right-hand side
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t off_M = sizeof(C) * E::BUF;
  static constexpr size_t off_E = off_M + sizeof(double) * MRMAX;
  static constexpr size_t smem_bytes = off_E + sizeof(C) * LINES * 2 * DMAX;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    const double* Ms = reinterpret_cast<const double*>(sm + off_M);
    const float2* Ms2 = reinterpret_cast<const float2*>(sm + off_M);
    C* Ev = reinterpret_cast<C*>(sm + off_E) + li_of(tid) * 2 * DMAX;
    const int r = tid / LINES, li = tid % LINES;
    const int f = (int)(bid / a.tiles);
    const long long line = (bid % a.tiles) * LINES + li;
    const bool valid = line < a.g.lines && (line % a.g.Kxp) < a.g.Kx;
    const int Nz = a.g.Nz, Np = a.g.Np, d = a.g.d;
    const long long Ls = a.g.lines;
    if constexpr (P == 0) {
      load_mr<T>(sm + off_M, a.t, a.g.Cc * d, tid, THREADS);
      if (r < L2) {
        const C* x = a.NL + lay(f, 0, line, Nz, a.g.ntiles);
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int n = r + L2 * j;
          C val = mk<T>(0, 0);
          if (j >= JN) {
            R.v[j] = val;
            continue;
          }
          if (valid && n < Nz) val = x[n * TL];
          R.v[j] = val;
          if (n < d) Ev[n] = val;
          if (n >= Nz - d && n < Nz) Ev[DMAX + n - (Nz - d)] = val;
        }
        // the rows of Xt, Xj and DZZ read after the filter transforms: into
        // L2 now, so that their latency overlaps the transforms; and the
        // input of block bid + pf
        if (valid) {
          prefetch_line<C, JN>(a.Xj, f, line, Np, Nz, a.g.ntiles, r, L2, li);
          prefetch_line<C, JN>(a.DZZ, f, line, Nz, Nz, a.g.ntiles, r, L2, li);
          if (a.Xt) prefetch_line<C, JN>(a.Xt, f, line, Np, Nz, a.g.ntiles, r, L2, li);
        }
        if (a.pf > 0 && bid + a.pf < a.nblocks) {
          const long long b2 = bid + a.pf, line2 = (b2 % a.tiles) * LINES + li;
          if (line2 < a.g.lines && (line2 % a.g.Kxp) < a.g.Kx)
            prefetch_line<C, JN>(a.NL, b2 / a.tiles, line2, Nz, Nz, a.g.ntiles, r, L2, li);
        }
      }
    } else if constexpr (P == 1) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < JN; ++j) {
          const int n = r + L2 * j;
          if (n >= Nz && n < Np) R.v[j] = continuation_value<T>(n - Nz, Ev, Ev + DMAX, d, a.g.Cc, Ms, Ms2);
        }
        E::template A<-1>(R.v, b0, a.t.tw, r, li);
      }
    } else if constexpr (P == 2) {
      if (r < L1) {
        E::template B<-1>(R.u, b0, r, li);
        E::mulH_real(R.u, a.t.Hf, r);   // even filter kernel: real spectrum
        E::template Bi<1>(R.u, b0, a.t.tw, r, li);
      }
    } else if constexpr (P == 3) {
      if (r < L2) {
        E::template Ai<1>(R.v, b0, r, li);
        const int kx = (int)(line % a.g.Kxp), ky = (int)(line / a.g.Kxp);
        const T fxy = valid ? a.t.fx[kx] * a.t.fy[ky] : T(0);
        const T ckp2 = valid ? a.t.kx[kx] * a.t.kx[kx] + a.t.ky[ky] * a.t.ky[ky] : T(0);
        const T cdt = (T)a.dtj, cnu = (T)(a.dif[f]);
        const long long fo = lay(f, 0, line, Np, a.g.ntiles);
        const C* xt = a.Xt + fo;
        const C* xj = a.Xj + fo;
        const C* dzz = a.DZZ + lay(f, 0, line, Nz, a.g.ntiles);
        C* xo = a.Xout + fo;
#pragma unroll
        for (int j = 0; j < JN; ++j) {
          const int n = r + L2 * j;
          if (n < Nz) {
            C vs = mk<T>(0, 0);
            if (valid) {
              const C vj = xj[n * TL];
              const C zz = dzz[n * TL];
              const C nlf = cscale(R.v[j], fxy);
              const C visc = csub(zz, cscale(vj, ckp2));
              const C base = a.Xt ? xt[n * TL] : mk<T>(0, 0);
              vs = cadd(base, cscale(cadd(nlf, cscale(visc, cnu)), cdt));
              if (a.inject && (n == 0 || n == Nz - 1)) {
                const int wall = (n == 0) ? 0 : 1;
                if (f < 2) {
                  const double2 gp = a.gradp[((long long)wall * 2 + f) * Ls + line];
                  vs = mk<T>((T)(a.dtj * gp.x), (T)(a.dtj * gp.y));
                } else if (f == 3) {
                  vs = mk<T>(0, 0);
                }
              }
              xo[n * TL] = vs;
            }
            if (n < d) Ev[n] = vs;
            if (n >= Nz - d) Ev[DMAX + n - (Nz - d)] = vs;
          }
        }
      }
    } else if constexpr (P == 4) {
      if (r < L2 && valid) {
        C* xo = a.Xout + lay(f, 0, line, Np, a.g.ntiles);
#pragma unroll
        for (int j = 0; j < JN; ++j) {
          const int n = r + L2 * j;
          if (n >= Nz && n < Np)
            xo[n * TL] = continuation_value<T>(n - Nz, Ev, Ev + DMAX, d, a.g.Cc, Ms, Ms2);
        }
      }
    }
  }
  static FC_HD int li_of(int tid) { return tid % LINES; }
};

// ===========================================================================
// K5b  zcontinue: X = [m; continuation of m] for mixed fields m (state from
// physical fields, Sec. 3), optionally with the wall injection of
// Sec. 4.1 (bound-v) for the stand-alone projection.
// ===========================================================================
template <class T, int LINES>
struct KZContinue {
  using C = cx<T>;
  static constexpr int G = 32;
  static constexpr int THREADS = G * LINES, NPHASE = 2, MINB = 1;
  struct Args {
    ZGeom g;
    ZTab<T> t;
    const C* M;     // [nf][Nz][lines]
    C* X;           // [nf][N'][lines]
    const double2* gradp;  // injection planes or nullptr
    double dtj;
    long long tiles;
  };
  struct Regs { int dummy; };
  static constexpr size_t off_E = sizeof(double) * MRMAX;
  static constexpr size_t smem_bytes = off_E + sizeof(C) * LINES * 2 * DMAX;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs&) {
    const double* Ms = reinterpret_cast<const double*>(sm);
    const float2* Ms2 = reinterpret_cast<const float2*>(sm);
    const int r = tid / LINES, li = tid % LINES;
    C* Ev = reinterpret_cast<C*>(sm + off_E) + li * 2 * DMAX;
    const int f = (int)(bid / a.tiles);
    const long long line = (bid % a.tiles) * LINES + li;
    const bool valid = line < a.g.lines && (line % a.g.Kxp) < a.g.Kx;
    const int Nz = a.g.Nz, Np = a.g.Np, d = a.g.d;
    const long long Ls = a.g.lines;
    const C* m = a.M + lay(f, 0, line, Nz, a.g.ntiles);
    C* x = a.X + lay(f, 0, line, Np, a.g.ntiles);
    if constexpr (P == 0) {
      load_mr<T>(sm, a.t, a.g.Cc * d, tid, THREADS);
      if (valid) {
        for (int n = r; n < Nz; n += G) {
          C val = m[n * TL];
          if (a.gradp && (n == 0 || n == Nz - 1)) {
            const int wall = (n == 0) ? 0 : 1;
            if (f < 2) {
              const double2 gp = a.gradp[((long long)wall * 2 + f) * Ls + line];
              val = mk<T>((T)(a.dtj * gp.x), (T)(a.dtj * gp.y));
            } else if (f == 3) {
              val = mk<T>(0, 0);
            }
          }
          x[n * TL] = val;
          if (n < d) Ev[n] = val;
          if (n >= Nz - d) Ev[DMAX + n - (Nz - d)] = val;
        }
      }
    } else {
      if (valid)
        for (int n = Nz + r; n < Np; n += G)
          x[n * TL] = continuation_value<T>(n - Nz, Ev, Ev + DMAX, d, a.g.Cc, Ms, Ms2);
    }
  }
};

// ===========================================================================
// K6  zproject: pressure solve and projection of the three velocity
// components of the continued v* (Sec. 4.2, Sec. 4.4 steps 3-5), with
// phi = dt_j p:
//   s      = (kx v^_x + ky v^_y + kz v^_z) / k^2   (0 where k = 0; odd-order
//            wavenumbers with the Nyquist entries zeroed)
//   grad phi^I = (kx sigma, ky sigma, sigma_z),  sigma = IDFT(s), sigma_z = IDFT(kz s)
//   b, t   = w* - sigma_z at z = 0, Lz
//   A, B   (Eqs. A, B), gamma = |k_perp| (Nyquist-zeroed wavenumbers);
//          D = (b + t)/2 where gamma = 0
//   grad phi^H = (i kx Phi, i ky Phi, Phi'),  Phi = A e^{g(z-Lz)} + B e^{-g z}
//   X     -= grad phi^I + FC(grad phi^H);  walls <- grad_par phi / dt_j.
// DFTs of length N' by Bluestein (chirp, circular convolution of length L,
// chirp), or, when N' itself is a compiled length (DIRECT, L = N'), by one
// length-N' transform each; done one after another through a single exchange
// buffer; the
// intermediate lines (Y^, s, sigma, sigma_z) go to two scratch lines per
// line: in shared memory when they fit in 24 KB per CTA (float32, short
// lengths or few lines per CTA), else in two global arrays G0, G1 of
// [N'][lines] (owned element by element by one thread; they stay in L2).
// ===========================================================================
template <class T, int L1, int L2, int LINES, bool DIRECT>
struct KZProject {
  using E = Eng<T, L1, L2, LINES>;
  static constexpr int JN = DIRECT ? L1 : L1 / 2;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 7;
  // phases 1..3 run four times (Y^, W^, sigma, sigma_z) from one copy of code
  static constexpr int LB = 1, LE = 4, NIT = 4;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  struct Args {
    ZGeom g;
    ZTab<T> t;
    C* X;                 // [3][N'][lines] in / out
    C* G0;                // scratch [N'][lines]
    C* G1;                // scratch [N'][lines]
    double2* gradp;       // [2][2][lines] out
    double dtj;
    long long tiles;
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t off_M = sizeof(C) * E::BUF;
  static constexpr size_t off_W = off_M + sizeof(double) * MRMAX;   // per line: b, t, sigma walls (complex double)
  static constexpr size_t off_E = off_W + sizeof(double) * LINES * 16;
  // per line: Phi and Phi' at the first / last d points
  static constexpr size_t off_G = off_E + sizeof(C) * LINES * 4 * DMAX;
  // scratch lines: N' <= NPC (padded: L >= 2 N' - 1; direct: N' = L)
  static constexpr int NPC = DIRECT ? L1 * L2 : (L1 * L2) / 2;
  static constexpr size_t sg_bytes = 2 * sizeof(C) * LINES * NPC;
  static constexpr bool SG = sizeof(T) == 4 && sg_bytes <= 24 * 1024;
  static constexpr int GS = SG ? LINES : TL;   // element stride of a scratch line
  static constexpr size_t smem_bytes = off_G + (SG ? sg_bytes : 0);

  // conj(chirp[n]) (1 outside the line)
  static FC_HD C cchirp(const ZTab<T>& t, int n, int Np) {
    C c = n < Np ? t.chirp[n] : mk<T>(1, 0);
    c.y = -c.y;
    return c;
  }

  // Output value n of DFT `it` from the raw transform result `val`, and what
  // the projection does with it (K = min(it, 2)):
  //   it 0: Y^ -> G0;  it 1: W^, s = (Y^ + kz W^) / k^2 -> G0;
  //   it 2: sigma -> G1 and its wall values;  it 3: sigma_z -> G0, b and t.
  template <int K>
  static FC_HD void post(const Args& a, int it, int n, C val, T kxo, T kyo, T invNp, C* g0, C* g1,
                         const C* xw, double* W) {
    const int Nz = a.g.Nz, Np = a.g.Np;
    if constexpr (K < 2) {
      if constexpr (!DIRECT) val = cmul(val, a.t.chirp[n]);
      if constexpr (K == 0) {
        g0[n * GS] = val;
      } else {
        const T kz = a.t.kzo[n];
        const T k2 = kxo * kxo + kyo * kyo + kz * kz;
        const T inv = k2 > T(0) ? T(1) / k2 : T(0);
        g0[n * GS] = cscale(cadd(g0[n * GS], cscale(val, kz)), inv);
      }
    } else {
      // direct: the inverse DFT is conj(DFT(conj(.)))
      if constexpr (DIRECT) val = mk<T>(val.x, -val.y);
      else val = cmul(val, cchirp(a.t, n, Np));
      const C sg = cscale(val, invNp);
      if (it == 2) {
        g1[n * GS] = sg;
        if (n == 0 || n == Nz - 1) {
          const int o = (n == 0) ? 4 : 6;
          W[o] = (double)sg.x;
          W[o + 1] = (double)sg.y;
        }
      } else {
        g0[n * GS] = sg;
        if (n == 0 || n == Nz - 1) {
          const C w = xw[n * TL];
          const int o = (n == 0) ? 0 : 2;
          W[o] = (double)w.x - (double)sg.x;
          W[o + 1] = (double)w.y - (double)sg.y;
        }
      }
    }
  }
  // f(integral_constant<K>) with K = min(it, 2), the branch taken outside the element loops
  template <class F>
  static FC_HD void by_kind(int it, F&& f) {
    if (it == 0) f(std::integral_constant<int, 0>{});
    else if (it == 1) f(std::integral_constant<int, 1>{});
    else f(std::integral_constant<int, 2>{});
  }

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, int it, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    const double* Ms = reinterpret_cast<const double*>(sm + off_M);
    const float2* Ms2 = reinterpret_cast<const float2*>(sm + off_M);
    const int r = tid / LINES, li = tid % LINES;
    double* W = reinterpret_cast<double*>(sm + off_W) + li * 16;
    C* Ev = reinterpret_cast<C*>(sm + off_E) + li * 4 * DMAX;   // Phi first, Phi last, Phi' first, Phi' last
    const long long line = bid * LINES + li;
    const bool valid = line < a.g.lines && (line % a.g.Kxp) < a.g.Kx;
    const int Nz = a.g.Nz, Np = a.g.Np, d = a.g.d;
    const long long Ls = a.g.lines;
    const int kxi = valid ? (int)(line % a.g.Kxp) : 0, kyi = valid ? (int)(line / a.g.Kxp) : 0;
    const T kxo = a.t.kxo[kxi], kyo = a.t.kyo[kyi];
    C* xu = a.X + lay(0, 0, line, Np, a.g.ntiles);
    C* xv = a.X + lay(1, 0, line, Np, a.g.ntiles);
    C* xw = a.X + lay(2, 0, line, Np, a.g.ntiles);
    C* g0 = SG ? reinterpret_cast<C*>(sm + off_G) + li : a.G0 + lay(0, 0, line, Np, a.g.ntiles);
    C* g1 = SG ? reinterpret_cast<C*>(sm + off_G) + LINES * NPC + li : a.G1 + lay(0, 0, line, Np, a.g.ntiles);
    const T invNp = T(1.0 / Np);

    if constexpr (P == 0) {
      load_mr<T>(sm + off_M, a.t, a.g.Cc * d, tid, THREADS);
    } else if constexpr (P == 1) {  // input of transform `it`
      if (r < L2) {
        if (it == 0) {  // Y = kx u + ky v
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            C y = mk<T>(0, 0);
            if (j < JN && valid && n < Np) {
              y = cadd(cscale(xu[n * TL], kxo), cscale(xv[n * TL], kyo));
              if constexpr (!DIRECT) y = cmul(y, a.t.chirp[n]);
            }
            R.v[j] = y;
          }
        } else if (it == 1) {  // w
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            C y = mk<T>(0, 0);
            if (j < JN && valid && n < Np) {
              y = xw[n * TL];
              if constexpr (!DIRECT) y = cmul(y, a.t.chirp[n]);
            }
            R.v[j] = y;
          }
        } else {  // s (it = 2) or kz s (it = 3), inverse DFT input
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = r + L2 * j;
            C x = mk<T>(0, 0);
            if (j < JN && valid && n < Np) {
              x = g0[n * GS];
              if (it == 3) x = cscale(x, a.t.kzo[n]);
              if constexpr (DIRECT) x.y = -x.y;
              else x = cmul(x, cchirp(a.t, n, Np));
            }
            R.v[j] = x;
          }
        }
        E::template A<-1>(R.v, b0, a.t.tw, r, li);
      }
    } else if constexpr (P == 2) {
      if (r < L1) {
        E::template B<-1>(R.u, b0, r, li);
        if constexpr (DIRECT) {
          // L = N': thread k1 holds DFT values k1 + L1 k2, final
          if (valid) {
            by_kind(it, [&](auto kc) {
              constexpr int K = decltype(kc)::value;
#pragma unroll
              for (int k2 = 0; k2 < L2; ++k2) post<K>(a, it, r + L1 * k2, R.u[k2], kxo, kyo, invNp, g0, g1, xw, W);
            });
          }
        } else {
          E::mulH(R.u, it < 2 ? a.t.Hbf : a.t.Hbi, r);
          E::template Bi<1>(R.u, b0, a.t.tw, r, li);
        }
      }
    } else if constexpr (P == 3) {  // Bluestein output of transform `it`
      if constexpr (!DIRECT) {
        if (r < L2) {
          E::template Ai<1>(R.v, b0, r, li);
          if (!valid) return;
          by_kind(it, [&](auto kc) {
            constexpr int K = decltype(kc)::value;
#pragma unroll
            for (int j = 0; j < JN; ++j) {
              const int n = r + L2 * j;
              if (n < Np) post<K>(a, it, n, R.v[j], kxo, kyo, invNp, g0, g1, xw, W);
            }
          });
        }
      }
    } else if constexpr (P == 4) {  // homogeneous coefficients (float64) -> W[8..12]
      if (r == 0) {
        const double br = W[0], bi = W[1], tr = W[2], ti = W[3];
        double Ar = 0, Aim = 0, Br = 0, Bim = 0, D = 0;
        // gamma = |k_perp| of the Nyquist-zeroed wavenumbers (the same ones as
        // the gradient i kx Phi, i ky Phi), so grad phi^H is divergence-free;
        // where it vanishes, phi^H = D z with D = (b + t)/2.
        const double kxd = a.t.kxo_d[kxi], kyd = a.t.kyo_d[kyi];
        if (kxd == 0.0 && kyd == 0.0) {
          D = 0.5 * (br + tr);
        } else {
          const double gam = sqrt(kxd * kxd + kyd * kyd);
          const double Ee = exp(-gam * a.g.Lz);
          const double den = gam * (1.0 - Ee * Ee);
          Ar = (tr - br * Ee) / den;
          Aim = (ti - bi * Ee) / den;
          Br = -(br - tr * Ee) / den;
          Bim = -(bi - ti * Ee) / den;
        }
        W[8] = Ar; W[9] = Aim; W[10] = Br; W[11] = Bim; W[12] = D;
      }
    } else if constexpr (P == 5) {  // Phi, Phi' at the 2d end points -> smem
      for (int q = r; q < 2 * d; q += E::G) {
        const int s = q < d ? q : Nz - 2 * d + q;
        C ph, dph;
        const T cf[5] = {(T)W[8], (T)W[9], (T)W[10], (T)W[11], (T)W[12]};
        phi_at(cf, kxo, kyo, (T)a.g.dz, (T)a.g.Lz, s, &ph, &dph);
        Ev[q < d ? q : DMAX + (q - d)] = ph;
        Ev[2 * DMAX + (q < d ? q : DMAX + (q - d))] = dph;
      }
    } else if constexpr (P == 6) {  // X -= grad phi^I + FC(grad phi^H); wall planes
      if (r < L2 && valid) {
        const T cf[5] = {(T)W[8], (T)W[9], (T)W[10], (T)W[11], (T)W[12]};
        const T tdz = (T)a.g.dz, tLz = (T)a.g.Lz;
#pragma unroll
        for (int j = 0; j < JN; ++j) {
          const int n = r + L2 * j;
          if (n < Np) {
            C ph, dph;
            if (n < Nz) {
              phi_at(cf, kxo, kyo, tdz, tLz, n, &ph, &dph);
            } else {
              ph = continuation_value<T>(n - Nz, Ev, Ev + DMAX, d, a.g.Cc, Ms, Ms2);
              dph = continuation_value<T>(n - Nz, Ev + 2 * DMAX, Ev + 3 * DMAX, d, a.g.Cc, Ms, Ms2);
            }
            const int o = n * TL;
            const C sg = g1[n * GS];
            const C sz = g0[n * GS];
            // i k Phi = (-k Phi.y, k Phi.x)
            const C gx = cadd(cscale(sg, kxo), mk<T>(-kxo * ph.y, kxo * ph.x));
            const C gy = cadd(cscale(sg, kyo), mk<T>(-kyo * ph.y, kyo * ph.x));
            const C gz = cadd(sz, dph);
            xu[o] = csub(xu[o], gx);
            xv[o] = csub(xv[o], gy);
            xw[o] = csub(xw[o], gz);
            if (n == 0 || n == Nz - 1) {
              const int wall = (n == 0) ? 0 : 1;
              const double s = 1.0 / a.dtj;
              a.gradp[((long long)wall * 2 + 0) * Ls + line] = make_double2((double)gx.x * s, (double)gx.y * s);
              a.gradp[((long long)wall * 2 + 1) * Ls + line] = make_double2((double)gy.x * s, (double)gy.y * s);
            }
          }
        }
      }
    }
  }

  // Phi and Phi' at physical point s from the float64 coefficients W[8..12]
  // (evaluated in the path's precision)
  static FC_NOINLINE void phi_at(const T* cf, T kxo, T kyo, T dz, T Lz, int s, C* ph, C* dph) {
    if (kxo == T(0) && kyo == T(0)) {
      *ph = mk<T>(0, 0);
      *dph = mk<T>(cf[4], 0);
      return;
    }
    const T z = (T)s * dz;
    T gam, e1, e2;
    if constexpr (sizeof(T) == 4) {
      gam = sqrtf(kxo * kxo + kyo * kyo);
      e1 = expf(gam * (z - Lz));
      e2 = expf(-gam * z);
    } else {
      gam = sqrt(kxo * kxo + kyo * kyo);
      e1 = exp(gam * (z - Lz));
      e2 = exp(-gam * z);
    }
    const T Ar = cf[0], Aim = cf[1], Br = cf[2], Bim = cf[3];
    *ph = mk<T>(Ar * e1 + Br * e2, Aim * e1 + Bim * e2);
    *dph = mk<T>(gam * (Ar * e1 - Br * e2), gam * (Aim * e1 - Bim * e2));
  }
};

// ===========================================================================
// Y transforms (length Ny, 2/3/5-smooth, no padding).  Lines are kx
// (contiguous), the transform runs over ky with stride Kx, one z plane per
// grid row.  Arrays are [nf][planes_total][Ny][Kx]; the kernel touches planes
// 0..Nz-1 of every field.
// ===========================================================================
struct YGeom {
  int Ny, Kx, Kxp, Nz;
  long long plane;          // Ny * Kxp (lines)
  long long ntiles;
};

// yinv3: V = IFFT_y(A), DY = IFFT_y(i ky A), DZ <- IFFT_y(DZ) (1/Ny included)
template <class T, int L1, int L2, int LINES>
struct KYInv3 {
  using E = Eng<T, L1, L2, LINES>;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 4;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  struct Args {
    YGeom g;
    const C* tw;
    const T* kyo;
    const C* A; long long a_fstride;   // rows per field of the source array
    C* V; C* DY; C* DZ;                 // [nf][Nz][Ny][Kx]
    long long tiles;                    // tiles per plane
    T scale;
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t smem_bytes = 2 * sizeof(C) * E::BUF;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    C* b1 = b0 + E::BUF;
    const int r = tid / LINES, li = tid % LINES;
    const long long tile = bid % a.tiles;
    const long long pz = bid / a.tiles;          // f * Nz + z
    const long long f = pz / a.g.Nz, z = pz % a.g.Nz;
    const int kx = (int)(tile * LINES + li);
    const bool valid = kx < a.g.Kx;
    // line = ky * Kxp + kx with Kxp a multiple of TL: element offset base + ky * Kxp * Z
    const int sb = lay(f, z, kx, a.a_fstride, a.g.ntiles), ss = a.g.Kxp * (int)a.a_fstride;
    const int mb = lay(f, z, kx, a.g.Nz, a.g.ntiles), ms = a.g.Kxp * a.g.Nz;
    auto src = [&](int ky) { return a.A[sb + ky * ss]; };
    auto mo = [&](int y) { return mb + y * ms; };
    if constexpr (P == 0) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          R.v[j] = valid ? src(r + L2 * j) : mk<T>(0, 0);
          b1[E::bidx(j, r, li)] = R.v[j];   // raw copy for the dy transform (own slots)
        }
        E::template A<1>(R.v, b0, a.tw, r, li);
      }
    } else if constexpr (P == 1) {
      if (r < L1) {
        E::template B<1>(R.u, b0, r, li);
        if (valid)
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) a.V[mo(r + L1 * k2)] = cscale(R.u[k2], a.scale);
      }
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int ky = r + L2 * j;
          const C x = b1[E::bidx(j, r, li)];
          const T k = a.kyo[ky];
          R.v[j] = mk<T>(-k * x.y, k * x.x);
        }
        E::template A<1>(R.v, b1, a.tw, r, li);
      }
    } else if constexpr (P == 2) {
      if (r < L1) {
        E::template B<1>(R.u, b1, r, li);
        if (valid)
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) a.DY[mo(r + L1 * k2)] = cscale(R.u[k2], a.scale);
      }
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) R.v[j] = valid ? a.DZ[mo(r + L2 * j)] : mk<T>(0, 0);
        E::template A<1>(R.v, b0, a.tw, r, li);
      }
    } else if constexpr (P == 3) {
      if (r < L1) {
        E::template B<1>(R.u, b0, r, li);
        if (valid)
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) a.DZ[mo(r + L1 * k2)] = cscale(R.u[k2], a.scale);
      }
    }
  }
};

// yinv3 with one exchange buffer (wide tiles: 16 lines = 128 contiguous bytes
// of every ky row): the three transforms run one after another, and the dy
// transform reads its input A again from global memory (the same CTA read it
// one transform earlier, so it comes from L2)
template <class T, int L1, int L2, int LINES>
struct KYInv3S {
  using E = Eng<T, L1, L2, LINES>;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 6;
  static constexpr int MINB = 1;
  using Args = typename KYInv3<T, L1, L2, LINES>::Args;
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t smem_bytes = sizeof(C) * E::BUF;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    const int r = tid / LINES, li = tid % LINES;
    const long long tile = bid % a.tiles;
    const long long pz = bid / a.tiles;          // f * Nz + z
    const long long f = pz / a.g.Nz, z = pz % a.g.Nz;
    const int kx = (int)(tile * LINES + li);
    const bool valid = kx < a.g.Kx;
    const int sb = lay(f, z, kx, a.a_fstride, a.g.ntiles), ss = a.g.Kxp * (int)a.a_fstride;
    const int mb = lay(f, z, kx, a.g.Nz, a.g.ntiles), ms = a.g.Kxp * a.g.Nz;
    auto mo = [&](int y) { return mb + y * ms; };
    if constexpr (P == 0 || P == 2 || P == 4) {
      if (r < L2) {
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int ky = r + L2 * j;
          C x = mk<T>(0, 0);
          if (valid) {
            if constexpr (P == 4) {
              x = a.DZ[mo(ky)];
            } else {
              x = a.A[sb + ky * ss];
              if constexpr (P == 2) {
                const T k = a.kyo[ky];
                x = mk<T>(-k * x.y, k * x.x);
              }
            }
          }
          R.v[j] = x;
        }
        E::template A<1>(R.v, b0, a.tw, r, li);
      }
    } else {
      if (r < L1) {
        E::template B<1>(R.u, b0, r, li);
        C* out = P == 1 ? a.V : (P == 3 ? a.DY : a.DZ);
        if (valid)
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) out[mo(r + L1 * k2)] = cscale(R.u[k2], a.scale);
      }
    }
  }
};

// y1: one transform per plane, OUT = scale * FFT_y^{SIGN}(IN) (may alias)
template <class T, int L1, int L2, int LINES, int SIGN>
struct KY1 {
  using E = Eng<T, L1, L2, LINES>;
  using C = cx<T>;
  static constexpr int THREADS = E::THREADS, NPHASE = 2;
  static constexpr int MINB = THREADS <= 160 ? 3 : (THREADS <= 320 ? 2 : 1);
  struct Args {
    YGeom g;
    const C* tw;
    const C* IN; long long in_fstride;   // planes between fields of IN
    C* OUT; long long out_fstride;
    long long tiles;
    T scale;
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t smem_bytes = sizeof(C) * E::BUF;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    C* b0 = reinterpret_cast<C*>(sm);
    const int r = tid / LINES, li = tid % LINES;
    const long long tile = bid % a.tiles;
    const long long pz = bid / a.tiles;
    const long long f = pz / a.g.Nz, z = pz % a.g.Nz;
    const int kx = (int)(tile * LINES + li);
    const bool valid = kx < a.g.Kx;
    if constexpr (P == 0) {
      if (r < L2) {
        const int ib = lay(f, z, kx, a.in_fstride, a.g.ntiles), is = a.g.Kxp * (int)a.in_fstride;
#pragma unroll
        for (int j = 0; j < L1; ++j) R.v[j] = valid ? a.IN[ib + (r + L2 * j) * is] : mk<T>(0, 0);
        E::template A<SIGN>(R.v, b0, a.tw, r, li);
      }
    } else {
      if (r < L1) {
        E::template B<SIGN>(R.u, b0, r, li);
        const int ob = lay(f, z, kx, a.out_fstride, a.g.ntiles), os = a.g.Kxp * (int)a.out_fstride;
        if (valid)
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) a.OUT[ob + (r + L1 * k2) * os] = cscale(R.u[k2], a.scale);
      }
    }
  }
};

// ===========================================================================
// X transforms: one CTA per (y, z) row (all fields), row FFTs of length Nx in
// shared memory; groups of G threads per transform.
// ===========================================================================
// factors of the length-Nx/2 transform of the x pass's forward half (real
// rows split into even / odd samples): L1 halved when even, else L2
constexpr int half_l1(int L1, int L2) { return L1 % 2 == 0 ? L1 / 2 : L1; }
constexpr int half_l2(int L1, int L2) { return L1 % 2 == 0 ? L2 : L2 / 2; }

template <class T, int L1_, int L2_>
struct RowEng {
  static constexpr int L1 = L1_, L2 = L2_;
  static constexpr int L = L1 * L2;
  static constexpr int G = L1 > L2 ? L1 : L2;
  static constexpr int ROW = L2 + 1;     // padded exchange row
  static constexpr int BUF = L1 * ROW;
  using C = cx<T>;
  static FC_HD C twid(const C* tw, int n2, int k1, int sign) {
    C w = tw[n2 * L1 + k1];
    if (sign > 0) w.y = -w.y;
    return w;
  }
  template <int SIGN>
  static FC_HD void A(C (&v)[L1], C* buf, const C* tw, int n2) {
    dft_reg<L1, SIGN, T>(v);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) {
      if (k1 % 6 == 0) FC_FENCE();
      C w = tw[L + k1 * L2 + n2];   // A-side copy of the twiddles: contiguous across lanes
      if (SIGN > 0) w.y = -w.y;
      buf[k1 * ROW + n2] = cmul(v[k1], w);
    }
  }
  template <int SIGN>
  static FC_HD void B(C (&u)[L2], const C* buf, int k1) {
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) u[n2] = buf[k1 * ROW + n2];
    dft_reg<L2, SIGN, T>(u);
  }
};

// xpass: nonlinear products of one row.  For every field f the real rows
// v_f, dx v_f, dy v_f, dz v_f are obtained by complex inverse transforms of
// pairs (v + i dx v), (dy v + i dz v) of Hermitian half spectra; the products
//   N_f = -(u dx + v dy + w dz) v_f (+ F on u; + gamma theta on w; + gamma w
//   on theta) are formed in physical space (Sec. 4.2, Sec. 6, Sec. 7) and
// transformed back in pairs (N_a + i N_b).
template <class T, int L1, int L2, int NF>
struct KXPass {
  using RE = RowEng<T, L1, L2>;
  // the forward transforms: one length-Nx/2 complex transform per real row
  using RH = RowEng<T, half_l1(L1, L2), half_l2(L1, L2)>;
  using C = cx<T>;
  static constexpr int Nx = L1 * L2, G = RE::G, NJOB = 2 * NF, NFWD = (NF + 1) / 2;
  static_assert(RH::G <= G && RH::BUF <= RE::BUF && Nx / 2 <= RE::BUF, "half-length row engine");
  // forward half: one length-Nx/2 transform per real row (all NF groups) for
  // Nx >= 1024, where it measured faster (1024^2 x 513 step 232.4 -> 228.4 ms);
  // else two real rows per length-Nx transform on NFWD groups (Nx = 256:
  // 0.85 against 0.93 ms per launch).  The host-check build switches at 32,
  // so that its x lengths (16, 32, 128) run both forms.
#ifdef FC_HOSTCHECK
  static constexpr bool HALF = Nx >= 32;
#else
  static constexpr bool HALF = Nx >= 1024;
#endif
  static constexpr int THREADS = NJOB * G, NPHASE = 8, MINB = 2;
  struct Args {
    int Kx, Kxp, Ny, Nz;
    long long rows;          // Nz * Ny
    long long ntiles;
    const C* tw;             // Nx engine twiddles
    const C* twh;            // Nx/2 engine twiddles (Nx entries), then e^{-2 pi i k/Nx}, k = 0..Nx/2
    const T* kxo;            // Kx
    const C* V; const C* DY; const C* DZ;   // [NF][rows][Kx]
    C* NL;                                  // [NF][rows][Kx]
    T forcing, gamma, scale;                // scale = 1/Nx
  };
  struct Regs { C v[L1]; C u[L2]; C vh[RH::L1]; C uh[RH::L2]; };
  // the real rows Pr alias the exchange buffers (phases separate every reuse)
  static constexpr size_t zb_bytes = sizeof(C) * RE::BUF * NJOB;
  static constexpr size_t pr_bytes = sizeof(T) * 4 * NF * Nx;
  static constexpr size_t smem_bytes = zb_bytes > pr_bytes ? zb_bytes : pr_bytes;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long row, Regs& R) {
    C* Zb = reinterpret_cast<C*>(sm);
    T* Pr = reinterpret_cast<T*>(sm);
    const int q = tid / G, g = tid % G;
    const long long Kx = a.Kx;
    if constexpr (P == 0) {  // pair spectra (v + i dx v), (dy v + i dz v), inverse first half
      if (g < L2) {
        const int f = q / 2, type = q % 2;
        const C* A = (type == 0 ? a.V : a.DY);
        const long long z = row / a.Ny, yb = (row % a.Ny) * a.Kxp;
#pragma unroll
        for (int j = 0; j < L1; ++j) {
          const int k = g + L2 * j;
          const bool up = k > Nx / 2;
          const int kk = up ? Nx - k : k;
          const long long o = lay(f, z, yb + kk, a.Nz, a.ntiles);
          C av = A[o], bv;
          if (type == 0) {
            const T kx = a.kxo[kk];
            bv = mk<T>(-kx * av.y, kx * av.x);
          } else {
            bv = a.DZ[o];
          }
          if (kk == 0 || kk == Nx / 2) { av.y = T(0); bv.y = T(0); }
          if (up) { av.y = -av.y; bv.y = -bv.y; }
          R.v[j] = mk<T>(av.x - bv.y, av.y + bv.x);  // A + i B
        }
        RE::template A<1>(R.v, Zb + q * RE::BUF, a.tw, g);
      }
    } else if constexpr (P == 1) {
      if (g < L1) RE::template B<1>(R.u, Zb + q * RE::BUF, g);
    } else if constexpr (P == 2) {  // real rows v_f, dx v_f, dy v_f, dz v_f
      if (g < L1) {
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) {
          const int n = g + L1 * k2;
          Pr[(2 * q) * Nx + n] = R.u[k2].x * a.scale;
          Pr[(2 * q + 1) * Nx + n] = R.u[k2].y * a.scale;
        }
      }
    } else if constexpr (P == 3) {  // products (Sec. 4.2, Sec. 6, Sec. 7)
      for (int n = tid; n < Nx; n += THREADS) {
        const T u = Pr[0 * Nx + n], v = Pr[4 * Nx + n], w = Pr[8 * Nx + n];
        T Nf[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f)
          Nf[f] = -(u * Pr[(4 * f + 1) * Nx + n] + v * Pr[(4 * f + 2) * Nx + n] + w * Pr[(4 * f + 3) * Nx + n]);
        Nf[0] += a.forcing;
        if constexpr (NF == 4) {
          Nf[2] += a.gamma * Pr[12 * Nx + n];
          Nf[3] += a.gamma * w;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) Pr[f * Nx + n] = Nf[f];
      }
    } else if constexpr (HALF) {
      if constexpr (P == 4) {  // z_f[m] = N_f[2m] + i N_f[2m+1], one group per field
        if (q < NF && g < RH::L2) {
#pragma unroll
          for (int j = 0; j < RH::L1; ++j) {
            const int m = g + RH::L2 * j;
            R.vh[j] = mk<T>(Pr[q * Nx + 2 * m], Pr[q * Nx + 2 * m + 1]);
          }
        }
      } else if constexpr (P == 5) {
        if (q < NF && g < RH::L2) RH::template A<-1>(R.vh, Zb + q * RE::BUF, a.twh, g);
      } else if constexpr (P == 6) {
        if (q < NF && g < RH::L1) {
          RH::template B<-1>(R.uh, Zb + q * RE::BUF, g);
          C* Zn = Zb + (NF + q) * RE::BUF;   // natural order spectrum Z_f (length Nx/2)
#pragma unroll
          for (int k2 = 0; k2 < RH::L2; ++k2) Zn[g + RH::L1 * k2] = R.uh[k2];
        }
      } else if constexpr (P == 7) {
        // half spectrum of the real row: with E = FFT(N_f[2m]) and
        // O = FFT(N_f[2m+1]) (length Nx/2, read off Z_f by its Hermitian
        // parts), X_k = E_k + e^{-2 pi i k/Nx} O_k, k = 0..Nx/2
        constexpr int H = Nx / 2;
        const long long z = row / a.Ny, yb = (row % a.Ny) * a.Kxp;
        for (int i = tid; i < NF * (H + 1); i += THREADS) {
          const int f = i / (H + 1), k = i % (H + 1);
          const C* Zn = Zb + (NF + f) * RE::BUF;
          const C zk = Zn[k % H], zm = Zn[(H - k) % H];
          const C Ev = mk<T>((zk.x + zm.x) * T(0.5), (zk.y - zm.y) * T(0.5));
          const C Ov = mk<T>((zk.y + zm.y) * T(0.5), (zm.x - zk.x) * T(0.5));
          a.NL[lay(f, z, yb + k, a.Nz, a.ntiles)] = cadd(Ev, cmul(a.twh[Nx + k], Ov));
        }
      }
    } else {
      if constexpr (P == 4) {  // pairs (N_a + i N_b) of real rows
        if (q < NFWD && g < L2) {
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = g + L2 * j;
            const T re = Pr[(2 * q) * Nx + n];
            const T im = (2 * q + 1 < NF) ? Pr[(2 * q + 1) * Nx + n] : T(0);
            R.v[j] = mk<T>(re, im);
          }
        }
      } else if constexpr (P == 5) {
        if (q < NFWD && g < L2) RE::template A<-1>(R.v, Zb + q * RE::BUF, a.tw, g);
      } else if constexpr (P == 6) {
        if (q < NFWD && g < L1) {
          RE::template B<-1>(R.u, Zb + q * RE::BUF, g);
          C* Zn = Zb + (NFWD + q) * RE::BUF;   // natural order spectrum
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) Zn[g + L1 * k2] = R.u[k2];
        }
      } else if constexpr (P == 7) {
        const long long z = row / a.Ny, yb = (row % a.Ny) * a.Kxp;
        for (int i = tid; i < NFWD * (Nx / 2 + 1); i += THREADS) {
          const int qq = i / (Nx / 2 + 1), k = i % (Nx / 2 + 1);
          const C* Zn = Zb + (NFWD + qq) * RE::BUF;
          const C zk = Zn[k], zm = Zn[(Nx - k) % Nx];
          // A = (Z_k + conj Z_{N-k}) / 2,  B = (Z_k - conj Z_{N-k}) / (2i)
          const C Av = mk<T>((zk.x + zm.x) * T(0.5), (zk.y - zm.y) * T(0.5));
          const C Bv = mk<T>((zk.y + zm.y) * T(0.5), (zm.x - zk.x) * T(0.5));
          a.NL[lay(2 * qq, z, yb + k, a.Nz, a.ntiles)] = Av;
          if (2 * qq + 1 < NF) a.NL[lay(2 * qq + 1, z, yb + k, a.Nz, a.ntiles)] = Bv;
        }
      }
    }
  }
};

// xfwd: real rows -> Hermitian half spectra, two rows per complex transform.
// xinv: half spectra -> real rows (scale 1/Nx), two rows per transform.
template <class T, int L1, int L2, int SIGN, int JOBS>
struct KXRow {
  using RE = RowEng<T, L1, L2>;
  using C = cx<T>;
  static constexpr int Nx = L1 * L2, G = RE::G;
  static constexpr int THREADS = JOBS * G, NPHASE = 3, MINB = 1;
  struct Args {
    int Kx, Kxp, Ny, Nz;
    long long pairs;        // number of row pairs (rows / 2)
    long long ntiles;
    const C* tw;
    const T* R; C* S;       // SIGN = -1: R -> S;  SIGN = +1: S -> R
    T scale;
  };
  struct Regs { C v[L1]; C u[L2]; };
  static constexpr size_t smem_bytes = sizeof(C) * RE::BUF * JOBS * 2;

  // element k of row R (rows ordered [f][z][y]) in the tiled layout
  static FC_HD long long sidx(const Args& a, long long R, long long k) {
    const long long y = R % a.Ny, fz = R / a.Ny;
    return lay(fz / a.Nz, fz % a.Nz, y * a.Kxp + k, a.Nz, a.ntiles);
  }
  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& Rg) {
    const int q = tid / G, g = tid % G;
    const long long pair = bid * JOBS + q;
    const bool valid = pair < a.pairs;
    C* Zb = reinterpret_cast<C*>(sm) + q * RE::BUF;
    C* Zn = reinterpret_cast<C*>(sm) + (JOBS + q) * RE::BUF;
    const long long Kx = a.Kx;
    if constexpr (SIGN < 0) {
      const T* r0 = a.R + (2 * pair) * Nx;
      if constexpr (P == 0) {
        if (g < L2) {
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int n = g + L2 * j;
            Rg.v[j] = valid ? mk<T>(r0[n], r0[Nx + n]) : mk<T>(0, 0);
          }
          RE::template A<-1>(Rg.v, Zb, a.tw, g);
        }
      } else if constexpr (P == 1) {
        if (g < L1) {
          RE::template B<-1>(Rg.u, Zb, g);
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) Zn[g + L1 * k2] = Rg.u[k2];
        }
      } else {
        if (valid)
          for (int k = g; k <= Nx / 2; k += G) {
            const C zk = Zn[k], zm = Zn[(Nx - k) % Nx];
            a.S[sidx(a, 2 * pair, k)] = mk<T>((zk.x + zm.x) * T(0.5), (zk.y - zm.y) * T(0.5));
            a.S[sidx(a, 2 * pair + 1, k)] = mk<T>((zk.y + zm.y) * T(0.5), (zm.x - zk.x) * T(0.5));
          }
      }
    } else {
      if constexpr (P == 0) {
        if (g < L2) {
#pragma unroll
          for (int j = 0; j < L1; ++j) {
            const int k = g + L2 * j;
            const bool up = k > Nx / 2;
            const int kk = up ? Nx - k : k;
            C av = valid ? a.S[sidx(a, 2 * pair, kk)] : mk<T>(0, 0);
            C bv = valid ? a.S[sidx(a, 2 * pair + 1, kk)] : mk<T>(0, 0);
            if (kk == 0 || kk == Nx / 2) { av.y = T(0); bv.y = T(0); }
            if (up) { av.y = -av.y; bv.y = -bv.y; }
            Rg.v[j] = mk<T>(av.x - bv.y, av.y + bv.x);
          }
          RE::template A<1>(Rg.v, Zb, a.tw, g);
        }
      } else if constexpr (P == 1) {
        if (g < L1) {
          RE::template B<1>(Rg.u, Zb, g);
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) Zn[g + L1 * k2] = Rg.u[k2];
        }
      } else {
        if (valid) {
          T* r0 = const_cast<T*>(a.R) + (2 * pair) * Nx;
          for (int n = g; n < Nx; n += G) {
            r0[n] = Zn[n].x * a.scale;
            r0[Nx + n] = Zn[n].y * a.scale;
          }
        }
      }
    }
  }
};

}  // namespace fcns

namespace fcns {

// ===========================================================================
// Diagnostics of the state (Sec. 6: divergence and wall velocities; Sec. 7:
// Nusselt number; channel flow rate), reduced in float64.  Mean squares over
// the physical grid follow from the mixed-space values by Parseval over the
// half spectrum: weight 1 at kx = 0 and kx = Nx/2, 2 elsewhere, / (Nx Ny)^2.
//   acc[0] += sum over z, lines of w |i kx u + i ky v + dz w|^2
//   acc[1] += sum over both walls of w |u|^2,   acc[2] += ... of w |w|^2
//   acc[3] += sum over z of Re u(kx=0, ky=0, z)          (flow rate)
//   acc[4] += Re dz theta(0, 0, z=0),  acc[5] += Re dz theta(0, 0, z=Lz)
// ===========================================================================
template <class T>
struct KDiag {
  using C = cx<T>;
  static constexpr int THREADS = 256, NPHASE = 2, MINB = 1;
  struct Args {
    ZGeom g;
    ZTab<T> t;
    int Nx;
    const C* X;     // state (extended), [nf][N'][lines]
    const C* DZ;    // dz of the state at the Nz points, [nf][Nz][lines]
    double* acc;    // 6 accumulators
  };
  struct Regs { double s[6]; };
  static constexpr size_t smem_bytes = sizeof(double) * 6 * THREADS;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    double* red = reinterpret_cast<double*>(sm);
    if constexpr (P == 0) {
      for (int i = 0; i < 6; ++i) R.s[i] = 0.0;
      const int li = tid % TL, zr = tid / TL;           // 16 lines x 16 z rows per pass
      const long long line = bid * TL + li;
      const int Nz = a.g.Nz, Np = a.g.Np;
      const int kx = (int)(line % a.g.Kxp), ky = (int)(line / a.g.Kxp);
      if (line < a.g.lines && kx < a.g.Kx) {
        const double wgt = (kx == 0 || 2 * kx == a.Nx) ? 1.0 : 2.0;
        const double kxo = (double)a.t.kxo[kx], kyo = (double)a.t.kyo[ky];
        const C* u = a.X + lay(0, 0, line, Np, a.g.ntiles);
        const C* v = a.X + lay(1, 0, line, Np, a.g.ntiles);
        const C* w = a.X + lay(2, 0, line, Np, a.g.ntiles);
        const C* dw = a.DZ + lay(2, 0, line, Nz, a.g.ntiles);
        for (int z = zr; z < Nz; z += THREADS / TL) {
          const C uu = u[z * TL], vv = v[z * TL], ww = w[z * TL], dd = dw[z * TL];
          // i kx u + i ky v + dz w
          const double re = -kxo * (double)uu.y - kyo * (double)vv.y + (double)dd.x;
          const double im = kxo * (double)uu.x + kyo * (double)vv.x + (double)dd.y;
          R.s[0] += wgt * (re * re + im * im);
          if (z == 0 || z == Nz - 1) {
            R.s[1] += wgt * ((double)uu.x * uu.x + (double)uu.y * uu.y);
            R.s[2] += wgt * ((double)ww.x * ww.x + (double)ww.y * ww.y);
          }
          if (kx == 0 && ky == 0) R.s[3] += (double)uu.x;
        }
        if (kx == 0 && ky == 0 && zr == 0 && a.g.nf == 4) {
          const C* dt = a.DZ + lay(3, 0, line, Nz, a.g.ntiles);
          R.s[4] = (double)dt[0].x;
          R.s[5] = (double)dt[(Nz - 1) * TL].x;
        }
      }
      for (int i = 0; i < 6; ++i) red[i * THREADS + tid] = R.s[i];
    } else {
      if (tid < 6) {
        double s = 0.0;
        for (int t = 0; t < THREADS; ++t) s += red[tid * THREADS + t];
        if (s != 0.0) {
#if defined(__CUDA_ARCH__)
          atomicAdd(a.acc + tid, s);
#else
          a.acc[tid] += s;
#endif
        }
      }
    }
  }
};

}  // namespace fcns

namespace fcns {

// ===========================================================================
// Float64 island of the float32 path: the RK accumulation of the mean-flow
// line (kx, ky) = (0, 0) of u, v and theta (the fields the projection leaves
// unchanged on that line) is redone in float64 from a float64 shadow of the
// line:  v* = v^t + dt_j [ (f_z * FC(N))(z) + nu dzz v^{j-1} ]  (direct sums
// with the float64 real-space kernels), wall injection, continuation, and
// both the shadow and the float32 state line are written.  One block per
// field; runs after the stage combine.
// ===========================================================================
template <class T>
struct KMean {
  using C = cx<T>;
  // NPMAX: the longest continued line held in shared memory (two lines); it
  // covers every compiled z length (N' <= 1536), and ns_layout refuses longer
  static constexpr int THREADS = 256, NPHASE = 4, MINB = 1, NPMAX = 1536;
  struct Args {
    ZGeom g;
    const double* Mr;       // C x d
    const double* d2;       // [Np + Nz - 1] real-space kernels (unit spacing)
    const double* hf;
    const C* NL;            // nonlinear term (mixed), float32 path
    const double2* Xt;      // shadows [3][Np] (u, v, theta)
    const double2* Xj;
    double2* Xn;
    C* Xo;                  // float32 state buffer of this stage
    const double2* gradp;   // wall planes (line 0 entries)
    double dtj;
    double dif[3];
    double fxy00;
    int fmap[3];            // field index of shadow entry 0, 1, 2
    int nmean;              // 2 (Navier-Stokes: u, v) or 3 (Boussinesq: u, v, theta)
  };
  struct Regs { int dummy; };
  static constexpr size_t smem_bytes = 2 * sizeof(double2) * NPMAX;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs&) {
    double2* nl = reinterpret_cast<double2*>(sm);
    double2* vs = nl + NPMAX;
    const int e = (int)bid, f = a.fmap[e];
    const int Nz = a.g.Nz, Np = a.g.Np, d = a.g.d, Cc = a.g.Cc;
    const int jlo = -(Np - 1);
    auto cont = [&](const double2* x, int jj) {
      dd re{0.0, 0.0}, im{0.0, 0.0};
      for (int i = 0; i < d; ++i) {
        const double m1 = a.Mr[jj * d + i], m2 = a.Mr[(Cc - 1 - jj) * d + (d - 1 - i)];
        dd_fma(re, m1, x[Nz - d + i].x);
        dd_fma(im, m1, x[Nz - d + i].y);
        dd_fma(re, m2, x[i].x);
        dd_fma(im, m2, x[i].y);
      }
      return make_double2(dd_round(re), dd_round(im));
    };
    if constexpr (P == 0) {
      const C* src = a.NL + lay(f, 0, 0, Nz, a.g.ntiles);
      for (int z = tid; z < Nz; z += THREADS) nl[z] = make_double2((double)src[z * TL].x, (double)src[z * TL].y);
    } else if constexpr (P == 1) {
      for (int z = Nz + tid; z < Np; z += THREADS) nl[z] = cont(nl, z - Nz);
    } else if constexpr (P == 2) {
      const double2* xt = a.Xt + (long long)e * Np;
      const double2* xj = a.Xj + (long long)e * Np;
      const double s2 = 1.0 / (a.g.dz * a.g.dz);
      for (int z = tid; z < Nz; z += THREADS) {
        double fr = 0, fi = 0, zr = 0, zi = 0;
        for (int m = 0; m < Np; ++m) {
          const double hk = a.hf[z - m - jlo], dk = a.d2[z - m - jlo];
          fr += hk * nl[m].x;
          fi += hk * nl[m].y;
          zr += dk * xj[m].x;
          zi += dk * xj[m].y;
        }
        double2 v = make_double2(xt[z].x + a.dtj * (a.fxy00 * fr + a.dif[e] * zr * s2),
                                 xt[z].y + a.dtj * (a.fxy00 * fi + a.dif[e] * zi * s2));
        if (z == 0 || z == Nz - 1) {
          const int wall = (z == 0) ? 0 : 1;
          if (f < 2) {
            const double2 gp = a.gradp[((long long)wall * 2 + f) * a.g.lines];
            v = make_double2(a.dtj * gp.x, a.dtj * gp.y);
          } else {
            v = make_double2(0.0, 0.0);
          }
        }
        vs[z] = v;
      }
    } else if constexpr (P == 3) {
      for (int z = Nz + tid; z < Np; z += THREADS) vs[z] = cont(vs, z - Nz);
    }
  }
  // final write (after a barrier): shadow and float32 line
  static FC_HD void write(const Args& a, unsigned char* sm, int tid, long long bid) {
    const double2* vs = reinterpret_cast<const double2*>(sm) + NPMAX;
    const int e = (int)bid, f = a.fmap[e];
    C* xo = a.Xo + lay(f, 0, 0, a.g.Np, a.g.ntiles);
    for (int z = tid; z < a.g.Np; z += THREADS) {
      a.Xn[(long long)e * a.g.Np + z] = vs[z];
      xo[z * TL] = mk<T>((T)vs[z].x, (T)vs[z].y);
    }
  }
};

// wrapper with the final write as its own phase
template <class T>
struct KMeanLine {
  using Base = KMean<T>;
  using Args = typename Base::Args;
  using Regs = typename Base::Regs;
  static constexpr int THREADS = Base::THREADS, NPHASE = 5, MINB = 1;
  static constexpr size_t smem_bytes = Base::smem_bytes;
  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& r) {
    if constexpr (P < 4) Base::template phase<P>(a, sm, tid, bid, r);
    else Base::write(a, sm, tid, bid);
  }
};

// ===========================================================================
// KInterp  restart on a finer grid (Sec. 6, spectral interpolation): for every
// (kx, ky) line of the destination grid, the source line with the same
// wavenumbers (zero padding in x, y; a coarse Nyquist coefficient, which
// stands for a cosine, split in half between +N/2 and -N/2) has its
// N'-periodic z series evaluated at the destination's Nz physical points:
//   M[f][s][line2] = scale * w * sum_n W[s][n] X1[f][n][line1].
// Block: 16 destination lines (one tile) x 16 rows s; thread (s % 16, line).
// ===========================================================================
template <class T>
struct KInterp {
  using C = cx<T>;
  static constexpr int THREADS = 256, NPHASE = 1, MINB = 2;
  struct Args {
    const C* X1;        // source state, tiled [nf][N'1][lines1]
    int Np1, Kx1, Kxp1, Ny1, Nx1;
    long long ntiles1;
    C* M2;              // destination mixed rows, tiled [nf][Nz2][lines2]
    int Nz2, Kx2, Kxp2, Ny2, Nx2;
    long long ntiles2;
    const C* W;         // [Nz2][N'1] evaluation weights (1/N'1 included)
    T scale;            // (Nx2 Ny2) / (Nx1 Ny1)
    int sblocks;        // ceil(Nz2 / 16)
  };
  struct Regs { int dummy; };
  static constexpr size_t smem_bytes = 16;

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char*, int tid, long long bid, Regs&) {
    const int li = tid & 15, sl = tid >> 4;
    const long long tile = (bid / a.sblocks) % a.ntiles2;
    const int f = (int)(bid / a.sblocks / a.ntiles2);
    const int s = (int)(bid % a.sblocks) * 16 + sl;
    if (s >= a.Nz2) return;
    const long long line2 = tile * TL + li;
    const int kx2 = (int)(line2 % a.Kxp2), ky2 = (int)(line2 / a.Kxp2);
    C acc = mk<T>(0, 0);
    // source line and weight of this destination mode (none: zero)
    int kx1 = -1, ky1 = -1;
    T w = a.scale;
    if (kx2 < a.Kx2 && ky2 < a.Ny2) {
      if (a.Nx2 == a.Nx1) kx1 = kx2;
      else if (kx2 < a.Nx1 / 2) kx1 = kx2;
      else if (kx2 == a.Nx1 / 2) { kx1 = kx2; w *= T(0.5); }
      const int m = ky2 < a.Ny2 / 2 ? ky2 : ky2 - a.Ny2;   // signed ky (sizes are even)
      if (a.Ny2 == a.Ny1) ky1 = ky2;
      else if (2 * (m < 0 ? -m : m) < a.Ny1) ky1 = m < 0 ? m + a.Ny1 : m;
      else if (2 * (m < 0 ? -m : m) == a.Ny1) { ky1 = a.Ny1 / 2; w *= T(0.5); }
    }
    if (kx1 >= 0 && ky1 >= 0) {
      const long long line1 = (long long)ky1 * a.Kxp1 + kx1;
      const C* x = a.X1 + lay(f, 0, line1, a.Np1, a.ntiles1);
      const C* wr = a.W + (long long)s * a.Np1;
      for (int n = 0; n < a.Np1; ++n) {
        const C xv = x[n * TL], wv = wr[n];
        acc.x += wv.x * xv.x - wv.y * xv.y;
        acc.y += wv.x * xv.y + wv.y * xv.x;
      }
      acc = cscale(acc, w);
    }
    if (line2 < (long long)a.Ny2 * a.Kxp2) a.M2[lay(f, s, line2, a.Nz2, a.ntiles2)] = acc;
  }
};

// ===========================================================================
// KProf  horizontal statistics per field and physical level z_s (Sec. 6
// r.m.s. profiles and spectra), by Parseval from the state rows n < Nz (the
// state is in (kx, ky, z') space and z' = z at the physical points):
//   sum[f][s]      = sum over (kx, ky) != (0, 0) of w |X|^2   (w = 2 for the
//                    kx stored once for +-kx, else 1)
//   mean[f][s]     = Re X(0, 0)
//   bins[f][s][j]  = sum of w |X|^2 over the modes of shell j = round(|k_perp| / dk)
// (all unnormalised; the host divides by (Nx Ny)^2).  One block per (f, s).
// ===========================================================================
template <class T>
struct KProf {
  using C = cx<T>;
  static constexpr int THREADS = 256, NPHASE = 3, MINB = 2;
  struct Args {
    ZGeom g;
    int Nx;
    const C* X;          // state [nf][N'][lines]
    double kx_unit, ky_unit, dk;   // 2 pi / Lx, 2 pi / Ly, shell width
    int nshell;
    double* out;         // [nf][Nz][2 + nshell]: sum, mean, bins
  };
  struct Regs { double s; };
  static constexpr int NSMAX = 2048;
  static constexpr size_t smem_bytes = sizeof(double) * (THREADS + NSMAX);

  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    double* red = reinterpret_cast<double*>(sm);
    double* bins = red + THREADS;
    const int f = (int)(bid / a.g.Nz), s = (int)(bid % a.g.Nz);
    double* o = a.out + ((long long)f * a.g.Nz + s) * (2 + a.nshell);
    if constexpr (P == 0) {
      for (int j = tid; j < a.nshell; j += THREADS) bins[j] = 0.0;
    } else if constexpr (P == 1) {
      R.s = 0.0;
      for (long long l = tid; l < a.g.lines; l += THREADS) {
        const int kx = (int)(l % a.g.Kxp), ky = (int)(l / a.g.Kxp);
        if (kx >= a.g.Kx) continue;
        const C v = a.X[lay(f, s, l, a.g.Np, a.g.ntiles)];
        if (kx == 0 && ky == 0) {
          o[1] = (double)v.x;
          continue;
        }
        const double w = (kx == 0 || 2 * kx == a.Nx) ? 1.0 : 2.0;
        const double p = w * ((double)v.x * v.x + (double)v.y * v.y);
        R.s += p;
        const int m = ky <= (a.g.Ny - 1) / 2 ? ky : ky - a.g.Ny;
        const double kxp = a.kx_unit * kx, kyp = a.ky_unit * m;
        int j = (int)floor(sqrt(kxp * kxp + kyp * kyp) / a.dk + 0.5);
        if (j >= a.nshell) j = a.nshell - 1;
#if defined(__CUDA_ARCH__)
        atomicAdd(bins + j, p);
#else
        bins[j] += p;
#endif
      }
      red[tid] = R.s;
    } else {
      if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < THREADS; ++i) t += red[i];
        o[0] = t;
      }
      for (int j = tid; j < a.nshell; j += THREADS) o[2 + j] = bins[j];
    }
  }
};

// shadow <- float32 state line 0 of u, v (, theta)
template <class T>
struct KMeanInit {
  using C = cx<T>;
  static constexpr int THREADS = 256, NPHASE = 1, MINB = 1;
  struct Args {
    ZGeom g;
    const C* X;
    double2* X64;
    int fmap[3];
  };
  struct Regs { int dummy; };
  static constexpr size_t smem_bytes = 16;
  template <int P>
  static FC_HD void phase(const Args& a, unsigned char*, int tid, long long bid, Regs&) {
    const int e = (int)bid;
    const C* x = a.X + lay(a.fmap[e], 0, 0, a.g.Np, a.g.ntiles);
    for (int z = tid; z < a.g.Np; z += THREADS)
      a.X64[(long long)e * a.g.Np + z] = make_double2((double)x[z * TL].x, (double)x[z * TL].y);
  }
};

// ===========================================================================
// Non-finite counts (an Inf or NaN in either part of a value counts once per
// real).  KFinite reads the physical lines (kx < Kx) of a state, every field
// and every continued row, one tile of TL lines per CTA; KCount reads a flat
// array of n reals, `per` of them per CTA.  Both add their count to *count.
// ===========================================================================
template <class T>
FC_HD int nonfinite(T v) {
#if defined(__CUDA_ARCH__)
  return isfinite(v) ? 0 : 1;
#else
  return std::isfinite(v) ? 0 : 1;
#endif
}

FC_HD void count_add(unsigned long long* count, unsigned long long n) {
#if defined(__CUDA_ARCH__)
  atomicAdd(count, n);
#else
  *count += n;
#endif
}

template <class T>
struct KFinite {
  using C = cx<T>;
  static constexpr int THREADS = 256, NPHASE = 2, MINB = 1;
  struct Args {
    ZGeom g;
    const C* X;                  // [nf][N'][lines] tiled
    unsigned long long* count;
  };
  struct Regs { unsigned n; };
  static constexpr size_t smem_bytes = sizeof(unsigned) * THREADS;
  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    unsigned* red = reinterpret_cast<unsigned*>(sm);
    if constexpr (P == 0) {
      R.n = 0;
      const int li = tid % TL, zr = tid / TL;
      const long long line = bid * TL + li;
      if (line < a.g.lines && (int)(line % a.g.Kxp) < a.g.Kx)
        for (int f = 0; f < a.g.nf; ++f) {
          const C* x = a.X + lay(f, 0, line, a.g.Np, a.g.ntiles);
          for (int z = zr; z < a.g.Np; z += THREADS / TL) {
            const C v = x[z * TL];
            R.n += nonfinite(v.x) + nonfinite(v.y);
          }
        }
      red[tid] = R.n;
    } else {
      if (tid == 0) {
        unsigned long long s = 0;
        for (int t = 0; t < THREADS; ++t) s += red[t];
        if (s) count_add(a.count, s);
      }
    }
  }
};

template <class T>
struct KCount {
  static constexpr int THREADS = 256, NPHASE = 2, MINB = 1;
  struct Args {
    const T* x;
    long long n, per;
    unsigned long long* count;
  };
  struct Regs { unsigned n; };
  static constexpr size_t smem_bytes = sizeof(unsigned) * THREADS;
  template <int P>
  static FC_HD void phase(const Args& a, unsigned char* sm, int tid, long long bid, Regs& R) {
    unsigned* red = reinterpret_cast<unsigned*>(sm);
    if constexpr (P == 0) {
      R.n = 0;
      const long long b0 = bid * a.per, b1 = b0 + a.per < a.n ? b0 + a.per : a.n;
      for (long long i = b0 + tid; i < b1; i += THREADS) R.n += nonfinite(a.x[i]);
      red[tid] = R.n;
    } else {
      if (tid == 0) {
        unsigned long long s = 0;
        for (int t = 0; t < THREADS; ++t) s += red[t];
        if (s) count_add(a.count, s);
      }
    }
  }
};

}  // namespace fcns
