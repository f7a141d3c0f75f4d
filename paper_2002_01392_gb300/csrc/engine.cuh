// Two-pass line FFT engine shared by the z, y and x kernels.
//
// A transform of length L = L1 * L2 over a tile of LINES lines: input index
// n = n2 + L2 n1 lives in thread r = n2 (register array v[L1]); output index
// k = k1 + L1 k2 lives in thread r = k1 (register array u[L2]).  One
// shared-memory exchange per transform (A: DFT_L1 + twiddle + store, barrier,
// B: load + DFT_L2).  Thread id = r * LINES + li (lines fastest, so global
// accesses of a warp are contiguous across lines).
#pragma once
#include "phases.cuh"

// Scheduling fence: keeps the compiler from hoisting the table loads of the
// next loop above a register DFT (which would hold both in registers at once).
#if defined(__CUDA_ARCH__)
#define FC_FENCE() asm volatile("" ::: "memory")
#else
#define FC_FENCE()
#endif

namespace fcns {

// Prefetch the 128-byte line holding p into L2 (no-op on the host).
FC_HD void prefetch_l2(const void* p) {
#if defined(__CUDA_ARCH__)
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
  (void)p;
#endif
}

template <class T, int L1_, int L2_, int LINES_>
struct Eng {
  static constexpr int L1 = L1_, L2 = L2_, L = L1 * L2, LINES = LINES_;
  static constexpr int G = L1 > L2 ? L1 : L2;
  static constexpr int THREADS = G * LINES;
  static constexpr int PAD = (LINES * 2 * (int)sizeof(T) < 128) ? LINES : 0;
  static constexpr int ROW = L2 * LINES + PAD;
  static constexpr size_t BUF = (size_t)ROW * L1;  // elements of one exchange buffer
  using C = cx<T>;

  static FC_HD int bidx(int k1, int n2, int li) { return k1 * ROW + n2 * LINES + li; }

  // twiddle e^{SIGN 2 pi i n2 k1 / L}; tw holds the SIGN = -1 values twice:
  // [n2 * L1 + k1] for the k1 threads and [L + k1 * L2 + n2] for the n2 threads
  template <int SIGN>
  static FC_HD C twid(const C* tw, int n2, int k1) {
    C w = tw[n2 * L1 + k1];
    if (SIGN > 0) w.y = -w.y;
    return w;
  }
  template <int SIGN>
  static FC_HD C twidA(const C* tw, int n2, int k1) {
    C w = tw[L + k1 * L2 + n2];
    if (SIGN > 0) w.y = -w.y;
    return w;
  }

  // twiddle loads in groups of TG, one group ahead of their use: the first
  // group is issued before the register DFT (its latency overlaps the DFT),
  // each later one while the previous group is multiplied and stored
  static constexpr int TG = 6;
  // A: thread n2 with v[n1] = x[n2 + L2 n1]
  template <int SIGN>
  static FC_HD void A(C (&v)[L1], C* buf, const C* tw, int n2, int li) {
    C t[TG];
#pragma unroll
    for (int i = 0; i < TG; ++i) t[i] = i < L1 ? twidA<SIGN>(tw, n2, i) : mk<T>(0, 0);
    dft_reg<L1, SIGN, T>(v);
#pragma unroll
    for (int g = 0; g < L1; g += TG) {
      C tn[TG];
#pragma unroll
      for (int i = 0; i < TG; ++i) tn[i] = (g + TG + i < L1) ? twidA<SIGN>(tw, n2, g + TG + i) : mk<T>(0, 0);
      FC_FENCE();
#pragma unroll
      for (int i = 0; i < TG; ++i)
        if (g + i < L1) buf[bidx(g + i, n2, li)] = cmul(v[g + i], t[i]);
#pragma unroll
      for (int i = 0; i < TG; ++i) t[i] = tn[i];
    }
  }
  // B: thread k1 -> u[k2] = X[k1 + L1 k2]
  template <int SIGN>
  static FC_HD void B(C (&u)[L2], const C* buf, int k1, int li) {
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) u[n2] = buf[bidx(k1, n2, li)];
    dft_reg<L2, SIGN, T>(u);
  }
  // inverse-direction B: thread k1 holds u[k2] = X[k1 + L1 k2]; stores for Ai
  template <int SIGN>
  static FC_HD void Bi(C (&u)[L2], C* buf, const C* tw, int k1, int li) {
    C t[TG];
#pragma unroll
    for (int i = 0; i < TG; ++i) t[i] = i < L2 ? twid<SIGN>(tw, i, k1) : mk<T>(0, 0);
    dft_reg<L2, SIGN, T>(u);
#pragma unroll
    for (int g = 0; g < L2; g += TG) {
      C tn[TG];
#pragma unroll
      for (int i = 0; i < TG; ++i) tn[i] = (g + TG + i < L2) ? twid<SIGN>(tw, g + TG + i, k1) : mk<T>(0, 0);
      FC_FENCE();
#pragma unroll
      for (int i = 0; i < TG; ++i)
        if (g + i < L2) buf[bidx(k1, g + i, li)] = cmul(u[g + i], t[i]);
#pragma unroll
      for (int i = 0; i < TG; ++i) t[i] = tn[i];
    }
  }
  // u[k2] *= h(H[k1 + L1 k2]): the table loads in groups of TG, one group
  // ahead of their use (so that not all of them are live at once, and each
  // group's latency overlaps the previous group's products)
  template <class F>
  static FC_HD void mulH_by(C (&u)[L2], const C* H, int k1, F&& mul) {
    C t[TG];
#pragma unroll
    for (int i = 0; i < TG; ++i) t[i] = i < L2 ? H[k1 + L1 * i] : mk<T>(0, 0);
#pragma unroll
    for (int g = 0; g < L2; g += TG) {
      C tn[TG];
#pragma unroll
      for (int i = 0; i < TG; ++i) tn[i] = (g + TG + i < L2) ? H[k1 + L1 * (g + TG + i)] : mk<T>(0, 0);
      FC_FENCE();
#pragma unroll
      for (int i = 0; i < TG; ++i)
        if (g + i < L2) u[g + i] = mul(u[g + i], t[i]);
#pragma unroll
      for (int i = 0; i < TG; ++i) t[i] = tn[i];
    }
  }
  // u[k2] *= H[k1 + L1 k2]
  static FC_HD void mulH(C (&u)[L2], const C* H, int k1) {
    mulH_by(u, H, k1, [](C a, C h) { return cmul(a, h); });
  }
  // u[k2] *= i Im(H[k1 + L1 k2]) for a purely imaginary H (odd real kernel)
  static FC_HD void mulH_imag(C (&u)[L2], const C* H, int k1) {
    mulH_by(u, H, k1, [](C a, C h) { return mk<T>(-h.y * a.y, h.y * a.x); });
  }
  // u[k2] *= Re(H[k1 + L1 k2]) for a purely real H (even real kernel)
  static FC_HD void mulH_real(C (&u)[L2], const C* H, int k1) {
    mulH_by(u, H, k1, [](C a, C h) { return cscale(a, h.x); });
  }
  // inverse-direction A: thread n2 -> v[n1] = x[n2 + L2 n1]
  template <int SIGN>
  static FC_HD void Ai(C (&v)[L1], const C* buf, int n2, int li) {
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) v[k1] = buf[bidx(k1, n2, li)];
    dft_reg<L1, SIGN, T>(v);
  }
};

}  // namespace fcns
