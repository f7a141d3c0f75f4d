// Orchestration of the Navier-Stokes simulation object: workspace layout,
// tables, and the kernel sequences of set/get fields, right-hand side,
// projection and the Runge-Kutta step.  Templated on a backend that runs a
// kernel (on the GPU for libfcns, on the CPU for the host-check library) and
// moves memory, so that the same sequence is what the CPU tests check.
#pragma once
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/fcns.h"
#include "host_tables.hpp"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {

#ifndef FC_LAYOUT_GUARD
#define FC_LAYOUT_GUARD 0
#endif

struct NsLayout {
  int Nx, Ny, Nz, Np, Kx, Kxp, nf, L, L1, L2, Lx1, Lx2, Ly1, Ly2;
  bool zdirect;   // L = N' (plain length-N' z transforms)
  long long lines, ntiles, plines;   // lines, tiles of TL lines, padded lines
  size_t es;  // bytes per real
  // byte offsets inside the workspace
  size_t X[3], DZ, DZZ, V, DY, NL, gradp, diag, nfin, dser;
  size_t X64[3], d2r, hfr;   // float64 mean-line shadows and real-space z kernels
  int nmean;
  size_t kxo, kyo, kzo, kx, ky, fx, fy, Mr, Mr2, twz, twz2, H1, H2, Hf, chirp, Hbf, Hbi, twx, twy, twxh;
  int L1alt;      // first-pass factor of the alternative z schedule (0: none)
  size_t tkxo, tkyo, tkzo, tkx, tky, tfx, tfy;   // copies in the simulation's precision
  size_t total;
#if FC_LAYOUT_GUARD
  std::vector<std::pair<size_t, size_t>> guards;  // [begin, end) byte ranges between arrays
#endif
};

// z transform for continued length Np: Np itself when it is a compiled direct
// length, else the smallest padded length >= max(Np + Nz - 1, 2 Np - 1)
inline bool z_shape_for(int Np, int Nz, int* L, int* L1, int* L2, bool* direct) {
  int best = 0;
#define FC_ZDIRECT(LL, A, B, D) \
  if (D && !best && LL == Np) { best = LL; *L1 = A; *L2 = B; *direct = true; }
  FC_ZSHAPES(FC_ZDIRECT)
#undef FC_ZDIRECT
  const int need = std::max(Np + Nz - 1, 2 * Np - 1);
#define FC_ZPICK(LL, A, B, D) \
  if (!D && !best && LL >= need) { best = LL; *L1 = A; *L2 = B; *direct = false; }
  FC_ZSHAPES(FC_ZPICK)
#undef FC_ZPICK
  *L = best;
  return best > 0;
}

inline bool xy_shape_for(int N, int* L1, int* L2) {
  bool ok = false;
#define FC_XYPICK(NN, A, B) \
  if (!ok && NN == N) { ok = true; *L1 = A; *L2 = B; }
  FC_XYSHAPES(FC_XYPICK)
#undef FC_XYPICK
  return ok;
}

// slots of the device-side diagnostic series (ns_set_diag_series)
constexpr int NS_DIAG_SLOTS = 4096;

inline fc_status ns_layout(const ns_params& p, NsLayout* o) {
  if (p.Nx < 2 || p.Ny < 2 || p.Nz < 2 * p.d || p.d < 2 || p.d > DMAX || p.C < p.d || p.C > 64 ||
      (p.nfields != 3 && p.nfields != 4) || p.rk_order < 1 || p.rk_order > 4 || !(p.Lx > 0) || !(p.Ly > 0) ||
      !(p.Lz > 0) || p.nu < 0 || p.kappa < 0 || (p.filter != 0 && p.filter != 1) || (p.prec != FC_F32 && p.prec != FC_F64))
    return FC_ERR_ARG;
  NsLayout& l = *o;
  l.Nx = p.Nx; l.Ny = p.Ny; l.Nz = p.Nz; l.Np = p.Nz + p.C; l.Kx = p.Nx / 2 + 1; l.nf = p.nfields;
  l.Kxp = (l.Kx + TL - 1) / TL * TL;
  l.lines = (long long)p.Ny * l.Kxp;
  l.ntiles = (l.lines + TL - 1) / TL;
  l.plines = l.ntiles * TL;
  l.es = p.prec == FC_F32 ? 4 : 8;
  if (!z_shape_for(l.Np, p.Nz, &l.L, &l.L1, &l.L2, &l.zdirect)) return FC_ERR_UNSUPPORTED;
  // the float64 mean-line kernel keeps two continued lines in shared memory
  if (l.Np > KMean<float>::NPMAX) return FC_ERR_UNSUPPORTED;
  l.L1alt = 0;
#define FC_ZALT(LL, A, B) \
  if (!l.zdirect && LL == l.L && p.prec == FC_F32) l.L1alt = A;
  FC_ZSHAPES_ALT(FC_ZALT)
#undef FC_ZALT
  if (!xy_shape_for(p.Nx, &l.Lx1, &l.Lx2) || !xy_shape_for(p.Ny, &l.Ly1, &l.Ly2)) return FC_ERR_UNSUPPORTED;
  if (p.prec == FC_F64 && (l.L > 576 || p.Nx > 512)) return FC_ERR_UNSUPPORTED;
  const size_t cs = 2 * l.es;
  size_t off = 0;
  // arrays start on 256-byte boundaries; a checking build (FC_LAYOUT_GUARD
  // bytes > 0) leaves a guard band after every array and records it
  auto take = [&](size_t bytes) {
    size_t o2 = off;
    off += (bytes + 255) / 256 * 256 + FC_LAYOUT_GUARD;
#if FC_LAYOUT_GUARD
    l.guards.push_back({o2 + bytes, off});
#endif
    return o2;
  };
  for (int i = 0; i < 3; ++i) l.X[i] = take(cs * l.nf * l.Np * l.plines);
  l.DZ = take(cs * l.nf * l.Nz * l.plines);
  l.DZZ = take(cs * l.nf * l.Nz * l.plines);
  l.V = take(cs * l.nf * l.Nz * l.plines);
  l.DY = take(cs * l.nf * l.Nz * l.plines);
  l.NL = take(cs * l.nf * l.Nz * l.plines);
  l.gradp = take(sizeof(double) * 2 * 4 * l.lines);
  l.diag = take(sizeof(double) * 8);
  l.dser = take(sizeof(double) * 8 * NS_DIAG_SLOTS);
  l.nfin = take(sizeof(unsigned long long));
  l.nmean = l.nf == 4 ? 3 : 2;
  for (int i = 0; i < 3; ++i) l.X64[i] = take(16 * (size_t)l.nmean * l.Np);
  l.d2r = take(8 * (size_t)(l.Np + p.Nz - 1));
  l.hfr = take(8 * (size_t)(l.Np + p.Nz - 1));
  l.kxo = take(8 * l.Kx); l.kyo = take(8 * p.Ny); l.kzo = take(8 * l.Np);
  l.kx = take(8 * l.Kx); l.ky = take(8 * p.Ny); l.fx = take(8 * l.Kx); l.fy = take(8 * p.Ny);
  l.tkxo = take(l.es * l.Kx); l.tkyo = take(l.es * p.Ny); l.tkzo = take(l.es * l.Np);
  l.tkx = take(l.es * l.Kx); l.tky = take(l.es * p.Ny); l.tfx = take(l.es * l.Kx); l.tfy = take(l.es * p.Ny);
  l.Mr = take(8 * p.C * p.d); l.Mr2 = take(8 * p.C * p.d);
  l.twz = take(cs * 2 * l.L); l.twz2 = take(cs * 2 * l.L); l.H1 = take(cs * l.L); l.H2 = take(cs * l.L); l.Hf = take(cs * l.L);
  l.chirp = take(cs * l.Np); l.Hbf = take(cs * l.L); l.Hbi = take(cs * l.L);
  l.twx = take(cs * 2 * p.Nx); l.twy = take(cs * 2 * p.Ny);
  l.twxh = take(cs * (p.Nx + p.Nx / 2 + 1));
  l.total = off;
  // every array is indexed with 32-bit element offsets
  if ((double)l.nf * l.Np * l.plines >= 2147483647.0) return FC_ERR_UNSUPPORTED;
  return FC_OK;
}

template <class BK>
struct NsCore {
  BK bk;
  ns_params p{};
  NsLayout l{};
  unsigned char* ws = nullptr;
  bool own_ws = false;
  int cur = 0;  // index of the state buffer
  int sms = 1;  // multiprocessors of the device (prefetch distances in blocks)

  template <class X> X* at(size_t off) const { return reinterpret_cast<X*>(ws + off); }

  // ---------------------------------------------------------------- tables
  fc_status create(const ns_params& prm, void* dev_ws, size_t bytes) {
    p = prm;
    fc_status s = ns_layout(p, &l);
    if (s) return s;
    sms = bk.sms();
    if (dev_ws) {
      if (bytes < l.total) return FC_ERR_NOMEM;
      ws = static_cast<unsigned char*>(dev_ws);
    } else {
      s = bk.alloc((void**)&ws, l.total);
      if (s) return s;
      own_ws = true;
    }
    FcTables T;
    if (!build_fc_tables(p.d, p.C, (2 * (p.d + p.C)) / 3, 20, &T)) return FC_ERR_ARG;
    const double dz = p.Lz / (p.Nz - 1);
    const double twopi = 6.283185307179586476925286766559;
    std::vector<double> kxo(l.Kx), kx(l.Kx), kyo(p.Ny), ky(p.Ny), kzo(l.Np), fx(l.Kx), fy(p.Ny);
    for (int i = 0; i < l.Kx; ++i) {
      kx[i] = twopi * i / p.Lx;
      kxo[i] = (p.Nx % 2 == 0 && i == p.Nx / 2) ? 0.0 : kx[i];
      fx[i] = p.filter == 1 ? (3 * i <= p.Nx ? 1.0 : 0.0)
                            : std::exp(-p.filter_beta * std::pow(i / (p.Nx / 2.0), p.filter_2p));
    }
    for (int i = 0; i < p.Ny; ++i) {
      const int is = (i <= (p.Ny - 1) / 2) ? i : i - p.Ny;
      ky[i] = twopi * is / p.Ly;
      kyo[i] = (p.Ny % 2 == 0 && i == p.Ny / 2) ? 0.0 : ky[i];
      fy[i] = p.filter == 1 ? (3 * std::abs(is) <= p.Ny ? 1.0 : 0.0)
                            : std::exp(-p.filter_beta * std::pow(std::abs(is) / (p.Ny / 2.0), p.filter_2p));
    }
    for (int i = 0; i < l.Np; ++i) {
      const int is = (i <= (l.Np - 1) / 2) ? i : i - l.Np;
      kzo[i] = (l.Np % 2 == 0 && i == l.Np / 2) ? 0.0 : twopi * is / (l.Np * dz);
    }
    std::vector<std::complex<double>> twz, twz2, H1, H2, Hf, chirp, Hbf, Hbi, twx, twy, twxh;
    engine_twiddles(l.L1, l.L2, &twz);
    if (l.L1alt) engine_twiddles(l.L1alt, l.L / l.L1alt, &twz2);
    else twz2 = twz;
    deriv_conv_spectra(p.Nz, l.Np, l.L, &H1, &H2);
    filter_conv_spectrum(p.Nz, l.Np, l.L, p.filter_beta, p.filter_2p, &Hf);
    if (l.zdirect) {  // no Bluestein DFTs
      chirp.assign(l.Np, 0);
      Hbf.assign(l.L, 0);
      Hbi.assign(l.L, 0);
    } else {
      bluestein_tables(l.Np, l.L, &chirp, &Hbf, &Hbi);
    }
    std::vector<double> d2r, hfr;
    z_kernels_real(p.Nz, l.Np, p.filter_beta, p.filter_2p, &d2r, &hfr);
    engine_twiddles(l.Lx1, l.Lx2, &twx);
    {  // the x pass's forward half: length-Nx/2 engine, then the even / odd split factors
      std::vector<std::complex<double>> sp;
      engine_twiddles(half_l1(l.Lx1, l.Lx2), half_l2(l.Lx1, l.Lx2), &twxh);
      split_twiddles(p.Nx, &sp);
      twxh.insert(twxh.end(), sp.begin(), sp.end());
    }
    engine_twiddles(l.Ly1, l.Ly2, &twy);
    std::vector<float2> mr2(T.Mr.size());
    for (size_t i = 0; i < mr2.size(); ++i) {
      mr2[i].x = (float)T.Mr[i];
      mr2[i].y = (float)(T.Mr[i] - (double)mr2[i].x);
    }
    s = put(l.kxo, kxo.data(), 8 * kxo.size());
    if (!s) s = put(l.kyo, kyo.data(), 8 * kyo.size());
    if (!s) s = put(l.kzo, kzo.data(), 8 * kzo.size());
    if (!s) s = put(l.kx, kx.data(), 8 * kx.size());
    if (!s) s = put(l.ky, ky.data(), 8 * ky.size());
    if (!s) s = put(l.fx, fx.data(), 8 * fx.size());
    if (!s) s = put(l.fy, fy.data(), 8 * fy.size());
    if (!s) s = putr(l.tkxo, kxo);
    if (!s) s = putr(l.tkyo, kyo);
    if (!s) s = putr(l.tkzo, kzo);
    if (!s) s = putr(l.tkx, kx);
    if (!s) s = putr(l.tky, ky);
    if (!s) s = putr(l.tfx, fx);
    if (!s) s = putr(l.tfy, fy);
    if (!s) s = put(l.Mr, T.Mr.data(), 8 * T.Mr.size());
    if (!s) s = put(l.Mr2, mr2.data(), 8 * mr2.size());
    if (!s) s = putc(l.twz, twz);
    if (!s) s = putc(l.twz2, twz2);
    if (!s) s = putc(l.H1, H1);
    if (!s) s = putc(l.H2, H2);
    if (!s) s = putc(l.Hf, Hf);
    if (!s) s = putc(l.chirp, chirp);
    if (!s) s = putc(l.Hbf, Hbf);
    if (!s) s = putc(l.Hbi, Hbi);
    if (!s) s = putc(l.twx, twx);
    if (!s) s = putc(l.twxh, twxh);
    if (!s) s = putc(l.twy, twy);
    if (!s) s = put(l.d2r, d2r.data(), 8 * d2r.size());
    if (!s) s = put(l.hfr, hfr.data(), 8 * hfr.size());
    if (!s) s = bk.memset(ws + l.X64[0], 0, 3 * 16 * (size_t)l.nmean * l.Np, nullptr);
    if (!s) s = bk.memset(ws + l.gradp, 0, sizeof(double) * 8 * l.lines, nullptr);
    if (!s) s = bk.memset(ws + l.nfin, 0, sizeof(unsigned long long), nullptr);
    if (!s) s = bk.memset(ws + l.X[0], 0, l.NL - l.X[0] + 2 * l.es * l.nf * l.Nz * l.plines, nullptr);
    if (!s) s = bk.sync(nullptr);
    return s;
  }

  fc_status destroy() {
    fc_status s = bk.sync(nullptr);
    if (own_ws && ws) bk.free(ws);
    ws = nullptr;
    return s;
  }

  fc_status put(size_t off, const void* src, size_t bytes) { return bk.h2d(ws + off, src, bytes); }
  fc_status putr(size_t off, const std::vector<double>& v) {
    if (l.es == 8) return put(off, v.data(), 8 * v.size());
    std::vector<float> f(v.begin(), v.end());
    return put(off, f.data(), 4 * f.size());
  }
  fc_status putc(size_t off, const std::vector<std::complex<double>>& v) {
    if (l.es == 8) return put(off, v.data(), 16 * v.size());
    std::vector<float2> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) { f[i].x = (float)v[i].real(); f[i].y = (float)v[i].imag(); }
    return put(off, f.data(), 8 * f.size());
  }

  template <class T>
  ZTab<T> ztab() const {
    ZTab<T> t;
    t.Mr = at<double>(l.Mr); t.Mr2 = at<float2>(l.Mr2);
    t.tw = at<cx<T>>(l.twz); t.H1 = at<cx<T>>(l.H1); t.H2 = at<cx<T>>(l.H2); t.Hf = at<cx<T>>(l.Hf);
    t.chirp = at<cx<T>>(l.chirp); t.Hbf = at<cx<T>>(l.Hbf); t.Hbi = at<cx<T>>(l.Hbi);
    t.kxo = at<T>(l.tkxo); t.kyo = at<T>(l.tkyo); t.kzo = at<T>(l.tkzo);
    t.kx = at<T>(l.tkx); t.ky = at<T>(l.tky); t.fx = at<T>(l.tfx); t.fy = at<T>(l.tfy);
    t.kxo_d = at<double>(l.kxo); t.kyo_d = at<double>(l.kyo);
    return t;
  }
  ZGeom zgeom(int nf) const {
    ZGeom g;
    g.Nz = p.Nz; g.Np = l.Np; g.d = p.d; g.Cc = p.C; g.Kx = l.Kx; g.Kxp = l.Kxp; g.Ny = p.Ny; g.nf = nf;
    g.lines = l.lines; g.ntiles = l.ntiles; g.Lz = p.Lz; g.dz = p.Lz / (p.Nz - 1);
    return g;
  }

  // ------------------------------------------------------------ launchers
  // Variant per kernel kind, see ns_tune: bit 0 = lines per CTA (0: the
  // built-in default of shapes.hpp, 1: its alternative tile_alt); bit 1 (z
  // kinds, float32 padded lengths of FC_ZSHAPES_ALT) = the alternative radix
  // schedule L1 <-> L2.  Every combination is compiled.
  enum { TK_ZD, TK_ZC, TK_ZP, TK_YI, TK_Y1, TK_N };
  int tile[TK_N] = {0, 0, 0, 0, 0};
  // the variant bits that exist for kind k on this simulation
  int variant_mask(int k) const { return (k <= TK_ZP && l.L1alt) ? 3 : 1; }
  // engine twiddles of the schedule whose first pass has length A
  template <class T>
  const cx<T>* ztw(int A) const { return at<cx<T>>(A == l.L1 ? l.twz : l.twz2); }

  template <class T, int A, int B, int LN, int JN>
  fc_status z_deriv_run(const cx<T>* X, int nf, void* st) {
    using K = KZDeriv<T, A, B, LN, JN>;
    typename K::Args a;
    a.g = zgeom(nf); a.t = ztab<T>(); a.t.tw = ztw<T>(A); a.X = X;
    a.DZ = at<cx<T>>(l.DZ); a.DZZ = at<cx<T>>(l.DZZ);
    a.tiles = (l.lines + LN - 1) / LN;
    const double dz = p.Lz / (p.Nz - 1);
    a.s1 = (T)(1.0 / dz); a.s2 = (T)(1.0 / (dz * dz));
    a.nblocks = a.tiles * nf; a.pf = (long long)sms * K::MINB;
    return bk.template run<K>(a, a.tiles * nf, st);
  }
  template <class T>
  fc_status z_deriv(const cx<T>* X, int nf, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
    if (tile[TK_ZD] & 2) {
      if constexpr (sizeof(T) == 4) {
#define FC_ZDA(LL, A, B)                                                                     \
  if (l.L == LL) {                                                                           \
    constexpr int LN = zderiv_lines<T, LL>();                                                \
    return (tile[TK_ZD] & 1) ? z_deriv_run<T, A, B, tile_alt<LN>(), A / 2>(X, nf, st)        \
                             : z_deriv_run<T, A, B, LN, A / 2>(X, nf, st);                   \
  }
        FC_ZSHAPES_ALT(FC_ZDA)
#undef FC_ZDA
      }
      return s;
    }
#define FC_ZD(LL, A, B, D)                                                                   \
  if (l.L == LL) {                                                                           \
    constexpr int LN = zderiv_lines<T, LL>();                                                \
    s = (tile[TK_ZD] & 1) ? z_deriv_run<T, A, B, tile_alt<LN>(), D ? A : A / 2>(X, nf, st) \
                    : z_deriv_run<T, A, B, LN, D ? A : A / 2>(X, nf, st);                    \
  }
    FC_ZSHAPES(FC_ZD)
#undef FC_ZD
    return s;
  }

  template <class T, int A, int B, int LN, int JN>
  fc_status z_combine_run(const cx<T>* NL, const cx<T>* Xt, const cx<T>* Xj, cx<T>* Xo, double dtj, int inject,
                          int nf, void* st) {
    using K = KZCombine<T, A, B, LN, JN>;
    typename K::Args a;
    a.g = zgeom(nf); a.t = ztab<T>(); a.t.tw = ztw<T>(A); a.NL = NL; a.Xt = Xt; a.Xj = Xj;
    a.DZZ = at<cx<T>>(l.DZZ); a.Xout = Xo; a.gradp = at<double2>(l.gradp);
    a.dtj = dtj; a.dif[0] = a.dif[1] = a.dif[2] = p.nu; a.dif[3] = p.kappa;
    a.inject = inject;
    a.tiles = (l.lines + LN - 1) / LN;
    a.nblocks = a.tiles * nf; a.pf = (long long)sms * K::MINB;
    return bk.template run<K>(a, a.tiles * nf, st);
  }
  template <class T>
  fc_status z_combine(const cx<T>* NL, const cx<T>* Xt, const cx<T>* Xj, cx<T>* Xo, double dtj, int inject,
                      int nf, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
    if (tile[TK_ZC] & 2) {
      if constexpr (sizeof(T) == 4) {
#define FC_ZCA(LL, A, B)                                                                                      \
  if (l.L == LL) {                                                                                            \
    constexpr int LN = z_lines<T, LL>();                                                                      \
    return (tile[TK_ZC] & 1) ? z_combine_run<T, A, B, tile_alt<LN>(), A / 2>(NL, Xt, Xj, Xo, dtj, inject, nf, st) \
                             : z_combine_run<T, A, B, LN, A / 2>(NL, Xt, Xj, Xo, dtj, inject, nf, st);    \
  }
        FC_ZSHAPES_ALT(FC_ZCA)
#undef FC_ZCA
      }
      return s;
    }
#define FC_ZC(LL, A, B, D)                                                                             \
  if (l.L == LL) {                                                                                     \
    constexpr int LN = z_lines<T, LL>();                                                               \
    s = (tile[TK_ZC] & 1) ? z_combine_run<T, A, B, tile_alt<LN>(), D ? A : A / 2>(NL, Xt, Xj, Xo, dtj, inject, nf, st) \
                    : z_combine_run<T, A, B, LN, D ? A : A / 2>(NL, Xt, Xj, Xo, dtj, inject, nf, st);  \
  }
    FC_ZSHAPES(FC_ZC)
#undef FC_ZC
    return s;
  }

  template <class T>
  fc_status z_continue(const cx<T>* M, cx<T>* X, int nf, const double2* gradp, double dtj, void* st) {
    using K = KZContinue<T, 8>;
    typename K::Args a;
    a.g = zgeom(nf); a.t = ztab<T>(); a.M = M; a.X = X; a.gradp = gradp; a.dtj = dtj;
    a.tiles = (l.lines + 7) / 8;
    return bk.template run<K>(a, a.tiles * nf, st);
  }

  template <class T, int A, int B, int LN, bool D>
  fc_status z_project_run(cx<T>* X, double dtj, void* st) {
    using K = KZProject<T, A, B, LN, D>;
    typename K::Args a;
    a.g = zgeom(3); a.t = ztab<T>(); a.t.tw = ztw<T>(A); a.X = X; a.gradp = at<double2>(l.gradp);
    a.G0 = at<cx<T>>(l.DZ); a.G1 = at<cx<T>>(l.DZZ); a.dtj = dtj;
    a.tiles = (l.lines + LN - 1) / LN;
    return bk.template run<K>(a, a.tiles, st);
  }
  template <class T>
  fc_status z_project(cx<T>* X, double dtj, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
    if (tile[TK_ZP] & 2) {
      if constexpr (sizeof(T) == 4) {
#define FC_ZPA(LL, A, B)                                                                 \
  if (l.L == LL) {                                                                       \
    constexpr int LN = zproj_lines<T, LL>();                                             \
    return (tile[TK_ZP] & 1) ? z_project_run<T, A, B, tile_alt<LN>(), false>(X, dtj, st) \
                             : z_project_run<T, A, B, LN, false>(X, dtj, st);            \
  }
        FC_ZSHAPES_ALT(FC_ZPA)
#undef FC_ZPA
      }
      return s;
    }
#define FC_ZP(LL, A, B, D)                                                               \
  if (l.L == LL) {                                                                       \
    constexpr int LN = zproj_lines<T, LL>();                                             \
    s = (tile[TK_ZP] & 1) ? z_project_run<T, A, B, tile_alt<LN>(), D>(X, dtj, st)        \
                    : z_project_run<T, A, B, LN, D>(X, dtj, st);                         \
  }
    FC_ZSHAPES(FC_ZP)
#undef FC_ZP
    return s;
  }

  YGeom ygeom() const {
    YGeom g;
    g.Ny = p.Ny; g.Kx = l.Kx; g.Kxp = l.Kxp; g.Nz = p.Nz; g.plane = l.lines; g.ntiles = l.ntiles;
    return g;
  }

  template <class T, int A1, int B1, int LN, bool ONEBUF = false>
  fc_status y_inv3_run(const cx<T>* A, long long a_fstride, int nf, void* st) {
    using K = std::conditional_t<ONEBUF, KYInv3S<T, A1, B1, LN>, KYInv3<T, A1, B1, LN>>;
    typename K::Args a;
    a.g = ygeom(); a.tw = at<cx<T>>(l.twy); a.kyo = at<T>(l.tkyo);
    a.A = A; a.a_fstride = a_fstride;
    a.V = at<cx<T>>(l.V); a.DY = at<cx<T>>(l.DY); a.DZ = at<cx<T>>(l.DZ);
    a.tiles = (l.Kx + LN - 1) / LN;
    a.scale = (T)(1.0 / p.Ny);
    return bk.template run<K>(a, a.tiles * nf * p.Nz, st);
  }
  template <class T>
  fc_status y_inv3(const cx<T>* A, long long a_fstride, int nf, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
#define FC_YI(NN, A1, B1)                                                           \
  if (p.Ny == NN) {                                                                \
    constexpr int LN = y_lines<T, NN>();                                           \
    s = tile[TK_YI] ? y_inv3_run<T, A1, B1, y_lines_alt<T, NN>(), y_wide<T, NN>()>(A, a_fstride, nf, st) \
                    : y_inv3_run<T, A1, B1, LN>(A, a_fstride, nf, st);             \
  }
    FC_XYSHAPES(FC_YI)
#undef FC_YI
    return s;
  }

  template <class T, int SIGN, int A1, int B1, int LN>
  fc_status y_one_run(const cx<T>* IN, long long in_fs, cx<T>* OUT, long long out_fs, int nf, double scale, void* st) {
    using K = KY1<T, A1, B1, LN, SIGN>;
    typename K::Args a;
    a.g = ygeom(); a.tw = at<cx<T>>(l.twy);
    a.IN = IN; a.in_fstride = in_fs; a.OUT = OUT; a.out_fstride = out_fs;
    a.tiles = (l.Kx + LN - 1) / LN;
    a.scale = (T)scale;
    return bk.template run<K>(a, a.tiles * nf * p.Nz, st);
  }
  template <class T, int SIGN>
  fc_status y_one(const cx<T>* IN, long long in_fs, cx<T>* OUT, long long out_fs, int nf, double scale, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
#define FC_Y1(NN, A1, B1)                                                                              \
  if (p.Ny == NN) {                                                                                   \
    constexpr int LN = y_lines<T, NN>();                                                              \
    s = tile[TK_Y1] ? y_one_run<T, SIGN, A1, B1, y_lines_alt<T, NN>()>(IN, in_fs, OUT, out_fs, nf, scale, st) \
                    : y_one_run<T, SIGN, A1, B1, LN>(IN, in_fs, OUT, out_fs, nf, scale, st);          \
  }
    FC_XYSHAPES(FC_Y1)
#undef FC_Y1
    return s;
  }

  template <class T>
  fc_status x_pass(void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
    const long long rows = (long long)p.Nz * p.Ny;
#define FC_XP(NN, A1, B1)                                                      \
  if (p.Nx == NN) {                                                           \
    if (l.nf == 3) {                                                          \
      using K = KXPass<T, A1, B1, 3>;                                         \
      s = x_pass_run<T, K>(rows, st);                                         \
    } else {                                                                  \
      using K = KXPass<T, A1, B1, 4>;                                         \
      s = x_pass_run<T, K>(rows, st);                                         \
    }                                                                         \
  }
    FC_XYSHAPES(FC_XP)
#undef FC_XP
    return s;
  }
  template <class T, class K>
  fc_status x_pass_run(long long rows, void* st) {
    if (K::smem_bytes > 227 * 1024) return FC_ERR_UNSUPPORTED;
    typename K::Args a;
    a.Kx = l.Kx; a.Kxp = l.Kxp; a.Ny = p.Ny; a.Nz = p.Nz; a.rows = rows; a.ntiles = l.ntiles;
    a.tw = at<cx<T>>(l.twx); a.twh = at<cx<T>>(l.twxh); a.kxo = at<T>(l.tkxo);
    a.V = at<cx<T>>(l.V); a.DY = at<cx<T>>(l.DY); a.DZ = at<cx<T>>(l.DZ); a.NL = at<cx<T>>(l.NL);
    a.forcing = (T)p.forcing_x; a.gamma = (T)p.gamma; a.scale = (T)(1.0 / p.Nx);
    return bk.template run<K>(a, rows, st);
  }

  template <class T, int SIGN>
  fc_status x_rows(T* R, cx<T>* S, int nf, void* st) {
    fc_status s = FC_ERR_UNSUPPORTED;
    const long long pairs = (long long)nf * p.Nz * p.Ny / 2;
#define FC_XR(NN, A1, B1)                                                      \
  if (p.Nx == NN) {                                                           \
    using K = KXRow<T, A1, B1, SIGN, x_jobs<NN>()>;                           \
    typename K::Args a;                                                       \
    a.Kx = l.Kx; a.Kxp = l.Kxp; a.Ny = p.Ny; a.Nz = p.Nz; a.ntiles = l.ntiles; \
    a.pairs = pairs; a.tw = at<cx<T>>(l.twx); a.R = R; a.S = S;               \
    a.scale = (T)(SIGN > 0 ? 1.0 / p.Nx : 1.0);                               \
    s = bk.template run<K>(a, (pairs + x_jobs<NN>() - 1) / x_jobs<NN>(), st); \
  }
    FC_XYSHAPES(FC_XR)
#undef FC_XR
    return s;
  }

  // ------------------------------------------------------------- sequences
  template <class T> cx<T>* Xb(int i) const { return at<cx<T>>(l.X[i]); }
  template <class T> cx<T>* buf(size_t off) const { return at<cx<T>>(off); }

  // physical [nf][Nz][Ny][Nx] -> extended state X (optionally with injection)
  template <class T>
  fc_status phys_to_state(const T* phys, cx<T>* X, int nf, const double2* gradp, double dtj, void* st) {
    cx<T>* V = buf<T>(l.V);
    fc_status s = x_rows<T, -1>(const_cast<T*>(phys), V, nf, st);
    if (!s) s = y_one<T, -1>(V, p.Nz, V, p.Nz, nf, 1.0, st);
    if (!s) s = z_continue<T>(V, X, nf, gradp, dtj, st);
    return s;
  }
  // extended state X -> physical (first Nz points)
  template <class T>
  fc_status state_to_phys(const cx<T>* X, T* phys, int nf, void* st) {
    cx<T>* V = buf<T>(l.V);
    fc_status s = y_one<T, 1>(X, l.Np, V, p.Nz, nf, 1.0 / p.Ny, st);
    if (!s) s = x_rows<T, 1>(phys, V, nf, st);
    return s;
  }

  // nonlinear term of the state Xj into NL (mixed, filtered later); DZZ filled
  template <class T>
  fc_status nonlinear(const cx<T>* Xj, void* st) {
    fc_status s = z_deriv<T>(Xj, l.nf, st);
    if (!s) s = y_inv3<T>(Xj, l.Np, l.nf, st);
    if (!s) s = x_pass<T>(st);
    if (!s) s = y_one<T, -1>(buf<T>(l.NL), p.Nz, buf<T>(l.NL), p.Nz, l.nf, 1.0, st);
    return s;
  }

  // float64 mean-line island (float32 path only)
  template <class T>
  void mean_fmap(int* fm) const { fm[0] = 0; fm[1] = 1; fm[2] = 3; }
  template <class T>
  fc_status mean_init(int ix, void* st) {
    if (sizeof(T) != 4) return FC_OK;
    using K = KMeanInit<T>;
    typename K::Args a;
    a.g = zgeom(l.nf); a.X = Xb<T>(ix); a.X64 = at<double2>(l.X64[ix]);
    mean_fmap<T>(a.fmap);
    return bk.template run<K>(a, l.nmean, st);
  }
  template <class T>
  fc_status mean_stage(int it, int ij, int in, double dtj, void* st) {
    if (sizeof(T) != 4) return FC_OK;
    using K = KMeanLine<T>;
    typename K::Args a;
    a.g = zgeom(l.nf); a.Mr = at<double>(l.Mr); a.d2 = at<double>(l.d2r); a.hf = at<double>(l.hfr);
    a.NL = buf<T>(l.NL); a.Xt = at<double2>(l.X64[it]); a.Xj = at<double2>(l.X64[ij]);
    a.Xn = at<double2>(l.X64[in]); a.Xo = Xb<T>(in); a.gradp = at<double2>(l.gradp);
    a.dtj = dtj; a.dif[0] = a.dif[1] = p.nu; a.dif[2] = p.kappa;
    a.fxy00 = 1.0;   // x, y filter / mask factor of the (0, 0) mode in both filter modes
    mean_fmap<T>(a.fmap);
    a.nmean = l.nmean;
    return bk.template run<K>(a, l.nmean, st);
  }
  fc_status mean_init_any(void* st) { return f32() ? mean_init<float>(cur, st) : FC_OK; }

  template <class T>
  fc_status set_fields(const T* phys, void* st) {
    fc_status s = phys_to_state<T>(phys, Xb<T>(cur), l.nf, nullptr, 0.0, st);
    if (!s) s = bk.memset(ws + l.gradp, 0, sizeof(double) * 8 * l.lines, st);
    if (!s) s = mean_init<T>(cur, st);
    return s;
  }
  template <class T>
  fc_status get_fields(T* phys, void* st) { return state_to_phys<T>(Xb<T>(cur), phys, l.nf, st); }

  // state := spectral interpolation of src's state onto this grid (Sec. 6
  // restarts; see KInterp), re-continued here; wall planes reset to zero.
  // The evaluation weights go to this simulation's DZZ work buffer.
  template <class T>
  fc_status interpolate_from(const NsCore& src, void* st) {
    const NsLayout& l1 = src.l;
    const size_t need = sizeof(cx<T>) * (size_t)p.Nz * l1.Np;
    if (need > 2 * l.es * l.nf * (size_t)p.Nz * l.plines) return FC_ERR_UNSUPPORTED;
    std::vector<cx<T>> W((size_t)p.Nz * l1.Np);
    const int Np1 = l1.Np;
    const double dz1 = src.p.Lz / (src.p.Nz - 1), L1 = Np1 * dz1, dz2 = p.Lz / (p.Nz - 1);
    // W[s][n] = (1/N'1) sum_l A_l(z_s) e^{-2 pi i l n / N'1}, A_l = e^{i k_l z}
    // (k_l = 2 pi l / L'1, signed l) and a cosine for the Nyquist term
    std::vector<std::complex<double>> Bt((size_t)Np1 * Np1), A(Np1);
    for (int ll = 0; ll < Np1; ++ll)
      for (int n = 0; n < Np1; ++n) {
        double c, sn;
        sincos2pi(-(long long)ll * n, Np1, &c, &sn);
        Bt[(size_t)ll * Np1 + n] = std::complex<double>(c, sn);
      }
    for (int s2 = 0; s2 < p.Nz; ++s2) {
      const double z = s2 * dz2;
      for (int ll = 0; ll < Np1; ++ll) {
        const int ls = (ll <= (Np1 - 1) / 2) ? ll : ll - Np1;
        if (Np1 % 2 == 0 && ll == Np1 / 2) A[ll] = std::cos(M_PI * Np1 * z / L1);
        else A[ll] = std::polar(1.0, 2 * M_PI * ls * z / L1);
      }
      for (int n = 0; n < Np1; ++n) {
        std::complex<double> acc = 0;
        for (int ll = 0; ll < Np1; ++ll) acc += A[ll] * Bt[(size_t)ll * Np1 + n];
        acc /= (double)Np1;
        W[(size_t)s2 * Np1 + n] = mk<T>((T)acc.real(), (T)acc.imag());
      }
    }
    fc_status s = bk.h2d(ws + l.DZZ, W.data(), sizeof(cx<T>) * W.size());
    if (s) return s;
    using K = KInterp<T>;
    typename K::Args a;
    a.X1 = reinterpret_cast<const cx<T>*>(src.ws + l1.X[src.cur]);
    a.Np1 = l1.Np; a.Kx1 = l1.Kx; a.Kxp1 = l1.Kxp; a.Ny1 = src.p.Ny; a.Nx1 = src.p.Nx; a.ntiles1 = l1.ntiles;
    a.M2 = buf<T>(l.V); a.Nz2 = p.Nz; a.Kx2 = l.Kx; a.Kxp2 = l.Kxp; a.Ny2 = p.Ny; a.Nx2 = p.Nx; a.ntiles2 = l.ntiles;
    a.W = buf<T>(l.DZZ);
    a.scale = (T)((double)p.Nx * p.Ny / ((double)src.p.Nx * src.p.Ny));
    a.sblocks = (p.Nz + 15) / 16;
    s = bk.template run<K>(a, (long long)a.sblocks * l.ntiles * l.nf, st);
    if (!s) s = z_continue<T>(buf<T>(l.V), Xb<T>(cur), l.nf, nullptr, 0.0, st);
    if (!s) s = bk.memset(ws + l.gradp, 0, sizeof(double) * 8 * l.lines, st);
    if (!s) s = mean_init<T>(cur, st);
    return s;
  }
  // horizontal statistics of the current state per field and physical level
  // (KProf); out: host [nf][Nz][2 + nshell] (unnormalised sums, see KProf)
  int nshell() const {
    const double kxm = M_PI * p.Nx / p.Lx, kym = M_PI * p.Ny / p.Ly;
    return (int)std::floor(std::sqrt(kxm * kxm + kym * kym) / shell_width() + 0.5) + 1;
  }
  double shell_width() const { return std::min(2 * M_PI / p.Lx, 2 * M_PI / p.Ly); }
  template <class T>
  fc_status profiles(double* out, void* st) {
    using K = KProf<T>;
    typename K::Args a;
    a.g = zgeom(l.nf); a.Nx = p.Nx; a.X = Xb<T>(cur);
    a.kx_unit = 2 * M_PI / p.Lx; a.ky_unit = 2 * M_PI / p.Ly; a.dk = shell_width();
    a.nshell = nshell();
    if (a.nshell > K::NSMAX) return FC_ERR_UNSUPPORTED;
    const size_t bytes = sizeof(double) * (size_t)l.nf * p.Nz * (2 + a.nshell);
    if (bytes > 2 * l.es * (size_t)l.nf * p.Nz * l.plines) return FC_ERR_UNSUPPORTED;
    a.out = reinterpret_cast<double*>(ws + l.NL);
    fc_status s = bk.memset(ws + l.NL, 0, bytes, st);
    if (!s) s = bk.template run<K>(a, (long long)l.nf * p.Nz, st);
    if (!s) s = bk.d2h(out, ws + l.NL, bytes, st);
    return s;
  }
  fc_status profiles_any(double* out, void* st) { return f32() ? profiles<float>(out, st) : profiles<double>(out, st); }

  // non-finite values of the current state, added to the device counter at
  // l.nfin (asynchronous; reset = true zeroes the counter first)
  template <class T>
  fc_status count_nonfinite(bool reset, void* st) {
    fc_status s = reset ? bk.memset(ws + l.nfin, 0, sizeof(unsigned long long), st) : FC_OK;
    if (!s) {
      using K = KFinite<T>;
      typename K::Args a;
      a.g = zgeom(l.nf); a.X = Xb<T>(cur); a.count = at<unsigned long long>(l.nfin);
      s = bk.template run<K>(a, l.ntiles, st);
    }
    return s;
  }
  fc_status count_nonfinite_any(bool reset, void* st) {
    return f32() ? count_nonfinite<float>(reset, st) : count_nonfinite<double>(reset, st);
  }

  // Autotuner of the kernel variants: each kernel kind of the RK step is
  // timed with every compiled variant (lines per CTA; for the z kinds of
  // float32 padded lengths also the second radix schedule) on this
  // simulation's buffers (two timed launches each after a warm-up) and the
  // fastest kept.  The state and the
  // wall planes are preserved (the projection runs on a spare buffer; the
  // planes it writes are restored).  Results are cached per process by size,
  // so instances of equal sizes are tuned once.
  template <class T>
  fc_status autotune(void* st) {
    static std::mutex mu;
    static std::map<std::vector<long long>, std::array<int, TK_N>> cache;
    const std::vector<long long> key = {(long long)p.prec, p.Nx, p.Ny, p.Nz, p.C, l.nf, l.L};
    {
      std::lock_guard<std::mutex> g(mu);
      auto it = cache.find(key);
      if (it != cache.end()) {
        for (int k = 0; k < TK_N; ++k) tile[k] = it->second[k];
        return FC_OK;
      }
    }
    std::vector<double> gp(8 * (size_t)l.lines);
    fc_status s = bk.d2h(gp.data(), ws + l.gradp, sizeof(double) * gp.size(), st);
    cx<T>* Xs = Xb<T>((cur + 1) % 3);
    cx<T>* Xo = Xb<T>((cur + 2) % 3);
    auto launch = [&](int k) -> fc_status {
      switch (k) {
        case TK_ZD: return z_deriv<T>(Xb<T>(cur), l.nf, st);
        case TK_ZC: return z_combine<T>(buf<T>(l.NL), Xb<T>(cur), Xb<T>(cur), Xo, 0.0, 0, l.nf, st);
        case TK_ZP: return z_project<T>(Xs, 1.0, st);
        case TK_YI: return y_inv3<T>(Xb<T>(cur), l.Np, l.nf, st);
        default: return y_one<T, -1>(buf<T>(l.NL), p.Nz, buf<T>(l.NL), p.Nz, l.nf, 1.0, st);
      }
    };
    std::array<int, TK_N> pick{};
    for (int k = 0; k < TK_N && !s; ++k) {
      float best[4] = {3e38f, 3e38f, 3e38f, 3e38f};
      const int nv = variant_mask(k) + 1;
      for (int c = 0; c < nv && !s; ++c) {
        tile[k] = c;
        fc_status w = launch(k);  // warm-up
        if (w == FC_ERR_UNSUPPORTED) continue;  // this tile does not fit the shared memory
        s = w;
        for (int r = 0; r < 2 && !s; ++r) {
          float ms = 0;
          s = bk.time_ms([&] { return launch(k); }, st, &ms);
          if (!s && ms < best[c]) best[c] = ms;
        }
      }
      pick[k] = 0;
      for (int c = 1; c < nv; ++c)
        if (best[c] < best[pick[k]]) pick[k] = c;
      tile[k] = pick[k];
    }
    if (!s) s = bk.h2d(ws + l.gradp, gp.data(), sizeof(double) * gp.size());
    if (s) {
      for (int k = 0; k < TK_N; ++k) tile[k] = 0;
      return s;
    }
    std::lock_guard<std::mutex> g(mu);
    cache[key] = pick;
    return FC_OK;
  }
  fc_status autotune_any(void* st) { return f32() ? autotune<float>(st) : autotune<double>(st); }

  fc_status interpolate_from_any(const NsCore& src, void* st) {
    if (src.p.prec != p.prec || src.p.nfields != p.nfields || p.Nx < src.p.Nx || p.Ny < src.p.Ny ||
        src.p.Lx != p.Lx || src.p.Ly != p.Ly || src.p.Lz != p.Lz)
      return FC_ERR_ARG;
    return f32() ? interpolate_from<float>(src, st) : interpolate_from<double>(src, st);
  }

  template <class T>
  fc_status rhs(const T* in, T* out, void* st) {
    cx<T>* Xs = Xb<T>((cur + 1) % 3);
    cx<T>* Xo = Xb<T>((cur + 2) % 3);
    fc_status s = phys_to_state<T>(in, Xs, l.nf, nullptr, 0.0, st);
    if (!s) s = nonlinear<T>(Xs, st);
    if (!s) s = z_combine<T>(buf<T>(l.NL), nullptr, Xs, Xo, 1.0, 0, l.nf, st);
    if (!s) s = state_to_phys<T>(Xo, out, l.nf, st);
    return s;
  }

  template <class T>
  fc_status project(double dtj, const T* vin, T* vout, void* gp_out, void* st) {
    cx<T>* Xs = Xb<T>((cur + 1) % 3);
    fc_status s = phys_to_state<T>(vin, Xs, 3, at<double2>(l.gradp), dtj, st);
    if (!s) s = z_project<T>(Xs, dtj, st);
    if (!s) s = state_to_phys<T>(Xs, vout, 3, st);
    if (!s && gp_out) s = gradp_out(gp_out, st);
    return s;
  }

  template <class T>
  fc_status step(double dt, void* st) {
    const int o = p.rk_order;
    const int it = cur, ia = (cur + 1) % 3, ib = (cur + 2) % 3;
    int ij = it;
    fc_status s = FC_OK;
    for (int j = 1; j <= o && !s; ++j) {
      const double dtj = dt / (o + 1 - j);  // stage step dt_j = dt / (o + 1 - j)
      const int in = (ij == ia) ? ib : ia;
      s = nonlinear<T>(Xb<T>(ij), st);
      if (!s) s = z_combine<T>(buf<T>(l.NL), Xb<T>(it), Xb<T>(ij), Xb<T>(in), dtj, 1, l.nf, st);
      if (!s) s = mean_stage<T>(it, ij, in, dtj, st);
      if (!s) s = z_project<T>(Xb<T>(in), dtj, st);
      ij = in;
    }
    if (!s) cur = ij;
    return s;
  }

  // ------------------------------------------------------------- dispatch
  bool f32() const { return p.prec == FC_F32; }
  fc_status set_fields_any(const void* phys, void* st) {
    return f32() ? set_fields<float>((const float*)phys, st) : set_fields<double>((const double*)phys, st);
  }
  fc_status get_fields_any(void* phys, void* st) {
    return f32() ? get_fields<float>((float*)phys, st) : get_fields<double>((double*)phys, st);
  }
  fc_status rhs_any(const void* in, void* out, void* st) {
    return f32() ? rhs<float>((const float*)in, (float*)out, st) : rhs<double>((const double*)in, (double*)out, st);
  }
  fc_status project_any(double dtj, const void* in, void* out, void* gp, void* st) {
    return f32() ? project<float>(dtj, (const float*)in, (float*)out, gp, st)
                 : project<double>(dtj, (const double*)in, (double*)out, gp, st);
  }
  fc_status step_any(double dt, void* st) { return f32() ? step<float>(dt, st) : step<double>(dt, st); }

  // diagnostics of the current state (Sec. 6, Sec. 7); synchronous
  template <class T>
  fc_status diagnostics(double out[6], void* st) {
    fc_status s = bk.memset(ws + l.diag, 0, sizeof(double) * 8, st);
    if (!s) s = z_deriv<T>(Xb<T>(cur), l.nf, st);
    if (!s) {
      using K = KDiag<T>;
      typename K::Args a;
      a.g = zgeom(l.nf); a.t = ztab<T>(); a.Nx = p.Nx;
      a.X = Xb<T>(cur); a.DZ = buf<T>(l.DZ); a.acc = at<double>(l.diag);
      s = bk.template run<K>(a, l.ntiles, st);
    }
    if (!s) s = bk.d2h(out, ws + l.diag, sizeof(double) * 6, st);
    return s;
  }
  fc_status diagnostics_any(double out[6], void* st) {
    return f32() ? diagnostics<float>(out, st) : diagnostics<double>(out, st);
  }
  // the same sums into slot `slot` of the device-side series (asynchronous)
  template <class T>
  fc_status diag_record(int slot, void* st) {
    double* acc = at<double>(l.dser) + 8 * (size_t)slot;
    fc_status s = bk.memset(acc, 0, sizeof(double) * 8, st);
    if (!s) s = z_deriv<T>(Xb<T>(cur), l.nf, st);
    if (!s) {
      using K = KDiag<T>;
      typename K::Args a;
      a.g = zgeom(l.nf); a.t = ztab<T>(); a.Nx = p.Nx;
      a.X = Xb<T>(cur); a.DZ = buf<T>(l.DZ); a.acc = acc;
      s = bk.template run<K>(a, l.ntiles, st);
    }
    return s;
  }
  fc_status diag_record_any(int slot, void* st) {
    return f32() ? diag_record<float>(slot, st) : diag_record<double>(slot, st);
  }
  size_t state_bytes() const { return 2 * l.es * l.nf * l.Np * l.plines; }
  // wall planes: internal [2][2][Ny][Kxp] <-> public [2][2][Ny][Kx] (complex double)
  fc_status gradp_out(void* dst, void* st) {
    return bk.d2d_2d(dst, 16 * (size_t)l.Kx, ws + l.gradp, 16 * (size_t)l.Kxp, 16 * (size_t)l.Kx, 4 * (size_t)p.Ny, st);
  }
  fc_status gradp_in(const void* src, void* st) {
    return bk.d2d_2d(ws + l.gradp, 16 * (size_t)l.Kxp, src, 16 * (size_t)l.Kx, 16 * (size_t)l.Kx, 4 * (size_t)p.Ny, st);
  }
};

}  // namespace fcns
