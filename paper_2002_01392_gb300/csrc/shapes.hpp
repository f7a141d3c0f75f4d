// Transform shapes compiled into the library.
//   Z shapes: length L = L1 * L2 of the z-line transforms and whether it is a
//             DIRECT length (used only when N' = L: z derivatives and filter
//             are spectral multipliers, the projection's DFTs are plain
//             length-N' transforms -- the paper's smooth N') or a padded one
//             (any N' with L >= N' + Nz - 1 and L >= 2 N' - 1: circular
//             convolutions and Bluestein DFTs).
//   XY shapes: x and y lengths Nx, Ny (2/3/5-smooth).
#pragma once

#ifdef FC_HOSTCHECK
#define FC_ZSHAPES_DIRECT(M) M(64, 8, 8, true) M(512, 16, 32, true) M(1536, 32, 48, true)
#define FC_ZSHAPES_PADDED(M) M(160, 10, 16, false) M(288, 16, 18, false) M(1080, 30, 36, false)
#define FC_XYSHAPES(M) M(16, 4, 4) M(32, 4, 8) M(128, 8, 16)
#else
#define FC_ZSHAPES_DIRECT(M) \
  M(64, 8, 8, true) M(128, 8, 16, true) M(256, 16, 16, true) M(512, 16, 32, true) M(768, 24, 32, true) \
  M(1024, 32, 32, true) M(1536, 32, 48, true)
#define FC_ZSHAPES_PADDED(M) \
  M(160, 10, 16, false) M(288, 16, 18, false) M(320, 16, 20, false) M(576, 24, 24, false) M(1080, 30, 36, false) \
  M(1152, 32, 36, false)
#define FC_XYSHAPES(M) \
  M(16, 4, 4) M(32, 4, 8) M(64, 8, 8) M(96, 8, 12) M(128, 8, 16) M(192, 12, 16) M(256, 16, 16) M(512, 16, 32) M(1024, 32, 32)
#endif
#define FC_ZSHAPES(M) FC_ZSHAPES_DIRECT(M) FC_ZSHAPES_PADDED(M)

// Alternative radix schedules of padded z lengths (float32 kernels only): the
// same length with the first-pass and second-pass factors swapped, M(L, L1,
// L2).  The autotuner of ns_tune times both schedules (and both tiles) of the
// z kernels; the default is the FC_ZSHAPES_PADDED one.
#ifdef FC_HOSTCHECK
#define FC_ZSHAPES_ALT(M) M(160, 16, 10) M(288, 18, 16)
#else
#define FC_ZSHAPES_ALT(M) M(160, 16, 10) M(288, 18, 16) M(320, 20, 16)
#endif

namespace fcns {
// lines per CTA of the z kernels and of the y kernels.  float: 8 lines (64
// contiguous bytes of every z / ky row per CTA); measured on the 1024^2 x 513
// Boussinesq step, 8 instead of 4 lines for the z kernels and the y transforms
// of length 1024 took the step from 314 to 256 ms (2 lines: 350-363 ms).
template <class T, int L> constexpr int z_lines() {
  return sizeof(T) == 4 ? 8 : (L >= 576 ? 2 : 4);
}
// the z-derivative kernel (two exchange buffers) keeps 4 lines at L >= 576:
// 14.7 ms against 17.8 ms per launch with 8 on the same step
template <class T, int L> constexpr int zderiv_lines() {
  return sizeof(T) == 4 ? (L >= 576 ? 4 : 8) : (L >= 576 ? 2 : 4);
}
template <class T, int L> constexpr int zproj_lines() {
  return sizeof(T) == 4 ? 8 : (L >= 576 ? 2 : 4);
}
template <class T, int N> constexpr int y_lines() {
  return sizeof(T) == 4 ? (N >= 128 ? 8 : 16) : (N >= 512 ? 2 : (N >= 128 ? 4 : 8));
}
// the alternative lines per CTA compiled beside each default (the autotuner
// of ns_tune times both)
template <int D> constexpr int tile_alt() { return D >= 8 ? D / 2 : 2 * D; }
// the alternative tile of the y transforms: float lengths >= 128 widen to 16
// lines (128 contiguous bytes of every ky row per CTA; the y inverse then runs
// with one exchange buffer, KYInv3S), else tile_alt
template <class T, int N> constexpr bool y_wide() { return sizeof(T) == 4 && N >= 128; }
template <class T, int N> constexpr int y_lines_alt() {
  return y_wide<T, N>() ? 16 : tile_alt<y_lines<T, N>()>();
}
// row-pair jobs per CTA of the x row transforms
template <int N> constexpr int x_jobs() { return N >= 512 ? 2 : (N >= 128 ? 4 : 8); }
}  // namespace fcns
