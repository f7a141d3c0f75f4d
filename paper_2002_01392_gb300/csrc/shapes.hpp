// Transform shapes compiled into the library.
//   Z shapes: padded length L = L1 * L2 of the z-line circular convolutions
//             and Bluestein DFTs (L >= N' + Nz - 1 and L >= 2 N' - 1).
//   XY shapes: x and y lengths Nx, Ny (2/3/5-smooth).
#pragma once

#ifdef FC_HOSTCHECK
#define FC_ZSHAPES(M) M(160, 10, 16) M(288, 16, 18)
#define FC_XYSHAPES(M) M(16, 4, 4) M(32, 4, 8)
#else
#define FC_ZSHAPES(M) M(160, 10, 16) M(288, 16, 18) M(320, 16, 20) M(576, 24, 24) M(1080, 30, 36)
#define FC_XYSHAPES(M) \
  M(16, 4, 4) M(32, 4, 8) M(64, 8, 8) M(96, 8, 12) M(128, 8, 16) M(192, 12, 16) M(256, 16, 16) M(512, 16, 32) M(1024, 32, 32)
#endif

namespace fcns {
// lines per CTA of the z kernels and of the y kernels
template <class T, int L> constexpr int z_lines() {
  return sizeof(T) == 4 ? (L >= 576 ? 4 : 8) : (L >= 576 ? 2 : 4);
}
template <class T, int L> constexpr int zproj_lines() {
  return sizeof(T) == 4 ? (L >= 576 ? 4 : 8) : (L >= 576 ? 2 : 4);
}
template <class T, int N> constexpr int y_lines() {
  return sizeof(T) == 4 ? (N >= 512 ? 4 : (N >= 128 ? 8 : 16)) : (N >= 512 ? 2 : (N >= 128 ? 4 : 8));
}
// row-pair jobs per CTA of the x row transforms
template <int N> constexpr int x_jobs() { return N >= 512 ? 2 : (N >= 128 ? 4 : 8); }
}  // namespace fcns
