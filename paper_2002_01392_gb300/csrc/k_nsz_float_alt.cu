// Instantiation of the z-line kernels of the Navier-Stokes step (float), the
// alternative radix schedules of padded lengths (first and second pass
// factors swapped), both tiles.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_ZA(LL, A, B)                                                                   \
  template struct DevRun<KZDeriv<float, A, B, zderiv_lines<float, LL>(), A / 2>>;              \
  template struct DevRun<KZDeriv<float, A, B, tile_alt<zderiv_lines<float, LL>()>(), A / 2>>;  \
  template struct DevRun<KZCombine<float, A, B, z_lines<float, LL>(), A / 2>>;                 \
  template struct DevRun<KZCombine<float, A, B, tile_alt<z_lines<float, LL>()>(), A / 2>>;     \
  template struct DevRun<KZProject<float, A, B, zproj_lines<float, LL>(), false>>;             \
  template struct DevRun<KZProject<float, A, B, tile_alt<zproj_lines<float, LL>()>(), false>>;
FC_ZSHAPES_ALT(FC_INST_ZA)
#undef FC_INST_ZA
}  // namespace fcns
