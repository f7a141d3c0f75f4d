// Instantiation of the z-line kernels of the Navier-Stokes step (float), direct lengths.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_Z(LL, A, B, D)                                                                          \
  template struct DevRun<KZDeriv<float, A, B, zderiv_lines<float, LL>(), D ? A : A / 2>>;                      \
  template struct DevRun<KZDeriv<float, A, B, tile_alt<zderiv_lines<float, LL>()>(), D ? A : A / 2>>;          \
  template struct DevRun<KZCombine<float, A, B, z_lines<float, LL>(), D ? A : A / 2>>;                         \
  template struct DevRun<KZCombine<float, A, B, tile_alt<z_lines<float, LL>()>(), D ? A : A / 2>>;             \
  template struct DevRun<KZProject<float, A, B, zproj_lines<float, LL>(), D>>;                                 \
  template struct DevRun<KZProject<float, A, B, tile_alt<zproj_lines<float, LL>()>(), D>>;
FC_ZSHAPES_DIRECT(FC_INST_Z)
#undef FC_INST_Z
}  // namespace fcns
