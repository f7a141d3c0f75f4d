// Instantiation of the z-line kernels of the Navier-Stokes step (double), direct lengths.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_Z(LL, A, B, D)                                                                          \
  template struct DevRun<KZDeriv<double, A, B, zderiv_lines<double, LL>(), D ? A : A / 2>>;                      \
  template struct DevRun<KZDeriv<double, A, B, tile_alt<zderiv_lines<double, LL>()>(), D ? A : A / 2>>;          \
  template struct DevRun<KZCombine<double, A, B, z_lines<double, LL>(), D ? A : A / 2>>;                         \
  template struct DevRun<KZCombine<double, A, B, tile_alt<z_lines<double, LL>()>(), D ? A : A / 2>>;             \
  template struct DevRun<KZProject<double, A, B, zproj_lines<double, LL>(), D>>;                                 \
  template struct DevRun<KZProject<double, A, B, tile_alt<zproj_lines<double, LL>()>(), D>>;
FC_ZSHAPES_DIRECT(FC_INST_Z)
#undef FC_INST_Z
}  // namespace fcns
