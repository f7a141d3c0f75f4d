// Instantiation of the z-line kernels of the Navier-Stokes step (double), padded lengths.
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
FC_ZSHAPES_PADDED(FC_INST_Z)
#undef FC_INST_Z
template struct DevRun<KZContinue<double, 8>>;
template struct DevRun<KDiag<double>>;
template struct DevRun<KMeanLine<double>>;
template struct DevRun<KMeanInit<double>>;
template struct DevRun<KInterp<double>>;
template struct DevRun<KProf<double>>;
template struct DevRun<KFinite<double>>;
template struct DevRun<KCount<double>>;
}  // namespace fcns
