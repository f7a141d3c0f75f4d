// Instantiation of the z-line kernels of the Navier-Stokes step (float), padded lengths.
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
FC_ZSHAPES_PADDED(FC_INST_Z)
#undef FC_INST_Z
template struct DevRun<KZContinue<float, 8>>;
template struct DevRun<KDiag<float>>;
template struct DevRun<KMeanLine<float>>;
template struct DevRun<KMeanInit<float>>;
template struct DevRun<KInterp<float>>;
template struct DevRun<KProf<float>>;
template struct DevRun<KFinite<float>>;
template struct DevRun<KCount<float>>;
}  // namespace fcns
