// Instantiation of the y transform kernels of the Navier-Stokes step (float), both
// compiled tile sizes.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_Y(NN, A, B)                                                             \
  template struct DevRun<KYInv3<float, A, B, y_lines<float, NN>()>>;                         \
  template struct DevRun<KYInv3<float, A, B, tile_alt<y_lines<float, NN>()>()>>;             \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), -1>>;                        \
  template struct DevRun<KY1<float, A, B, tile_alt<y_lines<float, NN>()>(), -1>>;            \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), 1>>;                         \
  template struct DevRun<KY1<float, A, B, tile_alt<y_lines<float, NN>()>(), 1>>;
FC_XYSHAPES(FC_INST_Y)
#undef FC_INST_Y
}  // namespace fcns
