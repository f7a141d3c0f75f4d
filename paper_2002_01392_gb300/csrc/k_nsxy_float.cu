// Instantiation of the y transform kernels of the Navier-Stokes step (float), both
// compiled tile sizes.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_Y(NN, A, B)                                                             \
  template struct DevRun<KYInv3<float, A, B, y_lines<float, NN>()>>;                         \
  template struct DevRun<std::conditional_t<y_wide<float, NN>(), KYInv3S<float, A, B, 16>, KYInv3<float, A, B, y_lines_alt<float, NN>()>>>;             \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), -1>>;                        \
  template struct DevRun<KY1<float, A, B, y_lines_alt<float, NN>(), -1>>;            \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), 1>>;                         \
  template struct DevRun<KY1<float, A, B, y_lines_alt<float, NN>(), 1>>;
FC_XYSHAPES(FC_INST_Y)
#undef FC_INST_Y
}  // namespace fcns
