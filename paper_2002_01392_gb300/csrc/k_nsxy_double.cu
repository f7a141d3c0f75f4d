// Instantiation of the y transform kernels of the Navier-Stokes step (double), both
// compiled tile sizes.
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_Y(NN, A, B)                                                             \
  template struct DevRun<KYInv3<double, A, B, y_lines<double, NN>()>>;                         \
  template struct DevRun<std::conditional_t<y_wide<double, NN>(), KYInv3S<double, A, B, 16>, KYInv3<double, A, B, y_lines_alt<double, NN>()>>>;             \
  template struct DevRun<KY1<double, A, B, y_lines<double, NN>(), -1>>;                        \
  template struct DevRun<KY1<double, A, B, y_lines_alt<double, NN>(), -1>>;            \
  template struct DevRun<KY1<double, A, B, y_lines<double, NN>(), 1>>;                         \
  template struct DevRun<KY1<double, A, B, y_lines_alt<double, NN>(), 1>>;
FC_XYSHAPES(FC_INST_Y)
#undef FC_INST_Y
}  // namespace fcns
