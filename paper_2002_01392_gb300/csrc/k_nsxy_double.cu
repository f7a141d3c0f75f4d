// Instantiation of the x and y transform kernels of the Navier-Stokes step (double).
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_XY(NN, A, B)                                                   \
  template struct DevRun<KYInv3<double, A, B, y_lines<double, NN>()>>;             \
  template struct DevRun<KY1<double, A, B, y_lines<double, NN>(), -1>>;            \
  template struct DevRun<KY1<double, A, B, y_lines<double, NN>(), 1>>;             \
  template struct DevRun<KXRow<double, A, B, -1, x_jobs<NN>()>>;                 \
  template struct DevRun<KXRow<double, A, B, 1, x_jobs<NN>()>>;                  \
  template struct DevRun<KXPass<double, A, B, 3>>;                               \
  template struct DevRun<KXPass<double, A, B, 4>>;
FC_XYSHAPES(FC_INST_XY)
#undef FC_INST_XY
}  // namespace fcns
