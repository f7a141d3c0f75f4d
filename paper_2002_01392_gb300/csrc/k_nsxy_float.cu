// Instantiation of the x and y transform kernels of the Navier-Stokes step (float).
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_XY(NN, A, B)                                                   \
  template struct DevRun<KYInv3<float, A, B, y_lines<float, NN>()>>;             \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), -1>>;            \
  template struct DevRun<KY1<float, A, B, y_lines<float, NN>(), 1>>;             \
  template struct DevRun<KXRow<float, A, B, -1, x_jobs<NN>()>>;                 \
  template struct DevRun<KXRow<float, A, B, 1, x_jobs<NN>()>>;                  \
  template struct DevRun<KXPass<float, A, B, 3>>;                               \
  template struct DevRun<KXPass<float, A, B, 4>>;
FC_XYSHAPES(FC_INST_XY)
#undef FC_INST_XY
}  // namespace fcns
