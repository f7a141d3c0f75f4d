// Instantiation of the x transform kernels of the Navier-Stokes step (double).
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_X(NN, A, B)                                                    \
  template struct DevRun<KXRow<double, A, B, -1, x_jobs<NN>()>>;                 \
  template struct DevRun<KXRow<double, A, B, 1, x_jobs<NN>()>>;                  \
  template struct DevRun<KXPass<double, A, B, 3>>;                               \
  template struct DevRun<KXPass<double, A, B, 4>>;
FC_XYSHAPES(FC_INST_X)
#undef FC_INST_X
}  // namespace fcns
