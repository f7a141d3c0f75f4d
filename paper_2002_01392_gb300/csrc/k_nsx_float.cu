// Instantiation of the x transform kernels of the Navier-Stokes step (float).
#include "dev_run.cuh"
#include "ns_kernels.cuh"
#include "shapes.hpp"

namespace fcns {
#define FC_INST_X(NN, A, B)                                                    \
  template struct DevRun<KXRow<float, A, B, -1, x_jobs<NN>()>>;                 \
  template struct DevRun<KXRow<float, A, B, 1, x_jobs<NN>()>>;                  \
  template struct DevRun<KXPass<float, A, B, 3>>;                               \
  template struct DevRun<KXPass<float, A, B, 4>>;
FC_XYSHAPES(FC_INST_X)
#undef FC_INST_X
}  // namespace fcns
