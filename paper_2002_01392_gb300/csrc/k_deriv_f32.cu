// fc_deriv_z kernels of every compiled length, float.
#include "deriv_launch.cuh"

namespace fcns {
template fc_status launch_deriv_typed<float>(const DerivDevTables&, const PlanData&, int, long long, double, const void*,
                                          void*, void*, cudaStream_t);
}  // namespace fcns
