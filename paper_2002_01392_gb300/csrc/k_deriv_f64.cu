// fc_deriv_z kernels of every compiled length, double.
#include "deriv_launch.cuh"

namespace fcns {
template fc_status launch_deriv_typed<double>(const DerivDevTables&, const PlanData&, int, long long, double, const void*,
                                          void*, void*, cudaStream_t);
}  // namespace fcns
