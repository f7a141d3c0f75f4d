// fc_deriv_z: compiled transform shapes and the dispatch by precision.
#include "internal.hpp"

namespace fcns {

template <class T>
fc_status launch_deriv_typed(const DerivDevTables& t, const PlanData& p, int batch, long long lines, double Lz,
                             const void* f, void* df, void* d2f, cudaStream_t stream);

const std::vector<EngineShape>& engine_shapes() {
  static const std::vector<EngineShape> s = {
      {64, 8, 8},     {96, 8, 12},    {128, 8, 16},   {160, 10, 16},  {192, 12, 16}, {256, 16, 16},
      {288, 16, 18},  {320, 16, 20},  {512, 16, 32},  {576, 24, 24},  {768, 24, 32}, {1024, 32, 32},
      {1080, 30, 36}, {1152, 32, 36}, {1536, 32, 48}};
  return s;
}

int pick_engine_length(int need) {
  for (auto& s : engine_shapes())
    if (s.L >= need) return s.L;
  return 0;
}

fc_status launch_deriv_z(const DerivDevTables& t, const PlanData& p, fc_dtype dtype, int batch,
                         long long lines, double Lz, const void* f, void* df, void* d2f,
                         cudaStream_t stream) {
  return dtype == FC_F32 ? launch_deriv_typed<float>(t, p, batch, lines, Lz, f, df, d2f, stream)
                         : launch_deriv_typed<double>(t, p, batch, lines, Lz, f, df, d2f, stream);
}

}  // namespace fcns
