// Internal declarations shared by the C ABI and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <complex>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fcns.h"

namespace fcns {

void set_error(const std::string& msg);
fc_status cuda_status(cudaError_t e, const char* what);
// host-side failure injection: the status an armed entry point must return
// now (FC_OK when it is not armed); checked first thing by the entry points
fc_status injected(const char* entry);

// lengths of the two-pass line engine that are compiled: L = L1 * L2
struct EngineShape { int L, L1, L2; };
const std::vector<EngineShape>& engine_shapes();
// smallest compiled L >= need (0 if none)
int pick_engine_length(int need);

// per-device copies of the derivative tables of one plan
struct DerivDevTables {
  int device = -1;
  int L = 0;
  double* Mr = nullptr;
  float2* Mr2 = nullptr;  // (hi, lo) float split of Mr
  void* tw32 = nullptr;  // float2[L]
  void* tw64 = nullptr;  // double2[L]
  void* H1_32 = nullptr; // spectra of d1 and d2 separately (paired-line kernel)
  void* H1_64 = nullptr;
  void* H2_32 = nullptr;
  void* H2_64 = nullptr;
  // staging of fc_deriv_z_host: three rotating slots of (input, d1, d2) slab
  // buffers of stage_bytes each, and the copy-in / compute / copy-out streams
  size_t stage_bytes = 0;
  void* stage[3][3] = {};
  cudaStream_t st_in = nullptr, st_run = nullptr, st_out = nullptr;
  cudaEvent_t ev_in[3] = {}, ev_run[3] = {}, ev_out[3] = {};
};

struct PlanData {
  int d, C, Nz, Np, M, n_os;
  double ls_residual;
  std::vector<double> Mr;
  std::mutex mtx;
  std::mutex host_mtx;   // serialises fc_deriv_z_host calls on the plan (shared staging)
  std::vector<DerivDevTables> dev;
};


// host copies of the derivative tables of one plan, in both precisions
struct PlanHostTables {
  unsigned long long serial = 0;  // unique per plan in the process (never reused)
  int L = 0, L1 = 0, L2 = 0;
  std::vector<std::complex<double>> tw;
  std::vector<float2> tw32, Mr2, H1_32, H2_32;
  std::vector<double2> tw64, H1_64, H2_64;
};

// argument checks shared by the fc_deriv_z entry points
fc_status check_deriv_args(const PlanData& p, const PlanHostTables& t, fc_dtype dtype, int batch, int Nx, int Ny,
                           double Lz, const void* f, void* df, void* d2f, const char* who);

}  // namespace fcns

struct fc_plan {
  fcns::PlanData data;
  fcns::PlanHostTables deriv;
};

namespace fcns {

fc_status launch_deriv_z(const DerivDevTables& t, const PlanData& p, fc_dtype dtype, int batch,
                         long long lines, double Lz, const void* f, void* df, void* d2f,
                         cudaStream_t stream);

}  // namespace fcns
