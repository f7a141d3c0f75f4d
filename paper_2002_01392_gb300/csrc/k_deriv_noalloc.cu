// fc_deriv_z_noalloc: fc_deriv_z without any device allocation.
//
// fc_deriv_z keeps its continuation matrix, kernel spectra and twiddles in
// device memory that the library allocates with cudaMalloc the first time a
// plan is used on a device.  Some callers cannot have the library allocate:
// applications whose device memory belongs to a host framework or to a
// fixed-size arena and that forbid allocations by plug-ins, and programs run
// under a device-memory budget that a library must not grow.  This entry point
// instead keeps those tables in one file-scope static device array of fixed
// size (kNoAllocBytes = 128 KiB, reserved by every GPU that loads the library
// until the process exits).  A call whose plan and precision differ from the
// tables the array holds on this device copies the plan's tables into it on
// the caller's stream first; a call with the same plan and precision as the
// previous call on the device launches the kernel at once.
#include <mutex>
#include <mutex>

#include "internal.hpp"

namespace fcns {
namespace {

constexpr size_t kNoAllocBytes = 128 * 1024;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the tables of the last call.
static __device__ __align__(256) unsigned char g_deriv_scratch[kNoAllocBytes];

std::mutex g_mtx;
void* g_scratch_addr[kMaxDevices] = {};
// which tables the array holds per device: the plan's serial number and the
// precision of the last upload (0: none, or an upload that failed part-way)
unsigned long long g_loaded_serial[kMaxDevices] = {};
int g_loaded_dtype[kMaxDevices] = {};

// Device address of g_deriv_scratch on the current device (the host-side
// symbol is only a stand-in and must never be passed to a kernel).
fc_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) { set_error("fc_deriv_z_noalloc: device index out of range"); return FC_ERR_UNSUPPORTED; }
  std::lock_guard<std::mutex> lk(g_mtx);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    fc_status s = cuda_status(cudaGetSymbolAddress(&p, g_deriv_scratch), "cudaGetSymbolAddress(g_deriv_scratch)");
    if (s) return s;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return FC_OK;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace
}  // namespace fcns

using namespace fcns;

extern "C" fc_status fc_deriv_z_noalloc(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                                        const void* f, void* df, void* d2f, fc_stream_t stream) {
  if (fc_status inj = injected("fc_deriv_z_noalloc")) return inj;
  if (!plan) { set_error("fc_deriv_z_noalloc: NULL plan"); return FC_ERR_ARG; }
  fc_status s = check_deriv_args(plan->data, plan->deriv, dtype, batch, Nx, Ny, Lz, f, df, d2f, "fc_deriv_z_noalloc");
  if (s) return s;
  const PlanHostTables& h = plan->deriv;
  const size_t cs = dtype == FC_F32 ? sizeof(float2) : sizeof(double2);
  const size_t nMr = plan->data.Mr.size();
  const size_t oMr = 0, oMr2 = align256(sizeof(double) * nMr), oH1 = oMr2 + align256(sizeof(float2) * nMr);
  const size_t oH2 = oH1 + align256(cs * h.L), oTw = oH2 + align256(cs * h.L), need = oTw + align256(cs * 2 * h.L);
  if (need > kNoAllocBytes) {
    set_error("fc_deriv_z_noalloc: tables of this plan exceed the 128 KiB static scratch");
    return FC_ERR_UNSUPPORTED;
  }
  int dev = -1;
  s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (s) return s;
  unsigned char* base = nullptr;
  s = scratch_address(dev, &base);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_mtx);
    if (g_loaded_serial[dev] != h.serial || g_loaded_dtype[dev] != (int)dtype) {
      g_loaded_serial[dev] = 0;
      const void* H1src = dtype == FC_F32 ? (const void*)h.H1_32.data() : (const void*)h.H1_64.data();
      const void* H2src = dtype == FC_F32 ? (const void*)h.H2_32.data() : (const void*)h.H2_64.data();
      const void* Tsrc = dtype == FC_F32 ? (const void*)h.tw32.data() : (const void*)h.tw64.data();
      // every table the kernel reads is overwritten in full, so nothing left
      // by an earlier call with other tables is read
      s = cuda_status(cudaMemcpyAsync(base + oMr, plan->data.Mr.data(), sizeof(double) * nMr, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(Mr)");
      if (!s) s = cuda_status(cudaMemcpyAsync(base + oMr2, h.Mr2.data(), sizeof(float2) * nMr, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(Mr2)");
      if (!s) s = cuda_status(cudaMemcpyAsync(base + oH1, H1src, cs * h.L, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(H1)");
      if (!s) s = cuda_status(cudaMemcpyAsync(base + oH2, H2src, cs * h.L, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(H2)");
      if (!s) s = cuda_status(cudaMemcpyAsync(base + oTw, Tsrc, cs * 2 * h.L, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(tw)");
      if (s) return s;
      g_loaded_serial[dev] = h.serial;
      g_loaded_dtype[dev] = (int)dtype;
    }
  }
  DerivDevTables t;
  t.device = dev;
  t.L = h.L;
  t.Mr = reinterpret_cast<double*>(base + oMr);
  t.Mr2 = reinterpret_cast<float2*>(base + oMr2);
  t.H1_32 = t.H1_64 = base + oH1;
  t.H2_32 = t.H2_64 = base + oH2;
  t.tw32 = t.tw64 = base + oTw;
  return launch_deriv_z(t, plan->data, dtype, batch, (long long)Nx * Ny, Lz, f, df, d2f, st);
}
