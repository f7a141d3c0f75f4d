// fc_alu_probe: arithmetic-pipe throughput of this GPU, for the ALU rooflines
// of the transform kernels (their float32 / float64 work is adds, multiplies
// and fused multiply-adds, scalar or packed two-wide).
//
// Each thread runs NACC independent dependency chains (enough to cover the
// pipe latency at full occupancy) of one instruction kind; the grid fills
// every SM.  The chains are seeded from the thread index and the sink is
// written only if a result equals an impossible value, so the work cannot be
// removed by the compiler and the memory traffic is nil.
#include "internal.hpp"

namespace fcns {
namespace {

constexpr int kNacc = 8;
constexpr int kUnroll = 16;

template <int KIND>
__global__ void __launch_bounds__(256) alu_probe_kernel(int iters, float* sink) {
  const float t = (float)threadIdx.x * 1e-7f;
  if constexpr (KIND == 0 || KIND == 1) {  // 0: FFMA, 1: FADD (scalar float32)
    float a[kNacc];
#pragma unroll
    for (int i = 0; i < kNacc; ++i) a[i] = t + (float)i;
    const float m = 0.999999f, c = 1e-7f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kNacc; ++i) a[i] = KIND == 0 ? __fmaf_rn(a[i], m, c) : __fadd_rn(a[i], c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kNacc; ++i) s += a[i];
    if (s == -1.2345f) sink[threadIdx.x] = s;
  } else if constexpr (KIND == 2 || KIND == 3) {  // 2: FFMA2, 3: FADD2 (packed 2 x float32)
    float2 a[kNacc];
#pragma unroll
    for (int i = 0; i < kNacc; ++i) a[i] = make_float2(t + (float)i, t - (float)i);
    const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kNacc; ++i) a[i] = KIND == 2 ? __ffma2_rn(a[i], m, c) : __fadd2_rn(a[i], c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kNacc; ++i) s += a[i].x + a[i].y;
    if (s == -1.2345f) sink[threadIdx.x] = s;
  } else {  // 4: DFMA (float64)
    double a[kNacc];
#pragma unroll
    for (int i = 0; i < kNacc; ++i) a[i] = (double)t + i;
    const double m = 0.9999999, c = 1e-9;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
#pragma unroll
        for (int i = 0; i < kNacc; ++i) a[i] = __fma_rn(a[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kNacc; ++i) s += a[i];
    if (s == -1.2345) sink[threadIdx.x] = (float)s;
  }
}

}  // namespace
}  // namespace fcns

using namespace fcns;

extern "C" fc_status fc_alu_probe(int kind, int iters, void* sink, double* lane_ops, fc_stream_t stream) {
  if (kind < 0 || kind > 4 || iters < 1 || !sink) {
    set_error("fc_alu_probe: kind must be 0..4, iters >= 1, sink non-NULL (256 floats of device memory)");
    return FC_ERR_ARG;
  }
  int dev = 0, sms = 0;
  fc_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (!s) s = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  if (s) return s;
  const int threads = 256, blocks = sms * 8;  // 2048 threads per SM: full occupancy
  cudaStream_t st = (cudaStream_t)stream;
  float* out = static_cast<float*>(sink);
  switch (kind) {
    case 0: alu_probe_kernel<0><<<blocks, threads, 0, st>>>(iters, out); break;
    case 1: alu_probe_kernel<1><<<blocks, threads, 0, st>>>(iters, out); break;
    case 2: alu_probe_kernel<2><<<blocks, threads, 0, st>>>(iters, out); break;
    case 3: alu_probe_kernel<3><<<blocks, threads, 0, st>>>(iters, out); break;
    default: alu_probe_kernel<4><<<blocks, threads, 0, st>>>(iters, out); break;
  }
  // lane operations: one per scalar instruction and thread, two per packed one
  if (lane_ops)
    *lane_ops = (double)blocks * threads * iters * kUnroll * kNacc * ((kind == 2 || kind == 3) ? 2.0 : 1.0);
  return cuda_status(cudaGetLastError(), "fc_alu_probe launch");
}
