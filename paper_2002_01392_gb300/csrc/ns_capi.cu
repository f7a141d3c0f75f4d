// Navier-Stokes entry points of the C ABI (GPU backend of NsCore).
#include <cstring>
#include <new>

#include "internal.hpp"
#include "ns_core.hpp"

namespace fcns {

template <class K>
struct DevRun {
  static fc_status run(const typename K::Args& a, long long grid, cudaStream_t s);
};

struct DeviceBK {
  int device = -1;
  template <class K>
  fc_status run(const typename K::Args& a, long long grid, void* st) {
    return DevRun<K>::run(a, grid, (cudaStream_t)st);
  }
  fc_status alloc(void** p, size_t b) { return cuda_status(cudaMalloc(p, b), "cudaMalloc(workspace)"); }
  void free(void* p) { cudaFree(p); }
  fc_status h2d(void* dst, const void* src, size_t b) {
    return cuda_status(cudaMemcpy(dst, src, b, cudaMemcpyHostToDevice), "cudaMemcpy(tables)");
  }
  fc_status d2d(void* dst, const void* src, size_t b, void* st) {
    return cuda_status(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, (cudaStream_t)st), "cudaMemcpyAsync");
  }
  fc_status d2d_2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows, void* st) {
    return cuda_status(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDeviceToDevice,
                                         (cudaStream_t)st), "cudaMemcpy2DAsync");
  }
  fc_status memset(void* dst, int v, size_t b, void* st) {
    return cuda_status(cudaMemsetAsync(dst, v, b, (cudaStream_t)st), "cudaMemsetAsync");
  }
  fc_status sync(void*) { return cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize"); }
  fc_status d2h(void* dst, const void* src, size_t b, void* st) {
    fc_status s = cuda_status(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, (cudaStream_t)st), "cudaMemcpyAsync(D2H)");
    if (!s) s = cuda_status(cudaStreamSynchronize((cudaStream_t)st), "cudaStreamSynchronize");
    return s;
  }
};

}  // namespace fcns

using namespace fcns;

struct ns_sim {
  NsCore<DeviceBK> core;
  int device = -1;
};

static fc_status check_sim(ns_sim_t s, const char* what) {
  if (!s) { set_error(std::string(what) + ": NULL simulation"); return FC_ERR_ARG; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) {
    set_error(std::string(what) + ": called with a different current device than ns_create");
    return FC_ERR_STATE;
  }
  return FC_OK;
}

extern "C" {

fc_status ns_params_default(ns_params* p) {
  if (!p) return FC_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->d = 5; p->C = 25; p->nfields = 3; p->rk_order = 3;
  p->Lx = p->Ly = 6.283185307179586; p->Lz = 1.0; p->nu = 1e-2;
  p->filter = 1; p->filter_beta = 16.0 * 2.302585092994046; p->filter_2p = 100.0; p->prec = FC_F64;
  return FC_OK;
}

fc_status ns_workspace_bytes(const ns_params* p, size_t* bytes) {
  if (!p || !bytes) { set_error("ns_workspace_bytes: NULL argument"); return FC_ERR_ARG; }
  NsLayout l;
  fc_status s = ns_layout(*p, &l);
  if (s) { set_error("ns_workspace_bytes: parameters invalid or outside the compiled shapes"); return s; }
  *bytes = l.total;
  return FC_OK;
}

fc_status ns_create(const ns_params* p, void* dev_workspace, size_t bytes, ns_sim_t* out) {
  if (!p || !out) { set_error("ns_create: NULL argument"); return FC_ERR_ARG; }
  *out = nullptr;
  ns_sim* s = new (std::nothrow) ns_sim;
  if (!s) return FC_ERR_NOMEM;
  cudaGetDevice(&s->device);
  fc_status st = s->core.create(*p, dev_workspace, bytes);
  if (st) {
    if (st == FC_ERR_ARG) set_error("ns_create: invalid parameters");
    if (st == FC_ERR_UNSUPPORTED) set_error("ns_create: sizes outside the compiled transform shapes");
    s->core.destroy();
    delete s;
    return st;
  }
  *out = s;
  return FC_OK;
}

fc_status ns_destroy(ns_sim_t s) {
  if (!s) return FC_ERR_ARG;
  fc_status st = s->core.destroy();
  delete s;
  return st;
}

fc_status ns_set_fields(ns_sim_t s, const void* phys, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_set_fields");
  if (st) return st;
  if (!phys) { set_error("ns_set_fields: NULL fields"); return FC_ERR_ARG; }
  return s->core.set_fields_any(phys, stream);
}

fc_status ns_get_fields(ns_sim_t s, void* phys, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_get_fields");
  if (st) return st;
  if (!phys) { set_error("ns_get_fields: NULL fields"); return FC_ERR_ARG; }
  return s->core.get_fields_any(phys, stream);
}

fc_status ns_get_state(ns_sim_t s, void* spec, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_get_state");
  if (st) return st;
  if (!spec) return FC_ERR_ARG;
  return s->core.bk.d2d(spec, s->core.ws + s->core.l.X[s->core.cur], s->core.state_bytes(), stream);
}

fc_status ns_put_state(ns_sim_t s, const void* spec, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_put_state");
  if (st) return st;
  if (!spec) return FC_ERR_ARG;
  st = s->core.bk.d2d(s->core.ws + s->core.l.X[s->core.cur], spec, s->core.state_bytes(), stream);
  if (!st) st = s->core.mean_init_any(stream);
  return st;
}

fc_status ns_get_wall_gradp(ns_sim_t s, void* gradp, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_get_wall_gradp");
  if (st) return st;
  if (!gradp) return FC_ERR_ARG;
  return s->core.gradp_out(gradp, stream);
}

fc_status ns_put_wall_gradp(ns_sim_t s, const void* gradp, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_put_wall_gradp");
  if (st) return st;
  if (!gradp) return FC_ERR_ARG;
  return s->core.gradp_in(gradp, stream);
}

fc_status ns_rhs(ns_sim_t s, const void* phys_in, void* rhs_out, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_rhs");
  if (st) return st;
  if (!phys_in || !rhs_out || phys_in == rhs_out) { set_error("ns_rhs: bad buffers"); return FC_ERR_ARG; }
  return s->core.rhs_any(phys_in, rhs_out, stream);
}

fc_status fc_poisson_project(ns_sim_t s, double dt_stage, const void* vstar_phys, void* v_phys, void* gradp_wall,
                             fc_stream_t stream) {
  fc_status st = check_sim(s, "fc_poisson_project");
  if (st) return st;
  if (!vstar_phys || !v_phys || !(dt_stage > 0)) { set_error("fc_poisson_project: bad arguments"); return FC_ERR_ARG; }
  return s->core.project_any(dt_stage, vstar_phys, v_phys, gradp_wall, stream);
}

fc_status rk_step(ns_sim_t s, double dt, fc_stream_t stream) {
  fc_status st = check_sim(s, "rk_step");
  if (st) return st;
  if (!(dt > 0)) { set_error("rk_step: dt must be positive"); return FC_ERR_ARG; }
  return s->core.step_any(dt, stream);
}

fc_status ns_diagnostics(ns_sim_t s, double* div_ms, double* wall_u_ms, double* wall_w_ms, double* flow_rate,
                         double* nusselt, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_diagnostics");
  if (st) return st;
  double acc[6];
  st = s->core.diagnostics_any(acc, stream);
  if (st) return st;
  const ns_params& p = s->core.p;
  const double n2 = (double)p.Nx * p.Ny * (double)p.Nx * p.Ny;
  if (div_ms) *div_ms = acc[0] / n2 / p.Nz;
  if (wall_u_ms) *wall_u_ms = acc[1] / n2 / 2.0;
  if (wall_w_ms) *wall_w_ms = acc[2] / n2 / 2.0;
  if (flow_rate) *flow_rate = acc[3] / ((double)p.Nx * p.Ny) / p.Nz;
  if (nusselt) {
    if (p.nfields == 4 && p.gamma != 0.0) {
      const double m0 = acc[4] / ((double)p.Nx * p.Ny), m1 = acc[5] / ((double)p.Nx * p.Ny);
      *nusselt = 0.5 * ((1.0 - m0 / p.gamma) + (1.0 - m1 / p.gamma));
    } else {
      *nusselt = 0.0;
    }
  }
  return FC_OK;
}

}  // extern "C"
