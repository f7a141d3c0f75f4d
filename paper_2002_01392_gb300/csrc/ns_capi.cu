// Navier-Stokes entry points of the C ABI (GPU backend of NsCore).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

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
  int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 1;
  }
  // duration of the launches made by f on stream st (synchronous)
  template <class F>
  fc_status time_ms(F&& f, void* st, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fc_status s = cuda_status(cudaEventCreate(&e0), "cudaEventCreate");
    if (!s) s = cuda_status(cudaEventCreate(&e1), "cudaEventCreate");
    if (!s) s = cuda_status(cudaEventRecord(e0, (cudaStream_t)st), "cudaEventRecord");
    if (!s) s = f();
    if (!s) s = cuda_status(cudaEventRecord(e1, (cudaStream_t)st), "cudaEventRecord");
    if (!s) s = cuda_status(cudaEventSynchronize(e1), "cudaEventSynchronize");
    if (!s) s = cuda_status(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return s;
  }
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
  // non-finite check after every check_every-th step: the device counter
  // (workspace) is copied into the pinned host word hflag after the count,
  // and later calls read hflag without synchronising
  int check_every = 0;
  long long nsteps = 0;
  unsigned long long* hflag = nullptr;
  // diagnostic series: after every diag_every-th rk_step the diagnostic sums
  // of the new state go to the next device slot; diag_at[i] = its step number
  int diag_every = 0;
  long long diag_steps = 0;
  std::vector<long long> diag_at;
};

// ns_diagnostics' normalisation of the six device sums
static void diag_scale(const ns_params& p, const double* acc, double* out5) {
  const double n2 = (double)p.Nx * p.Ny * (double)p.Nx * p.Ny;
  out5[0] = acc[0] / n2 / p.Nz;
  out5[1] = acc[1] / n2 / 2.0;
  out5[2] = acc[2] / n2 / 2.0;
  out5[3] = acc[3] / ((double)p.Nx * p.Ny) / p.Nz;
  if (p.nfields == 4 && p.gamma != 0.0) {
    const double m0 = acc[4] / ((double)p.Nx * p.Ny), m1 = acc[5] / ((double)p.Nx * p.Ny);
    out5[4] = 0.5 * ((1.0 - m0 / p.gamma) + (1.0 - m1 / p.gamma));
  } else {
    out5[4] = 0.0;
  }
}

static fc_status check_enqueue(ns_sim* s, cudaStream_t st) {
  fc_status r = s->core.count_nonfinite_any(false, st);
  if (!r) r = cuda_status(cudaMemcpyAsync(s->hflag, s->core.ws + s->core.l.nfin, sizeof(unsigned long long),
                                          cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync(non-finite flag)");
  return r;
}

static fc_status check_flag(ns_sim* s, const char* what) {
  if (s->check_every <= 0 || !s->hflag) return FC_OK;
  const unsigned long long n = *static_cast<volatile unsigned long long*>(s->hflag);
  if (!n) return FC_OK;
  set_error(std::string(what) + ": a checked step left " + std::to_string(n) + " non-finite state values");
  return FC_ERR_NONFINITE;
}

// A set of simulations whose RK steps are replayed from captured CUDA graphs.
// Members are spread over NB capture branches (fork / join on events), so
// independent instances run concurrently inside one graph launch.  A graph
// depends on the members' buffer rotation (NsCore::cur) and on the step
// sizes, which form the cache key.
struct ns_batch {
  static constexpr int NB = 8;
  std::vector<ns_sim_t> sims;
  int device = -1;
  cudaStream_t cap = nullptr;
  cudaStream_t br[NB] = {};
  cudaEvent_t fork = nullptr, join[NB] = {};
  struct Entry {
    std::vector<int> cur_in, cur_out;
    std::vector<double> dt;
    std::vector<char> chk;   // members checked for non-finite values after the step
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Entry> cache;
  int launches_per_graph = 0;
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
  if (fc_status inj = injected("ns_create")) return inj;
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
  if (s->hflag) cudaFreeHost(s->hflag);
  delete s;
  return st;
}

fc_status ns_set_fields(ns_sim_t s, const void* phys, fc_stream_t stream) {
  if (fc_status inj = injected("ns_set_fields")) return inj;
  fc_status st = check_sim(s, "ns_set_fields");
  if (st) return st;
  if (!phys) { set_error("ns_set_fields: NULL fields"); return FC_ERR_ARG; }
  return s->core.set_fields_any(phys, stream);
}

fc_status ns_get_fields(ns_sim_t s, void* phys, fc_stream_t stream) {
  if (fc_status inj = injected("ns_get_fields")) return inj;
  fc_status st = check_sim(s, "ns_get_fields");
  if (st) return st;
  if (!phys) { set_error("ns_get_fields: NULL fields"); return FC_ERR_ARG; }
  return s->core.get_fields_any(phys, stream);
}

fc_status ns_get_state(ns_sim_t s, void* spec, fc_stream_t stream) {
  if (fc_status inj = injected("ns_get_state")) return inj;
  fc_status st = check_sim(s, "ns_get_state");
  if (st) return st;
  if (!spec) return FC_ERR_ARG;
  return s->core.bk.d2d(spec, s->core.ws + s->core.l.X[s->core.cur], s->core.state_bytes(), stream);
}

fc_status ns_put_state(ns_sim_t s, const void* spec, fc_stream_t stream) {
  if (fc_status inj = injected("ns_put_state")) return inj;
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
  if (fc_status inj = injected("ns_rhs")) return inj;
  fc_status st = check_sim(s, "ns_rhs");
  if (st) return st;
  if (!phys_in || !rhs_out || phys_in == rhs_out) { set_error("ns_rhs: bad buffers"); return FC_ERR_ARG; }
  return s->core.rhs_any(phys_in, rhs_out, stream);
}

fc_status fc_poisson_project(ns_sim_t s, double dt_stage, const void* vstar_phys, void* v_phys, void* gradp_wall,
                             fc_stream_t stream) {
  if (fc_status inj = injected("fc_poisson_project")) return inj;
  fc_status st = check_sim(s, "fc_poisson_project");
  if (st) return st;
  if (!vstar_phys || !v_phys || !(dt_stage > 0)) { set_error("fc_poisson_project: bad arguments"); return FC_ERR_ARG; }
  return s->core.project_any(dt_stage, vstar_phys, v_phys, gradp_wall, stream);
}

fc_status rk_step(ns_sim_t s, double dt, fc_stream_t stream) {
  fc_status st = injected("rk_step");
  if (!st) st = check_sim(s, "rk_step");
  if (st) return st;
  if (!(dt > 0)) { set_error("rk_step: dt must be positive"); return FC_ERR_ARG; }
  st = check_flag(s, "rk_step");
  if (!st) st = s->core.step_any(dt, stream);
  if (!st && s->check_every > 0 && ++s->nsteps % s->check_every == 0) st = check_enqueue(s, (cudaStream_t)stream);
  if (!st && s->diag_every > 0 && ++s->diag_steps % s->diag_every == 0 && (int)s->diag_at.size() < NS_DIAG_SLOTS) {
    st = s->core.diag_record_any((int)s->diag_at.size(), stream);
    if (!st) s->diag_at.push_back(s->diag_steps);
  }
  return st;
}

fc_status ns_set_diag_series(ns_sim_t s, int every) {
  fc_status st = check_sim(s, "ns_set_diag_series");
  if (st) return st;
  if (every < 0) { set_error("ns_set_diag_series: every must be >= 0"); return FC_ERR_ARG; }
  s->diag_every = every;
  s->diag_steps = 0;
  s->diag_at.clear();
  return FC_OK;
}

fc_status ns_get_diag_series(ns_sim_t s, int max, double* values, long long* steps, int* count, fc_stream_t stream) {
  fc_status st = check_sim(s, "ns_get_diag_series");
  if (st) return st;
  if (max < 0 || (max > 0 && !values)) { set_error("ns_get_diag_series: max >= 0 and values non-NULL"); return FC_ERR_ARG; }
  const int n = std::min(max, (int)s->diag_at.size());
  if (count) *count = (int)s->diag_at.size();
  if (n == 0) return FC_OK;
  std::vector<double> acc(8 * (size_t)n);
  st = cuda_status(cudaMemcpyAsync(acc.data(), s->core.ws + s->core.l.dser, sizeof(double) * acc.size(),
                                   cudaMemcpyDeviceToHost, (cudaStream_t)stream), "cudaMemcpyAsync(diagnostic series)");
  if (!st) st = cuda_status(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    diag_scale(s->core.p, &acc[8 * (size_t)i], values + 5 * (size_t)i);
    if (steps) steps[i] = s->diag_at[i];
  }
  return FC_OK;
}

fc_status ns_set_finite_check(ns_sim_t s, int every) {
  fc_status st = check_sim(s, "ns_set_finite_check");
  if (st) return st;
  if (every < 0) { set_error("ns_set_finite_check: every must be >= 0"); return FC_ERR_ARG; }
  if (every > 0 && !s->hflag) {
    void* h = nullptr;
    st = cuda_status(cudaHostAlloc(&h, sizeof(unsigned long long), cudaHostAllocDefault), "cudaHostAlloc");
    if (st) return st;
    s->hflag = static_cast<unsigned long long*>(h);
    *s->hflag = 0;
  }
  s->check_every = every;
  s->nsteps = 0;
  return FC_OK;
}

fc_status ns_check_finite(ns_sim_t s, long long* count, fc_stream_t stream) {
  fc_status st = injected("ns_check_finite");
  if (!st) st = check_sim(s, "ns_check_finite");
  if (st) return st;
  if (!count) { set_error("ns_check_finite: NULL count"); return FC_ERR_ARG; }
  unsigned long long n = 0;
  st = s->core.count_nonfinite_any(true, stream);
  if (!st) st = s->core.bk.d2h(&n, s->core.ws + s->core.l.nfin, sizeof(n), stream);
  if (st) return st;
  if (s->hflag) *static_cast<volatile unsigned long long*>(s->hflag) = n;
  *count = (long long)n;
  if (n) {
    set_error("ns_check_finite: " + std::to_string(n) + " non-finite state values");
    return FC_ERR_NONFINITE;
  }
  return FC_OK;
}

fc_status fc_count_nonfinite(fc_dtype dtype, const void* data, long long n, long long* count, fc_stream_t stream) {
  fc_status st = injected("fc_count_nonfinite");
  if (st) return st;
  if (!count || n < 0 || (n > 0 && !data) || (dtype != FC_F32 && dtype != FC_F64)) {
    set_error("fc_count_nonfinite: bad arguments");
    return FC_ERR_ARG;
  }
  *count = 0;
  if (n == 0) return FC_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  unsigned long long* dc = nullptr;
  st = cuda_status(cudaMallocAsync((void**)&dc, sizeof(unsigned long long), cs), "cudaMallocAsync");
  if (st) return st;
  st = cuda_status(cudaMemsetAsync(dc, 0, sizeof(unsigned long long), cs), "cudaMemsetAsync");
  const long long per = 256 * 64;
  const long long grid = (n + per - 1) / per;
  if (!st) {
    if (dtype == FC_F32) {
      KCount<float>::Args a{static_cast<const float*>(data), n, per, dc};
      st = DevRun<KCount<float>>::run(a, grid, cs);
    } else {
      KCount<double>::Args a{static_cast<const double*>(data), n, per, dc};
      st = DevRun<KCount<double>>::run(a, grid, cs);
    }
  }
  unsigned long long h = 0;
  if (!st) st = cuda_status(cudaMemcpyAsync(&h, dc, sizeof(h), cudaMemcpyDeviceToHost, cs), "cudaMemcpyAsync(D2H)");
  cudaFreeAsync(dc, cs);
  if (!st) st = cuda_status(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
  if (st) return st;
  *count = (long long)h;
  if (h) {
    set_error("fc_count_nonfinite: " + std::to_string(h) + " non-finite values");
    return FC_ERR_NONFINITE;
  }
  return FC_OK;
}

fc_status ns_spectrum_shells(ns_sim_t s, int* nshell, double* dk) {
  fc_status st = check_sim(s, "ns_spectrum_shells");
  if (st) return st;
  if (nshell) *nshell = s->core.nshell();
  if (dk) *dk = s->core.shell_width();
  return FC_OK;
}

fc_status ns_profiles(ns_sim_t s, double* mean, double* rms, double* spectrum, fc_stream_t stream) {
  if (fc_status inj = injected("ns_profiles")) return inj;
  fc_status st = check_sim(s, "ns_profiles");
  if (st) return st;
  const ns_params& p = s->core.p;
  const int nf = p.nfields, Nz = p.Nz, ns = s->core.nshell();
  std::vector<double> raw((size_t)nf * Nz * (2 + ns));
  st = s->core.profiles_any(raw.data(), stream);
  if (st) return st;
  const double n1 = (double)p.Nx * p.Ny, n2 = n1 * n1;
  if (spectrum) std::memset(spectrum, 0, sizeof(double) * nf * ns);
  for (int f = 0; f < nf; ++f)
    for (int z = 0; z < Nz; ++z) {
      const double* r = raw.data() + ((size_t)f * Nz + z) * (2 + ns);
      if (mean) mean[(size_t)f * Nz + z] = r[1] / n1;
      if (rms) rms[(size_t)f * Nz + z] = std::sqrt(r[0] / n2);
      if (spectrum) {
        const double wz = (z == 0 || z == Nz - 1) ? 0.5 / (Nz - 1) : 1.0 / (Nz - 1);  // trapezoid, / Lz
        for (int j = 0; j < ns; ++j) spectrum[(size_t)f * ns + j] += wz * r[2 + j] / n2;
      }
    }
  return FC_OK;
}

fc_status ns_interpolate(ns_sim_t dst, ns_sim_t src, fc_stream_t stream) {
  if (fc_status inj = injected("ns_interpolate")) return inj;
  fc_status st = check_sim(dst, "ns_interpolate");
  if (!st) st = check_sim(src, "ns_interpolate");
  if (st) return st;
  if (dst == src) { set_error("ns_interpolate: source and destination are the same"); return FC_ERR_ARG; }
  st = dst->core.interpolate_from_any(src->core, stream);
  if (st == FC_ERR_ARG) set_error("ns_interpolate: grids not compatible (finer Nx, Ny; same box, fields, precision)");
  return st;
}

fc_status ns_tune(ns_sim_t s, int mode, int* tiles, fc_stream_t stream) {
  if (fc_status inj = injected("ns_tune")) return inj;
  fc_status st = check_sim(s, "ns_tune");
  if (st) return st;
  auto& c = s->core;
  if (mode == 0) {
    for (int k = 0; k < c.TK_N; ++k) c.tile[k] = 0;
  } else if (mode == 1) {
    st = c.autotune_any(stream);
  } else if (mode == 2) {
    if (!tiles) { set_error("ns_tune: NULL tiles"); return FC_ERR_ARG; }
    for (int k = 0; k < c.TK_N; ++k) c.tile[k] = tiles[k] & c.variant_mask(k);
  } else {
    set_error("ns_tune: mode must be 0, 1 or 2");
    return FC_ERR_ARG;
  }
  if (!st && tiles)
    for (int k = 0; k < c.TK_N; ++k) tiles[k] = c.tile[k];
  return st;
}

fc_status ns_batch_create(ns_sim_t* sims, int n, ns_batch_t* out) {
  if (fc_status inj = injected("ns_batch_create")) return inj;
  if (!sims || !out || n < 1) { set_error("ns_batch_create: bad arguments"); return FC_ERR_ARG; }
  *out = nullptr;
  int dev = -1;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i) {
    if (!sims[i]) { set_error("ns_batch_create: NULL member"); return FC_ERR_ARG; }
    if (sims[i]->device != dev) { set_error("ns_batch_create: members on another device"); return FC_ERR_STATE; }
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) { set_error("ns_batch_create: a simulation appears twice"); return FC_ERR_ARG; }
  }
  for (int i = 0; i < n; ++i) {  // kernel variants of every member picked by measurement (cached per size)
    fc_status t = sims[i]->core.autotune_any(nullptr);
    if (t) return t;
  }
  ns_batch* b = new (std::nothrow) ns_batch;
  if (!b) return FC_ERR_NOMEM;
  b->sims.assign(sims, sims + n);
  b->device = dev;
  fc_status st = cuda_status(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
  for (int i = 0; i < ns_batch::NB && !st; ++i) {
    st = cuda_status(cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking), "cudaStreamCreate");
    if (!st) st = cuda_status(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming), "cudaEventCreate");
  }
  if (!st) st = cuda_status(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "cudaEventCreate");
  if (st) { ns_batch_destroy(b); return st; }
  *out = b;
  return FC_OK;
}

fc_status ns_batch_destroy(ns_batch_t b) {
  if (!b) return FC_ERR_ARG;
  for (auto& e : b->cache)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  for (int i = 0; i < ns_batch::NB; ++i) {
    if (b->br[i]) cudaStreamDestroy(b->br[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return FC_OK;
}

// Capture one RK step of every member (step sizes dt) into a graph.
static fc_status batch_capture(ns_batch_t b, const double* dt, ns_batch::Entry* e) {
  const int n = (int)b->sims.size();
  e->cur_in.resize(n);
  e->dt.assign(dt, dt + n);
  for (int i = 0; i < n; ++i) e->cur_in[i] = b->sims[i]->core.cur;
  fc_status st = cuda_status(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (st) return st;
  st = cuda_status(cudaEventRecord(b->fork, b->cap), "cudaEventRecord");
  const int nb = n < ns_batch::NB ? n : ns_batch::NB;
  for (int k = 0; k < nb && !st; ++k) st = cuda_status(cudaStreamWaitEvent(b->br[k], b->fork, 0), "cudaStreamWaitEvent");
  e->chk.resize(n);
  for (int i = 0; i < n && !st; ++i) {
    ns_sim* m = b->sims[i];
    e->chk[i] = m->check_every > 0;
    st = m->core.step_any(dt[i], b->br[i % nb]);
    if (!st && e->chk[i]) st = check_enqueue(m, b->br[i % nb]);
  }
  for (int k = 0; k < nb && !st; ++k) {
    st = cuda_status(cudaEventRecord(b->join[k], b->br[k]), "cudaEventRecord");
    if (!st) st = cuda_status(cudaStreamWaitEvent(b->cap, b->join[k], 0), "cudaStreamWaitEvent");
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
  if (!st) st = cuda_status(ec, "cudaStreamEndCapture");
  e->cur_out.resize(n);
  for (int i = 0; i < n; ++i) {  // capture ran the host side of step(): keep its rotation, undo it for now
    e->cur_out[i] = b->sims[i]->core.cur;
    b->sims[i]->core.cur = e->cur_in[i];
  }
  if (!st) {
    size_t nodes = 0;
    cudaGraphGetNodes(g, nullptr, &nodes);
    b->launches_per_graph = (int)nodes;
    st = cuda_status(cudaGraphInstantiate(&e->exec, g, 0), "cudaGraphInstantiate");
  }
  if (g) cudaGraphDestroy(g);
  return st;
}

fc_status ns_batch_step(ns_batch_t b, const double* dt, fc_stream_t stream) {
  if (fc_status inj = injected("ns_batch_step")) return inj;
  if (!b || !dt) { set_error("ns_batch_step: NULL argument"); return FC_ERR_ARG; }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) {
    set_error("ns_batch_step: called with a different current device than ns_batch_create");
    return FC_ERR_STATE;
  }
  const int n = (int)b->sims.size();
  for (int i = 0; i < n; ++i)
    if (!(dt[i] > 0)) { set_error("ns_batch_step: dt must be positive"); return FC_ERR_ARG; }
  for (int i = 0; i < n; ++i)
    if (b->sims[i]->check_every > 0) {
      fc_status c = check_flag(b->sims[i], ("ns_batch_step: member " + std::to_string(i)).c_str());
      if (c) return c;
    }
  ns_batch::Entry* hit = nullptr;
  for (auto& e : b->cache) {
    bool same = true;
    for (int i = 0; i < n && same; ++i)
      same = e.cur_in[i] == b->sims[i]->core.cur && e.dt[i] == dt[i] && e.chk[i] == (b->sims[i]->check_every > 0);
    if (same) { hit = &e; break; }
  }
  if (!hit) {
    if (b->cache.size() >= 6) {  // a new set of step sizes: drop the old graphs
      for (auto& e : b->cache) cudaGraphExecDestroy(e.exec);
      b->cache.clear();
    }
    ns_batch::Entry e;
    fc_status st = batch_capture(b, dt, &e);
    if (st) {
      if (e.exec) cudaGraphExecDestroy(e.exec);
      return st;
    }
    b->cache.push_back(e);
    hit = &b->cache.back();
  }
  fc_status st = cuda_status(cudaGraphLaunch(hit->exec, (cudaStream_t)stream), "cudaGraphLaunch");
  if (st) return st;
  for (int i = 0; i < n; ++i) b->sims[i]->core.cur = hit->cur_out[i];
  return FC_OK;
}

fc_status ns_batch_info(ns_batch_t b, int* members, int* graph_nodes, int* graphs_cached) {
  if (!b) return FC_ERR_ARG;
  if (members) *members = (int)b->sims.size();
  if (graph_nodes) *graph_nodes = b->launches_per_graph;
  if (graphs_cached) *graphs_cached = (int)b->cache.size();
  return FC_OK;
}

fc_status ns_diagnostics(ns_sim_t s, double* div_ms, double* wall_u_ms, double* wall_w_ms, double* flow_rate,
                         double* nusselt, fc_stream_t stream) {
  if (fc_status inj = injected("ns_diagnostics")) return inj;
  fc_status st = check_sim(s, "ns_diagnostics");
  if (st) return st;
  double acc[6];
  st = s->core.diagnostics_any(acc, stream);
  if (st) return st;
  double v[5];
  diag_scale(s->core.p, acc, v);
  if (div_ms) *div_ms = v[0];
  if (wall_u_ms) *wall_u_ms = v[1];
  if (wall_w_ms) *wall_w_ms = v[2];
  if (flow_rate) *flow_rate = v[3];
  if (nusselt) *nusselt = v[4];
  return FC_OK;
}

}  // extern "C"
