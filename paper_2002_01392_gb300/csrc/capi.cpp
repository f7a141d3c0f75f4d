// C ABI of libfcns: argument validation, plan objects, dispatch to launchers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "host_tables.hpp"
#include "slabs.hpp"
#include "internal.hpp"

namespace fcns {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

fc_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FC_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FC_ERR_NOMEM : FC_ERR_CUDA;
}

// Failure injection (tests of callers' error handling; nothing reaches the
// GPU): rules "entry:status:skip:count" from fc_inject_failure or from the
// FCNS_INJECT environment variable (comma-separated rules, read on the first
// check).  A rule lets `skip` calls of its entry point through, then fails
// the next `count` calls (count < 0: every later call); entry "*" matches
// every entry point that checks.
namespace {
struct InjectRule {
  std::string entry;
  fc_status status;
  long long skip, count;
};
std::mutex g_inj_mtx;
std::vector<InjectRule> g_inj;
std::atomic<int> g_inj_state{-1};  // -1: environment not read; 0: no rules; 1: rules armed

bool parse_status(const std::string& t, fc_status* out) {
  static const char* names[] = {"FC_OK", "FC_ERR_ARG", "FC_ERR_UNSUPPORTED", "FC_ERR_CUDA",
                                "FC_ERR_NOMEM", "FC_ERR_TIMEOUT", "FC_ERR_NONFINITE", "FC_ERR_STATE"};
  for (int i = 1; i < 8; ++i)
    if (t == names[i] || t == std::to_string(i)) { *out = (fc_status)i; return true; }
  return false;
}

// caller holds g_inj_mtx
void read_env_rules() {
  const char* env = std::getenv("FCNS_INJECT");
  std::string all = env ? env : "";
  size_t pos = 0;
  while (pos < all.size()) {
    size_t end = all.find(',', pos);
    if (end == std::string::npos) end = all.size();
    std::string rule = all.substr(pos, end - pos), f[4];
    pos = end + 1;
    int k = 0;
    size_t q = 0;
    while (k < 4) {
      size_t c = rule.find(':', q);
      f[k++] = rule.substr(q, c == std::string::npos ? std::string::npos : c - q);
      if (c == std::string::npos) break;
      q = c + 1;
    }
    fc_status st;
    if (f[0].empty() || !parse_status(f[1], &st)) continue;
    g_inj.push_back({f[0], st, f[2].empty() ? 0 : std::atoll(f[2].c_str()), f[3].empty() ? 1 : std::atoll(f[3].c_str())});
  }
  g_inj_state.store(g_inj.empty() ? 0 : 1);
}
}  // namespace

fc_status injected(const char* entry) {
  if (g_inj_state.load(std::memory_order_acquire) == 0) return FC_OK;
  std::lock_guard<std::mutex> lk(g_inj_mtx);
  if (g_inj_state.load() < 0) read_env_rules();
  fc_status out = FC_OK;
  for (auto& r : g_inj) {
    if (r.entry != "*" && r.entry != entry) continue;
    if (r.skip > 0) { --r.skip; continue; }
    if (r.count == 0) continue;
    if (r.count > 0) --r.count;
    out = r.status;
    break;
  }
  std::vector<InjectRule> live;
  for (auto& r : g_inj)
    if (r.count != 0) live.push_back(r);
  g_inj.swap(live);
  g_inj_state.store(g_inj.empty() ? 0 : 1);
  if (out) set_error(std::string(entry) + ": injected failure");
  return out;
}

}  // namespace fcns

using namespace fcns;

extern "C" {

const char* fc_status_str(fc_status s) {
  switch (s) {
    case FC_OK: return "FC_OK";
    case FC_ERR_ARG: return "FC_ERR_ARG";
    case FC_ERR_UNSUPPORTED: return "FC_ERR_UNSUPPORTED";
    case FC_ERR_CUDA: return "FC_ERR_CUDA";
    case FC_ERR_NOMEM: return "FC_ERR_NOMEM";
    case FC_ERR_TIMEOUT: return "FC_ERR_TIMEOUT";
    case FC_ERR_NONFINITE: return "FC_ERR_NONFINITE";
    case FC_ERR_STATE: return "FC_ERR_STATE";
  }
  return "FC_ERR_UNKNOWN";
}

const char* fc_last_error(void) { return g_last_error.c_str(); }

fc_status fc_inject_failure(const char* entry, fc_status status, long long skip, long long count) {
  std::lock_guard<std::mutex> lk(g_inj_mtx);
  if (g_inj_state.load() < 0) read_env_rules();
  if (!entry) {
    g_inj.clear();
    g_inj_state.store(0);
    return FC_OK;
  }
  if (status == FC_OK || (int)status < 0 || (int)status > 7 || skip < 0 || count == 0) {
    set_error("fc_inject_failure: status must be an error code, skip >= 0 and count != 0");
    return FC_ERR_ARG;
  }
  g_inj.push_back({entry, status, skip, count});
  g_inj_state.store(1);
  return FC_OK;
}

fc_status fc_setup_ex(int d, int C, int Nz, int M, int n_os, fc_plan_t* out) {
  if (fc_status inj = injected("fc_setup")) return inj;
  if (!out) { set_error("fc_setup: out is NULL"); return FC_ERR_ARG; }
  *out = nullptr;
  if (d < 2 || d > 10 || C < d || C > 64 || Nz < 2 * d || M < 1 || n_os < 1 || 2 * M + 1 > 2 * ((d - 1) * n_os + 1)) {
    set_error("fc_setup: invalid d, C, Nz, M or n_os");
    return FC_ERR_ARG;
  }
  fc_plan* p = new (std::nothrow) fc_plan;
  if (!p) return FC_ERR_NOMEM;
  static std::atomic<unsigned long long> next_serial{1};
  p->deriv.serial = next_serial.fetch_add(1);
  FcTables T;
  if (!build_fc_tables(d, C, M, n_os, &T)) { delete p; set_error("fc_setup: table construction failed"); return FC_ERR_ARG; }
  p->data.d = d; p->data.C = C; p->data.Nz = Nz; p->data.Np = Nz + C;
  p->data.M = M; p->data.n_os = n_os; p->data.ls_residual = T.ls_residual;
  // per-device tables are handed out by address and used outside the plan's
  // lock: the vector never reallocates (one entry per device, at most 64)
  p->data.dev.reserve(64);
  p->data.Mr = T.Mr;
  // transform length: N' itself when it is one of the compiled (smooth)
  // lengths -- the paper's choice of N' (Sec. 6, Sec. 7 tables) -- else the
  // padded circular-convolution length L >= N' + Nz - 1
  int L = 0;
  for (auto& sh : engine_shapes())
    if (sh.L == p->data.Np) L = sh.L;
  if (!L) L = pick_engine_length(p->data.Np + Nz - 1);
  if (L > 0) {
    for (auto& s : engine_shapes())
      if (s.L == L) { p->deriv.L = L; p->deriv.L1 = s.L1; p->deriv.L2 = s.L2; }
    engine_twiddles(p->deriv.L1, p->deriv.L2, &p->deriv.tw);
    auto& t = p->deriv;
    std::vector<std::complex<double>> H1, H2;
    deriv_conv_spectra(Nz, p->data.Np, L, &H1, &H2);
    t.H1_32.resize(L); t.H2_32.resize(L); t.H1_64.resize(L); t.H2_64.resize(L);
    for (int i = 0; i < L; ++i) {
      t.H1_32[i] = make_float2((float)H1[i].real(), (float)H1[i].imag());
      t.H2_32[i] = make_float2((float)H2[i].real(), (float)H2[i].imag());
      t.H1_64[i] = make_double2(H1[i].real(), H1[i].imag());
      t.H2_64[i] = make_double2(H2[i].real(), H2[i].imag());
    }
    t.tw32.resize(2 * L); t.tw64.resize(2 * L);
    for (int i = 0; i < 2 * L; ++i) {
      t.tw32[i] = make_float2((float)t.tw[i].real(), (float)t.tw[i].imag());
      t.tw64[i] = make_double2(t.tw[i].real(), t.tw[i].imag());
    }
  }
  p->deriv.Mr2.resize(p->data.Mr.size());
  for (size_t i = 0; i < p->data.Mr.size(); ++i) {
    const float hi = (float)p->data.Mr[i];
    p->deriv.Mr2[i] = make_float2(hi, (float)(p->data.Mr[i] - (double)hi));
  }
  *out = p;
  return FC_OK;
}

fc_status fc_setup(int d, int C, int Nz, fc_plan_t* out) {
  return fc_setup_ex(d, C, Nz, (2 * (d + C)) / 3, 20, out);
}

fc_status fc_plan_matrix(fc_plan_t plan, double* Mr_out) {
  if (!plan || !Mr_out) { set_error("fc_plan_matrix: NULL argument"); return FC_ERR_ARG; }
  std::memcpy(Mr_out, plan->data.Mr.data(), sizeof(double) * plan->data.Mr.size());
  return FC_OK;
}

fc_status fc_plan_info(fc_plan_t plan, int* d, int* C, int* Nz, int* M, int* n_os, double* ls_residual) {
  if (!plan) { set_error("fc_plan_info: NULL plan"); return FC_ERR_ARG; }
  if (d) *d = plan->data.d;
  if (C) *C = plan->data.C;
  if (Nz) *Nz = plan->data.Nz;
  if (M) *M = plan->data.M;
  if (n_os) *n_os = plan->data.n_os;
  if (ls_residual) *ls_residual = plan->data.ls_residual;
  return FC_OK;
}

fc_status fc_destroy(fc_plan_t plan) {
  if (!plan) return FC_ERR_ARG;
  int cur = -1;
  if (!plan->data.dev.empty() && cudaGetDevice(&cur) == cudaSuccess) {
    for (auto& t : plan->data.dev) {
      cudaSetDevice(t.device);
      cudaDeviceSynchronize();
      cudaFree(t.Mr); cudaFree(t.Mr2); cudaFree(t.tw32); cudaFree(t.tw64);
      cudaFree(t.H1_32); cudaFree(t.H1_64); cudaFree(t.H2_32); cudaFree(t.H2_64);
      for (auto& slot : t.stage)
        for (void* b : slot) cudaFree(b);
      for (int k = 0; k < 3; ++k) {
        if (t.ev_in[k]) cudaEventDestroy(t.ev_in[k]);
        if (t.ev_run[k]) cudaEventDestroy(t.ev_run[k]);
        if (t.ev_out[k]) cudaEventDestroy(t.ev_out[k]);
      }
      if (t.st_in) cudaStreamDestroy(t.st_in);
      if (t.st_run) cudaStreamDestroy(t.st_run);
      if (t.st_out) cudaStreamDestroy(t.st_out);
    }
    cudaSetDevice(cur);
  }
  delete plan;
  return FC_OK;
}

}  // extern "C"

namespace fcns {

template <class C>
static fc_status upload(const std::vector<std::complex<double>>& v, void** dst) {
  std::vector<C> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) { h[i].x = (decltype(h[i].x))v[i].real(); h[i].y = (decltype(h[i].y))v[i].imag(); }
  fc_status s = cuda_status(cudaMalloc(dst, sizeof(C) * h.size()), "cudaMalloc(tables)");
  if (s) return s;
  return cuda_status(cudaMemcpy(*dst, h.data(), sizeof(C) * h.size(), cudaMemcpyHostToDevice), "cudaMemcpy(tables)");
}

static fc_status deriv_tables_locked(fc_plan* plan, DerivDevTables** out) {
  int dev = -1;
  fc_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (s) return s;
  for (auto& t : plan->data.dev)
    if (t.device == dev) { *out = &t; return FC_OK; }
  if (plan->data.dev.size() >= plan->data.dev.capacity()) {
    set_error("fc_deriv_z: more devices than the plan supports (64)");
    return FC_ERR_UNSUPPORTED;
  }
  DerivDevTables t;
  t.device = dev;
  t.L = plan->deriv.L;
  s = cuda_status(cudaMalloc((void**)&t.Mr, sizeof(double) * plan->data.Mr.size()), "cudaMalloc(Mr)");
  if (!s) s = cuda_status(cudaMemcpy(t.Mr, plan->data.Mr.data(), sizeof(double) * plan->data.Mr.size(),
                                     cudaMemcpyHostToDevice), "cudaMemcpy(Mr)");
  if (!s) s = cuda_status(cudaMalloc((void**)&t.Mr2, sizeof(float2) * plan->deriv.Mr2.size()), "cudaMalloc(Mr2)");
  if (!s) s = cuda_status(cudaMemcpy(t.Mr2, plan->deriv.Mr2.data(), sizeof(float2) * plan->deriv.Mr2.size(),
                                     cudaMemcpyHostToDevice), "cudaMemcpy(Mr2)");
  auto up = [&](const void* src, size_t bytes, void** dst) {
    fc_status st = cuda_status(cudaMalloc(dst, bytes), "cudaMalloc(tables)");
    if (!st) st = cuda_status(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "cudaMemcpy(tables)");
    return st;
  };
  const size_t L = plan->deriv.L;
  if (!s) s = up(plan->deriv.H1_32.data(), 8 * L, &t.H1_32);
  if (!s) s = up(plan->deriv.H2_32.data(), 8 * L, &t.H2_32);
  if (!s) s = up(plan->deriv.H1_64.data(), 16 * L, &t.H1_64);
  if (!s) s = up(plan->deriv.H2_64.data(), 16 * L, &t.H2_64);
  if (!s) s = upload<float2>(plan->deriv.tw, &t.tw32);
  if (!s) s = upload<double2>(plan->deriv.tw, &t.tw64);
  if (s) {
    cudaFree(t.Mr); cudaFree(t.Mr2); cudaFree(t.tw32); cudaFree(t.tw64);
      cudaFree(t.H1_32); cudaFree(t.H1_64); cudaFree(t.H2_32); cudaFree(t.H2_64);
    return s;
  }
  plan->data.dev.push_back(t);
  *out = &plan->data.dev.back();
  return FC_OK;
}

}  // namespace fcns

fc_status fcns::check_deriv_args(const PlanData& pd, const PlanHostTables& t, fc_dtype dtype, int batch, int Nx,
                                 int Ny, double Lz, const void* f, void* df, void* d2f, const char* who) {
  std::string w(who);
  if (!f || (!df && !d2f)) { set_error(w + ": NULL input or both outputs"); return FC_ERR_ARG; }
  if (dtype != FC_F32 && dtype != FC_F64) { set_error(w + ": bad dtype"); return FC_ERR_ARG; }
  if (batch < 1 || Nx < 1 || Ny < 1 || !(Lz > 0) || !std::isfinite(Lz)) { set_error(w + ": bad sizes"); return FC_ERR_ARG; }
  const long long lines = (long long)Nx * Ny;
  if (lines * batch >= (1LL << 31)) { set_error(w + ": too many lines"); return FC_ERR_UNSUPPORTED; }
  if (t.L == 0) { set_error(w + ": N' + Nz - 1 exceeds the compiled transform lengths"); return FC_ERR_UNSUPPORTED; }
  const size_t es = dtype == FC_F32 ? 4 : 8;
  const size_t bytes = es * (size_t)lines * pd.Nz * batch;
  auto overlap = [&](const void* a, const void* b) {
    if (!a || !b) return false;
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + bytes && y < x + bytes;
  };
  if (overlap(f, df) || overlap(f, d2f) || overlap(df, d2f)) { set_error(w + ": overlapping buffers"); return FC_ERR_ARG; }
  return FC_OK;
}

extern "C" fc_status fc_deriv_z(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                                const void* f, void* df, void* d2f, fc_stream_t stream) {
  if (fc_status inj = injected("fc_deriv_z")) return inj;
  if (!plan) { set_error("fc_deriv_z: NULL plan"); return FC_ERR_ARG; }
  fc_status s = check_deriv_args(plan->data, plan->deriv, dtype, batch, Nx, Ny, Lz, f, df, d2f, "fc_deriv_z");
  if (s) return s;
  DerivDevTables* t = nullptr;
  {
    std::lock_guard<std::mutex> lk(plan->data.mtx);
    s = deriv_tables_locked(plan, &t);
  }
  if (s) return s;
  return launch_deriv_z(*t, plan->data, dtype, batch, (long long)Nx * Ny, Lz, f, df, d2f, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// fc_deriv_z on host arrays: slabs of y rows (all z, all x) are copied in,
// differentiated and copied out on three streams, so that the copies of one
// slab overlap the kernel of another and the two copy directions overlap
// each other.
// ---------------------------------------------------------------------------
static fc_status stage_for(DerivDevTables* t, size_t bytes) {
  fc_status s = FC_OK;
  if (!t->st_in) {
    s = cuda_status(cudaStreamCreateWithFlags(&t->st_in, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!s) s = cuda_status(cudaStreamCreateWithFlags(&t->st_run, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!s) s = cuda_status(cudaStreamCreateWithFlags(&t->st_out, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int k = 0; k < 3 && !s; ++k) {
      s = cuda_status(cudaEventCreateWithFlags(&t->ev_in[k], cudaEventDisableTiming), "cudaEventCreate");
      if (!s) s = cuda_status(cudaEventCreateWithFlags(&t->ev_run[k], cudaEventDisableTiming), "cudaEventCreate");
      if (!s) s = cuda_status(cudaEventCreateWithFlags(&t->ev_out[k], cudaEventDisableTiming), "cudaEventCreate");
    }
    if (s) return s;
  }
  if (t->stage_bytes >= bytes) return FC_OK;
  for (auto& slot : t->stage)
    for (void*& b : slot) {
      cudaFree(b);
      b = nullptr;
    }
  t->stage_bytes = 0;
  for (auto& slot : t->stage)
    for (void*& b : slot) {
      s = cuda_status(cudaMalloc(&b, bytes), "cudaMalloc(fc_deriv_z_host staging)");
      if (s) return s;
    }
  t->stage_bytes = bytes;
  return FC_OK;
}

extern "C" fc_status fc_deriv_z_host_ex(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                                        const void* f, void* df, void* d2f, size_t slab_bytes, fc_stream_t stream) {
  if (fc_status inj = injected("fc_deriv_z_host")) return inj;
  if (!plan) { set_error("fc_deriv_z_host: NULL plan"); return FC_ERR_ARG; }
  fc_status s = check_deriv_args(plan->data, plan->deriv, dtype, batch, Nx, Ny, Lz, f, df, d2f, "fc_deriv_z_host");
  if (s) return s;
  DerivDevTables* t = nullptr;
  {
    std::lock_guard<std::mutex> lk(plan->data.mtx);
    s = deriv_tables_locked(plan, &t);
  }
  if (s) return s;
  std::lock_guard<std::mutex> hl(plan->data.host_mtx);
  const size_t es = dtype == FC_F32 ? 4 : 8;
  const int Nz = plan->data.Nz;
  const size_t yrow = (size_t)Nz * Nx * es;   // bytes of one y row over all z
  std::vector<Slab> slabs;
  const long long Yc = plan_slabs(batch, Ny, yrow, slab_bytes, &slabs);
  s = stage_for(t, (size_t)Yc * yrow);
  if (s) return s;
  // the slabs start after the work already queued on the caller's stream
  cudaEvent_t e0 = nullptr;
  s = cuda_status(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming), "cudaEventCreate");
  if (!s) s = cuda_status(cudaEventRecord(e0, (cudaStream_t)stream), "cudaEventRecord");
  if (!s) s = cuda_status(cudaStreamWaitEvent(t->st_in, e0, 0), "cudaStreamWaitEvent");
  const char* fh = static_cast<const char*>(f);
  char* oh[2] = {static_cast<char*>(df), static_cast<char*>(d2f)};
  const size_t hp = (size_t)Ny * Nx * es;     // host pitch between z rows
  long long i = 0;
  for (size_t si = 0; si < slabs.size() && !s; ++si, ++i) {
    {  // slab si in staging slot i % 3
      const int b = slabs[si].b;
      const long long y0 = slabs[si].y0, yc = slabs[si].yc;
      const int k = (int)(i % 3);
      const size_t w = (size_t)yc * Nx * es, off = ((size_t)b * Nz * Ny + (size_t)y0) * Nx * es;
      if (i >= 3) s = cuda_status(cudaStreamWaitEvent(t->st_in, t->ev_out[k], 0), "cudaStreamWaitEvent");
      if (!s) s = cuda_status(cudaMemcpy2DAsync(t->stage[k][0], w, fh + off, hp, w, Nz, cudaMemcpyHostToDevice, t->st_in),
                              "cudaMemcpy2DAsync(H2D)");
      if (!s) s = cuda_status(cudaEventRecord(t->ev_in[k], t->st_in), "cudaEventRecord");
      if (!s) s = cuda_status(cudaStreamWaitEvent(t->st_run, t->ev_in[k], 0), "cudaStreamWaitEvent");
      if (!s) s = launch_deriv_z(*t, plan->data, dtype, 1, (long long)Nx * yc, Lz, t->stage[k][0],
                                 df ? t->stage[k][1] : nullptr, d2f ? t->stage[k][2] : nullptr, t->st_run);
      if (!s) s = cuda_status(cudaEventRecord(t->ev_run[k], t->st_run), "cudaEventRecord");
      if (!s) s = cuda_status(cudaStreamWaitEvent(t->st_out, t->ev_run[k], 0), "cudaStreamWaitEvent");
      for (int o = 0; o < 2 && !s; ++o)
        if (oh[o])
          s = cuda_status(cudaMemcpy2DAsync(oh[o] + off, hp, t->stage[k][1 + o], w, w, Nz, cudaMemcpyDeviceToHost,
                                            t->st_out), "cudaMemcpy2DAsync(D2H)");
      if (!s) s = cuda_status(cudaEventRecord(t->ev_out[k], t->st_out), "cudaEventRecord");
    }
  }
  // synchronous: the outputs are in host memory on return (also after an error)
  const fc_status s1 = cuda_status(cudaStreamSynchronize(t->st_in), "cudaStreamSynchronize");
  const fc_status s2 = cuda_status(cudaStreamSynchronize(t->st_run), "cudaStreamSynchronize");
  const fc_status s3 = cuda_status(cudaStreamSynchronize(t->st_out), "cudaStreamSynchronize");
  if (e0) cudaEventDestroy(e0);
  return s ? s : (s1 ? s1 : (s2 ? s2 : s3));
}

extern "C" fc_status fc_deriv_z_host(fc_plan_t plan, fc_dtype dtype, int batch, int Nx, int Ny, double Lz,
                                     const void* f, void* df, void* d2f, fc_stream_t stream) {
  // 256 MB slabs: every copy moves Nz rows of ~0.5 MB; with 64 MB slabs (rows
  // of 128 KB at 512^2 x 513) the strided copies ran at half the speed
  return fc_deriv_z_host_ex(plan, dtype, batch, Nx, Ny, Lz, f, df, d2f, (size_t)256 << 20, stream);
}
