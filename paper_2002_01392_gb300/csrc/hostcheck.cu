// Host-check library: runs the kernel phase functions on the CPU, one block
// after another, so that tests without a GPU can compare the kernels' index
// arithmetic and data flow with the oracle.  Not part of libfcns and never
// loaded by the product path.
#define FC_HOSTCHECK 1
#include <chrono>
#include <complex>
#include <vector>

#include "deriv_kernel.cuh"
#include "host_tables.hpp"
#include "slabs.hpp"

namespace fcns {

template <class T, int L1, int L2, int LINES, int JN, bool SYM, int JI = 0, bool FULL = false>
static int emu_deriv_k(const double* Mr, int d, int Cc, int Nz, int batch, long long lines, double Lz,
                       const T* f, T* df, T* d2f) {
  using K = DerivPair<T, L1, L2, LINES, JN, SYM, JI, FULL>;
  const int L = L1 * L2;
  std::vector<std::complex<double>> H1, H2, tw;
  deriv_conv_spectra(Nz, Nz + Cc, L, &H1, &H2);
  engine_twiddles(L1, L2, &tw);
  std::vector<cx<T>> H1t(L), H2t(L), twt(2 * L);
  for (int i = 0; i < L; ++i) {
    H1t[i] = mk<T>((T)H1[i].real(), (T)H1[i].imag());
    H2t[i] = mk<T>((T)H2[i].real(), (T)H2[i].imag());
  }
  for (int i = 0; i < 2 * L; ++i) twt[i] = mk<T>((T)tw[i].real(), (T)tw[i].imag());
  typename K::Args a;
  a.f = f; a.df = df; a.d2f = d2f;
  a.Nz = Nz; a.Np = Nz + Cc; a.d = d; a.Cc = Cc;
  a.lines = lines; a.pairs = (lines + 1) / 2; a.tiles = (a.pairs + LINES - 1) / LINES;
  a.zstride = lines; a.bstride = lines * Nz;
  const double dz = Lz / (Nz - 1);
  a.s1 = T(1.0 / dz); a.s2 = T(1.0 / (dz * dz));
  std::vector<float2> Mr2(Cc * d);
  for (int i = 0; i < Cc * d; ++i) { Mr2[i].x = (float)Mr[i]; Mr2[i].y = (float)(Mr[i] - (double)Mr2[i].x); }
  a.Mr = Mr; a.Mr2 = Mr2.data(); a.H1 = H1t.data(); a.H2 = H2t.data(); a.tw = twt.data();

  a.nblocks = a.tiles * batch;
  a.pf_dist = 3;
  a.vec = lines % 2 == 0 ? 1 : 0;
  phased_emulate<K>(a, a.tiles * batch, K::smem_bytes);
  return 0;
}

// the variant fc_deriv_z launches: symmetric kernel spectra when L >= 2 N' - 1 or L = N'
template <class T, int L1, int L2, int LINES, int JN>
static int emu_deriv(const double* Mr, int d, int Cc, int Nz, int batch, long long lines, double Lz,
                     const T* f, T* df, T* d2f) {
  const int L = L1 * L2, Np = Nz + Cc;
  // the interior-row form fc_deriv_z runs for float32 at L = 1080, Nz >= 481
  if constexpr (sizeof(T) == 4 && L1 == 30 && L2 == 36 && JN == 16)
    if (L >= 2 * Np - 1 && Nz >= 481)
      return lines % 8 == 0 ? emu_deriv_k<T, L1, L2, LINES, JN, true, 13, true>(Mr, d, Cc, Nz, batch, lines, Lz, f, df, d2f)
                            : emu_deriv_k<T, L1, L2, LINES, JN, true, 13>(Mr, d, Cc, Nz, batch, lines, Lz, f, df, d2f);
  if (L == Np || L >= 2 * Np - 1)
    return emu_deriv_k<T, L1, L2, LINES, JN, true>(Mr, d, Cc, Nz, batch, lines, Lz, f, df, d2f);
  return emu_deriv_k<T, L1, L2, LINES, JN, false>(Mr, d, Cc, Nz, batch, lines, Lz, f, df, d2f);
}

}  // namespace fcns

using namespace fcns;

// The slab plan of fc_deriv_z_host: out[3 i + 0..2] = field, first y row, rows
// of slab i (at most max slabs); returns the staging rows, *n the slab count.
extern "C" long long fchc_slab_plan(int batch, long long Ny, size_t yrow, size_t slab_bytes, long long* out, int max,
                                    int* n) {
  std::vector<Slab> sl;
  const long long Yc = plan_slabs(batch, Ny, yrow, slab_bytes, &sl);
  *n = (int)sl.size();
  for (int i = 0; i < (int)sl.size() && i < max; ++i) {
    out[3 * i] = sl[i].b;
    out[3 * i + 1] = sl[i].y0;
    out[3 * i + 2] = sl[i].yc;
  }
  return Yc;
}

// Emulate fc_deriv_z for transform length L (must be one of the compiled
// shapes and >= N' + Nz - 1).  dtype 0 = float, 1 = double.
extern "C" int fchc_deriv_z(int dtype, int L, const double* Mr, int d, int Cc, int Nz, int batch, int Nx,
                            int Ny, double Lz, const void* f, void* df, void* d2f) {
  const long long lines = (long long)Nx * Ny;
#define HC(LL, A, B, LF, LD)                                                                                 \
  if (L == LL) {                                                                                            \
    if (Nz + Cc <= B * (A / 2 + 1)) {                                                                       \
      if (dtype == 0)                                                                                       \
        return emu_deriv<float, A, B, LF, A / 2 + 1>(Mr, d, Cc, Nz, batch, lines, Lz, (const float*)f, (float*)df, (float*)d2f); \
      return emu_deriv<double, A, B, LD, A / 2 + 1>(Mr, d, Cc, Nz, batch, lines, Lz, (const double*)f, (double*)df, (double*)d2f); \
    }                                                                                                       \
    if (dtype == 0)                                                                                         \
      return emu_deriv<float, A, B, LF, A>(Mr, d, Cc, Nz, batch, lines, Lz, (const float*)f, (float*)df, (float*)d2f); \
    return emu_deriv<double, A, B, LD, A>(Mr, d, Cc, Nz, batch, lines, Lz, (const double*)f, (double*)df, (double*)d2f); \
  }
  HC(64, 8, 8, 16, 8)
  HC(96, 8, 12, 16, 8)
  HC(160, 10, 16, 16, 8)
  HC(288, 16, 18, 16, 8)
  HC(1080, 30, 36, 4, 2)
#undef HC
  return -1;
}

// ---------------------------------------------------------------------------
// Navier-Stokes simulation run on the CPU with the same kernel sequence
// (NsCore with an emulating backend; host memory throughout).
// ---------------------------------------------------------------------------
#include <cstdlib>
#include <cstring>
#if defined(__SANITIZE_ADDRESS__)
#include <sanitizer/asan_interface.h>
#endif

#include "ns_core.hpp"

namespace fcns {
void set_error(const std::string&) {}
fc_status cuda_status(cudaError_t, const char*) { return FC_OK; }

struct EmuBK {
  template <class K>
  fc_status run(const typename K::Args& a, long long grid, void*) {
    phased_emulate<K>(a, grid, K::smem_bytes);
    return FC_OK;
  }
  fc_status alloc(void** p, size_t b) { *p = std::calloc(1, b); return *p ? FC_OK : FC_ERR_NOMEM; }
  void free(void* p) { std::free(p); }
  fc_status h2d(void* d, const void* s, size_t b) { std::memcpy(d, s, b); return FC_OK; }
  fc_status d2d(void* d, const void* s, size_t b, void*) { std::memmove(d, s, b); return FC_OK; }
  fc_status memset(void* d, int v, size_t b, void*) { std::memset(d, v, b); return FC_OK; }
  fc_status d2d_2d(void* dst, size_t dp, const void* src, size_t sp, size_t w, size_t rows, void*) {
    for (size_t r = 0; r < rows; ++r) std::memmove((char*)dst + r * dp, (const char*)src + r * sp, w);
    return FC_OK;
  }
  fc_status sync(void*) { return FC_OK; }
  int sms() { return 1; }
  fc_status d2h(void* d, const void* s, size_t b, void*) { std::memcpy(d, s, b); return FC_OK; }
  // host wall time of the emulated launches (lets the autotuner's logic run on the CPU)
  template <class F>
  fc_status time_ms(F&& f, void*, float* ms) {
    const auto t0 = std::chrono::steady_clock::now();
    const fc_status s = f();
    *ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
  }
};
}  // namespace fcns

extern "C" {
void* fchc_ns_create(const ns_params* p) {
  auto* c = new NsCore<EmuBK>();
  if (c->create(*p, nullptr, 0)) { c->destroy(); delete c; return nullptr; }
#if FC_LAYOUT_GUARD && defined(__SANITIZE_ADDRESS__)
  // the guard bands between the workspace arrays become unaddressable: a
  // kernel or copy that strays out of its array is reported by the sanitizer
  for (auto& g : c->l.guards) {
    const size_t b = (g.first + 7) / 8 * 8;
    if (g.second > b) ASAN_POISON_MEMORY_REGION(c->ws + b, g.second - b);
  }
#endif
  return c;
}
void fchc_ns_destroy(void* h) {
  auto* c = (NsCore<EmuBK>*)h;
#if FC_LAYOUT_GUARD && defined(__SANITIZE_ADDRESS__)
  ASAN_UNPOISON_MEMORY_REGION(c->ws, c->l.total);
#endif
  c->destroy();
  delete c;
}
int fchc_ns_set_fields(void* h, const void* phys) { return ((NsCore<EmuBK>*)h)->set_fields_any(phys, nullptr); }
int fchc_ns_get_fields(void* h, void* phys) { return ((NsCore<EmuBK>*)h)->get_fields_any(phys, nullptr); }
int fchc_ns_rhs(void* h, const void* in, void* out) { return ((NsCore<EmuBK>*)h)->rhs_any(in, out, nullptr); }
int fchc_ns_project(void* h, double dt, const void* in, void* out, void* gp) {
  return ((NsCore<EmuBK>*)h)->project_any(dt, in, out, gp, nullptr);
}
int fchc_ns_step(void* h, double dt) { return ((NsCore<EmuBK>*)h)->step_any(dt, nullptr); }
int fchc_ns_set_tiles(void* h, const int* tiles) {
  auto* c = (NsCore<EmuBK>*)h;
  for (int k = 0; k < NsCore<EmuBK>::TK_N; ++k) c->tile[k] = tiles[k] & c->variant_mask(k);
  return 0;
}
int fchc_ns_profiles_raw(void* h, double* out) { return ((NsCore<EmuBK>*)h)->profiles_any(out, nullptr); }
int fchc_ns_interpolate(void* dst, void* src) {
  return ((NsCore<EmuBK>*)dst)->interpolate_from_any(*(NsCore<EmuBK>*)src, nullptr);
}
int fchc_ns_diag_raw(void* h, double* acc6) { return ((NsCore<EmuBK>*)h)->diagnostics_any(acc6, nullptr); }
int fchc_ns_get_state(void* h, void* out) {
  auto* c = (NsCore<EmuBK>*)h;
  std::memcpy(out, c->ws + c->l.X[c->cur], c->state_bytes());
  return 0;
}
int fchc_ns_put_state(void* h, const void* in) {
  auto* c = (NsCore<EmuBK>*)h;
  std::memcpy(c->ws + c->l.X[c->cur], in, c->state_bytes());
  return c->mean_init_any(nullptr);
}
int fchc_ns_count_nonfinite(void* h, long long* count) {
  auto* c = (NsCore<EmuBK>*)h;
  fc_status s = c->count_nonfinite_any(true, nullptr);
  unsigned long long n = 0;
  if (!s) s = c->bk.d2h(&n, c->ws + c->l.nfin, sizeof(n), nullptr);
  *count = (long long)n;
  return s;
}
// ns_tune mode 1 on the CPU: every variant timed by host wall clock; the
// choice is written to tiles (5 ints)
int fchc_ns_autotune(void* h, int* tiles) {
  auto* c = (NsCore<EmuBK>*)h;
  const fc_status s = c->autotune_any(nullptr);
  for (int k = 0; k < NsCore<EmuBK>::TK_N; ++k) tiles[k] = c->tile[k];
  return s;
}
// thread order inside a phase (0 ascending, 1 descending) and shared-memory
// poisoning of the emulation (see phased_emulate)
void fchc_set_emulation(int order, int poison) {
  emu_order() = order;
  emu_poison() = poison;
}
}
