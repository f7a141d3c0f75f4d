// Host-check library: runs the kernel phase functions on the CPU, one block
// after another, so that tests without a GPU can compare the kernels' index
// arithmetic and data flow with the oracle.  Not part of libfcns and never
// loaded by the product path.
#define FC_HOSTCHECK 1
#include <complex>
#include <vector>

#include "deriv_kernel.cuh"
#include "host_tables.hpp"

namespace fcns {

template <class T, int L1, int L2, int LINES>
static int emu_deriv(const double* Mr, int d, int Cc, int Nz, int batch, long long lines, double Lz,
                     const T* f, T* df, T* d2f) {
  using K = DerivConv<T, L1, L2, LINES>;
  const int L = L1 * L2;
  std::vector<std::complex<double>> H, tw;
  deriv_conv_spectrum(Nz, Nz + Cc, L, &H);
  engine_twiddles(L1, L2, &tw);
  std::vector<cx<T>> Ht(L), twt(L);
  for (int i = 0; i < L; ++i) {
    Ht[i] = mk<T>((T)H[i].real(), (T)H[i].imag());
    twt[i] = mk<T>((T)tw[i].real(), (T)tw[i].imag());
  }
  typename K::Args a;
  a.f = f; a.df = df; a.d2f = d2f;
  a.Nz = Nz; a.Np = Nz + Cc; a.d = d; a.Cc = Cc;
  a.lines = lines; a.tiles = (lines + LINES - 1) / LINES;
  a.zstride = lines; a.bstride = lines * Nz;
  const double dz = Lz / (Nz - 1);
  a.s1 = T(1.0 / dz); a.s2 = T(1.0 / (dz * dz));
  a.Mr = Mr; a.H = Ht.data(); a.tw = twt.data();
  phased_emulate<K>(a, a.tiles * batch, K::smem_bytes);
  return 0;
}

}  // namespace fcns

using namespace fcns;

// Emulate fc_deriv_z for transform length L (must be one of the compiled
// shapes and >= N' + Nz - 1).  dtype 0 = float, 1 = double.
extern "C" int fchc_deriv_z(int dtype, int L, const double* Mr, int d, int Cc, int Nz, int batch, int Nx,
                            int Ny, double Lz, const void* f, void* df, void* d2f) {
  const long long lines = (long long)Nx * Ny;
#define HC(LL, A, B, LF, LD)                                                                                 \
  if (L == LL) {                                                                                            \
    if (dtype == 0)                                                                                         \
      return emu_deriv<float, A, B, LF>(Mr, d, Cc, Nz, batch, lines, Lz, (const float*)f, (float*)df, (float*)d2f); \
    return emu_deriv<double, A, B, LD>(Mr, d, Cc, Nz, batch, lines, Lz, (const double*)f, (double*)df, (double*)d2f); \
  }
  HC(96, 8, 12, 32, 16)
  HC(160, 10, 16, 32, 16)
  HC(288, 16, 18, 32, 16)
  HC(1080, 30, 36, 16, 8)
#undef HC
  return -1;
}
