// fc_noise: the random solenoidal no-slip perturbation of App. A, built on
// the device from caller-supplied uniform draws.
//
//   q = curl curl(phi z_hat) + curl(psi z_hat)
//     = (d_x d_z phi + d_y psi, d_y d_z phi - d_x psi, -(d_xx + d_yy) phi),
//   phi = sum a e^{i(kx x + ky y)} g_m(z'),  psi = sum b e^{i(kx x + ky y)} sin(m pi (z' + 1/2)),
//   z' = z/Lz - 1/2,  g_m the Chandrasekhar-Reid functions (cosh/cos for odd
//   m, sinh/sin for even m) with lambda_m from g_m'(+-1/2) = 0,
//   a = k^slope_phi e^{2 pi i u_a}, b = k^slope_psi e^{2 pi i u_b},
//   k^2 = kx^2 + ky^2 + lambda_m^2, over the half plane of horizontal modes in
//   the annulus kperp2_min <= kx^2 + ky^2 <= kperp2_max and m_min <= m <= m_max;
//   the real part, scaled to a largest component magnitude of `amplitude`.
//
// Five launches, all in float64 arithmetic: the vertical profiles of every
// horizontal mode (sum over m), the e^{i kx x} / e^{i ky y} tables (exact
// argument reduction: the phase 2 pi n i / Nx is taken modulo 2 pi in
// integers), the synthesis (one block per (z, y) row: first the sums over the
// modes that share kx, then one real sum over kx per point), the largest
// magnitude (a block-max reduction into one device word) and the scaling.
#include "internal.hpp"

#include <cmath>
#include <cstring>

namespace fcns {
namespace {

constexpr int kMaxM = 64;

__device__ __forceinline__ double2 cmulD(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// P[(h * Nz + s) * 3 + c]: the z-profile of component c of horizontal mode h
__global__ void noise_profiles(int H, int nm, int m_min, int Nz, double Lz, const double2* __restrict__ kxy,
                               const double2* __restrict__ ab, const double* __restrict__ lam,
                               double2* __restrict__ P) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)H * Nz) return;
  const int h = (int)(idx / Nz), s = (int)(idx % Nz);
  const double zp = (double)(2 * s - (Nz - 1)) / (double)(2 * (Nz - 1));
  const double kx = kxy[h].x, ky = kxy[h].y, kp2 = kx * kx + ky * ky;
  double2 pu = make_double2(0, 0), pv = make_double2(0, 0), pw = make_double2(0, 0);
  for (int mi = 0; mi < nm; ++mi) {
    const int m = m_min + mi;
    const double L = lam[mi];
    double g, dg;
    if (m & 1) {
      const double ch = cosh(0.5 * L), co = cos(0.5 * L);
      g = cosh(L * zp) / ch - cos(L * zp) / co;
      dg = L * (sinh(L * zp) / ch + sin(L * zp) / co);
    } else {
      const double sh = sinh(0.5 * L), si = sin(0.5 * L);
      g = sinh(L * zp) / sh - sin(L * zp) / si;
      dg = L * (cosh(L * zp) / sh - cos(L * zp) / si);
    }
    const double dgdz = dg / Lz;
    // sin(m pi (z' + 1/2)) = sin(pi m s / (Nz - 1)), reduced exactly modulo 2
    const long long num = ((long long)m * s) % (2LL * (Nz - 1));
    const double sn = sinpi((double)num / (double)(Nz - 1));
    const double2 a = ab[2 * (h * nm + mi)], b = ab[2 * (h * nm + mi) + 1];
    // i c = (-c.y, c.x)
    pu.x += -kx * a.y * dgdz - ky * b.y * sn;
    pu.y += kx * a.x * dgdz + ky * b.x * sn;
    pv.x += -ky * a.y * dgdz + kx * b.y * sn;
    pv.y += ky * a.x * dgdz - kx * b.x * sn;
    pw.x += kp2 * a.x * g;
    pw.y += kp2 * a.y * g;
  }
  P[idx * 3 + 0] = pu;
  P[idx * 3 + 1] = pv;
  P[idx * 3 + 2] = pw;
}

// Ex[(n + nmax) * Nx + i] = e^{2 pi i n i / Nx}, Ey[l * Ny + j] = e^{2 pi i l j / Ny}
__global__ void noise_phases(int nmax, int lmax, int Nx, int Ny, double2* __restrict__ Ex,
                             double2* __restrict__ Ey) {
  const long long nx = (long long)(2 * nmax + 1) * Nx, ny = (long long)(lmax + 1) * Ny;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nx) {
    const int n = (int)(idx / Nx) - nmax, i = (int)(idx % Nx);
    long long r = ((long long)n * i) % Nx;
    if (r < 0) r += Nx;
    double sv, cv;
    sincospi(2.0 * (double)r / (double)Nx, &sv, &cv);
    Ex[idx] = make_double2(cv, sv);
  } else if (idx < nx + ny) {
    const long long k = idx - nx;
    const int l = (int)(k / Ny), j = (int)(k % Ny);
    const long long r = ((long long)l * j) % Ny;
    double sv, cv;
    sincospi(2.0 * (double)r / (double)Ny, &sv, &cv);
    Ey[k] = make_double2(cv, sv);
  }
}

// one block per (z, y) row: Q[c][n] = sum over modes h with kx index n of
// P[h][z][c] e^{i ky_h y}, then out[c][z][y][x] = sum_n Re(Q[c][n] e^{i kx_n x})
template <class T>
__global__ void noise_synth(int H, int nmax, int Nx, int Ny, int Nz, const int2* __restrict__ nl,
                            const double2* __restrict__ P, const double2* __restrict__ Ex,
                            const double2* __restrict__ Ey, T* __restrict__ out) {
  extern __shared__ double2 Q[];  // [3][2 nmax + 1]
  const int NN = 2 * nmax + 1;
  const long long row = blockIdx.x;
  const int s = (int)(row / Ny), j = (int)(row % Ny);
  for (int t = threadIdx.x; t < 3 * NN; t += blockDim.x) {
    const int c = t / NN, ni = t % NN;
    double2 acc = make_double2(0, 0);
    for (int h = 0; h < H; ++h) {
      const int2 q = nl[h];
      if (q.x + nmax != ni) continue;
      const double2 v = cmulD(P[((long long)h * Nz + s) * 3 + c], Ey[(long long)q.y * Ny + j]);
      acc.x += v.x;
      acc.y += v.y;
    }
    Q[t] = acc;
  }
  __syncthreads();
  const long long plane = (long long)Nz * Ny * Nx;
  T* o = out + ((long long)s * Ny + j) * Nx;
  for (int i = threadIdx.x; i < Nx; i += blockDim.x) {
    double r0 = 0, r1 = 0, r2 = 0;
    for (int ni = 0; ni < NN; ++ni) {
      const double2 e = Ex[(long long)ni * Nx + i];
      const double2 a = Q[ni], b = Q[NN + ni], c = Q[2 * NN + ni];
      r0 += a.x * e.x - a.y * e.y;
      r1 += b.x * e.x - b.y * e.y;
      r2 += c.x * e.x - c.y * e.y;
    }
    o[i] = (T)r0;
    o[plane + i] = (T)r1;
    o[2 * plane + i] = (T)r2;
  }
}

// largest |out| into *word (bits of a non-negative double: their unsigned order is the numeric order)
template <class T>
__global__ void noise_absmax(const T* __restrict__ out, long long n, unsigned long long* word) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)out[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(word, (unsigned long long)__double_as_longlong(m));
  }
}

template <class T>
__global__ void noise_scale(T* __restrict__ out, long long n, const unsigned long long* word, double amplitude) {
  const double mx = __longlong_as_double((long long)*word);
  if (!(mx > 0.0)) return;
  const double f = amplitude / mx;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)((double)out[i] * f);
}

// lambda_m: root of tanh t + tan t (odd m) or tanh t - tan t (even m), t = lambda/2,
// on the m-th bracket; bisection to adjacent doubles
double cr_lambda(int m) {
  const double pi = 3.14159265358979323846;
  const bool odd = (m & 1) != 0;
  const int j = odd ? (m + 1) / 2 : m / 2;
  double lo = odd ? j * pi - pi / 2 : j * pi, hi = odd ? j * pi : j * pi + pi / 2;
  lo += 1e-9;
  hi -= 1e-9;
  auto f = [odd](double t) { return odd ? std::tanh(t) + std::tan(t) : std::tanh(t) - std::tan(t); };
  const double flo = f(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double fm = f(mid);
    if (fm == 0.0) return 2.0 * mid;
    if ((fm < 0) == (flo < 0)) lo = mid;
    else hi = mid;
  }
  return std::fabs(f(lo)) <= std::fabs(f(hi)) ? 2.0 * lo : 2.0 * hi;
}

struct NoiseModes {
  int nmax = 0, lmax = 0;
  std::vector<int2> nl;        // horizontal modes (n, l), enumeration order
  std::vector<double2> kxy;    // their (kx, ky)
};

fc_status check_params(const fc_noise_params* p) {
  if (!p) {
    set_error("fc_noise: NULL parameters");
    return FC_ERR_ARG;
  }
  const bool ok = std::isfinite(p->Lx) && std::isfinite(p->Ly) && std::isfinite(p->Lz) && p->Lx > 0 && p->Ly > 0 &&
                  p->Lz > 0 && std::isfinite(p->kperp2_min) && std::isfinite(p->kperp2_max) && p->kperp2_min >= 0 &&
                  p->kperp2_max >= p->kperp2_min && p->kperp2_max * p->Lx * p->Lx < 4e8 &&
                  p->kperp2_max * p->Ly * p->Ly < 4e8 && p->m_min >= 1 && p->m_max >= p->m_min &&
                  p->m_max <= kMaxM && std::isfinite(p->slope_phi) && std::isfinite(p->slope_psi) &&
                  std::isfinite(p->amplitude);
  if (!ok) {
    set_error("fc_noise: need Lx, Ly, Lz > 0, 0 <= kperp2_min <= kperp2_max (kperp2_max Lx^2, kperp2_max Ly^2 < 4e8), "
              "1 <= m_min <= m_max <= 64, finite slopes and amplitude");
    return FC_ERR_ARG;
  }
  return FC_OK;
}

NoiseModes enumerate_modes(const fc_noise_params& p) {
  const double pi = 3.14159265358979323846;
  NoiseModes r;
  const int nmax = (int)std::floor(std::sqrt(p.kperp2_max) * p.Lx / (2 * pi)) + 1;
  const int lmax = (int)std::floor(std::sqrt(p.kperp2_max) * p.Ly / (2 * pi)) + 1;
  for (int n = -nmax; n <= nmax; ++n)
    for (int l = 0; l <= lmax; ++l) {
      if (l == 0 && n <= 0) continue;
      const double kx = 2 * pi * n / p.Lx, ky = 2 * pi * l / p.Ly, kp2 = kx * kx + ky * ky;
      if (!(p.kperp2_min * (1 - 1e-12) <= kp2 && kp2 <= p.kperp2_max * (1 + 1e-12))) continue;
      r.nl.push_back(make_int2(n, l));
      r.kxy.push_back(make_double2(kx, ky));
      r.nmax = std::max(r.nmax, n < 0 ? -n : n);
      r.lmax = std::max(r.lmax, l);
    }
  return r;
}

}  // namespace
}  // namespace fcns

using namespace fcns;

extern "C" fc_status fc_noise_params_default(fc_noise_params* p) {
  if (!p) {
    set_error("fc_noise_params_default: NULL");
    return FC_ERR_ARG;
  }
  p->Lx = p->Ly = 2 * 3.14159265358979323846;
  p->Lz = 1.0;
  p->kperp2_min = 4.0;
  p->kperp2_max = 25.0;
  p->m_min = 2;
  p->m_max = 5;
  p->slope_phi = -4.0;
  p->slope_psi = -3.0;
  p->amplitude = 1.0;
  return FC_OK;
}

extern "C" fc_status fc_noise_modes(const fc_noise_params* p, int* count) {
  if (fc_status s = check_params(p)) return s;
  if (!count) {
    set_error("fc_noise_modes: NULL count");
    return FC_ERR_ARG;
  }
  *count = (int)enumerate_modes(*p).nl.size() * (p->m_max - p->m_min + 1);
  return FC_OK;
}

extern "C" fc_status fc_noise(const fc_noise_params* p, fc_dtype dtype, int Nx, int Ny, int Nz, const double* draws,
                              int ndraws, void* out, fc_stream_t stream) {
  if (fc_status inj = injected("fc_noise")) return inj;
  if (fc_status s = check_params(p)) return s;
  if ((dtype != FC_F32 && dtype != FC_F64) || Nx < 1 || Ny < 1 || Nz < 2 || !out || !draws) {
    set_error("fc_noise: dtype must be FC_F32 or FC_F64, Nx, Ny >= 1, Nz >= 2, draws and out non-NULL");
    return FC_ERR_ARG;
  }
  const NoiseModes md = enumerate_modes(*p);
  const int H = (int)md.nl.size(), nm = p->m_max - p->m_min + 1;
  if (H == 0) {
    set_error("fc_noise: no horizontal mode in the annulus");
    return FC_ERR_ARG;
  }
  if ((long long)ndraws != 2LL * H * nm) {
    set_error("fc_noise: ndraws must be 2 x fc_noise_modes()");
    return FC_ERR_ARG;
  }
  if (Nx <= 2 * md.nmax || Ny <= 2 * md.lmax) {
    set_error("fc_noise: the grid must resolve every mode (Nx > 2 max|n|, Ny > 2 max l)");
    return FC_ERR_ARG;
  }
  if (2 * md.nmax + 1 > 1024) {   // the synthesis keeps 3 x (2 nmax + 1) complex sums in 48 KB of shared memory
    set_error("fc_noise: at most 511 kx indices on each side of the annulus");
    return FC_ERR_UNSUPPORTED;
  }
  if ((long long)Nz * Ny > 0x7fffffffLL || 3LL * Nz * Ny * Nx > (1LL << 40)) {
    set_error("fc_noise: grid too large");
    return FC_ERR_ARG;
  }
  for (int i = 0; i < ndraws; ++i)
    if (!std::isfinite(draws[i])) {
      set_error("fc_noise: non-finite draw");
      return FC_ERR_ARG;
    }
  // host side: lambda_m and the complex amplitudes a, b of every (n, l, m) mode
  const double pi = 3.14159265358979323846;
  std::vector<double> lam(nm);
  for (int mi = 0; mi < nm; ++mi) lam[mi] = cr_lambda(p->m_min + mi);
  std::vector<double2> ab(2 * (size_t)H * nm);
  for (int h = 0; h < H; ++h)
    for (int mi = 0; mi < nm; ++mi) {
      const double kx = md.kxy[h].x, ky = md.kxy[h].y;
      const double k = std::sqrt(kx * kx + ky * ky + lam[mi] * lam[mi]);
      const size_t j = (size_t)h * nm + mi;
      const double ra = std::pow(k, p->slope_phi), rb = std::pow(k, p->slope_psi);
      ab[2 * j] = make_double2(ra * std::cos(2 * pi * draws[2 * j]), ra * std::sin(2 * pi * draws[2 * j]));
      ab[2 * j + 1] = make_double2(rb * std::cos(2 * pi * draws[2 * j + 1]), rb * std::sin(2 * pi * draws[2 * j + 1]));
    }
  // one device block of scratch: tables, profiles, phase tables, max word
  const size_t nEx = (size_t)(2 * md.nmax + 1) * Nx, nEy = (size_t)(md.lmax + 1) * Ny;
  const size_t nP = (size_t)H * Nz * 3;
  size_t off = 0;
  auto take = [&off](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  const size_t o_word = take(sizeof(unsigned long long)), o_kxy = take(sizeof(double2) * H),
               o_nl = take(sizeof(int2) * H), o_ab = take(sizeof(double2) * ab.size()),
               o_lam = take(sizeof(double) * nm), o_P = take(sizeof(double2) * nP),
               o_Ex = take(sizeof(double2) * nEx), o_Ey = take(sizeof(double2) * nEy);
  const size_t host_bytes = o_P;  // everything before the profiles comes from the host
  std::vector<unsigned char> h(host_bytes, 0);
  std::memcpy(h.data() + o_kxy, md.kxy.data(), sizeof(double2) * H);
  std::memcpy(h.data() + o_nl, md.nl.data(), sizeof(int2) * H);
  std::memcpy(h.data() + o_ab, ab.data(), sizeof(double2) * ab.size());
  std::memcpy(h.data() + o_lam, lam.data(), sizeof(double) * nm);

  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* buf = nullptr;
  const cudaError_t ae = cudaMallocAsync((void**)&buf, off, st);
  if (ae == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error("fc_noise: cudaMallocAsync of the scratch failed");
    return FC_ERR_NOMEM;
  }
  fc_status s = cuda_status(ae, "cudaMallocAsync");
  if (s) return s;
  // pageable source: the call returns once the bytes are staged, so `h` may go
  s = cuda_status(cudaMemcpyAsync(buf, h.data(), host_bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  auto* word = reinterpret_cast<unsigned long long*>(buf + o_word);
  auto* kxy = reinterpret_cast<double2*>(buf + o_kxy);
  auto* nl = reinterpret_cast<int2*>(buf + o_nl);
  auto* dab = reinterpret_cast<double2*>(buf + o_ab);
  auto* dlam = reinterpret_cast<double*>(buf + o_lam);
  auto* P = reinterpret_cast<double2*>(buf + o_P);
  auto* Ex = reinterpret_cast<double2*>(buf + o_Ex);
  auto* Ey = reinterpret_cast<double2*>(buf + o_Ey);
  const long long n = 3LL * Nz * Ny * Nx;
  if (!s) {
    const long long np = (long long)H * Nz;
    noise_profiles<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(H, nm, p->m_min, Nz, p->Lz, kxy, dab, dlam, P);
    const long long ne = (long long)(nEx + nEy);
    noise_phases<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(md.nmax, md.lmax, Nx, Ny, Ex, Ey);
    const unsigned rows = (unsigned)((long long)Nz * Ny);
    const int thr = Nx >= 128 ? 128 : 32;
    const size_t shm = sizeof(double2) * 3 * (2 * md.nmax + 1);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const unsigned gb = (unsigned)std::max(1LL, std::min<long long>(want, (long long)std::max(sms, 1) * 8));
    if (dtype == FC_F32) {
      float* o = static_cast<float*>(out);
      noise_synth<float><<<rows, thr, shm, st>>>(H, md.nmax, Nx, Ny, Nz, nl, P, Ex, Ey, o);
      noise_absmax<float><<<gb, 256, 0, st>>>(o, n, word);
      noise_scale<float><<<gb, 256, 0, st>>>(o, n, word, p->amplitude);
    } else {
      double* o = static_cast<double*>(out);
      noise_synth<double><<<rows, thr, shm, st>>>(H, md.nmax, Nx, Ny, Nz, nl, P, Ex, Ey, o);
      noise_absmax<double><<<gb, 256, 0, st>>>(o, n, word);
      noise_scale<double><<<gb, 256, 0, st>>>(o, n, word, p->amplitude);
    }
    s = cuda_status(cudaGetLastError(), "fc_noise launch");
  }
  const fc_status s2 = cuda_status(cudaFreeAsync(buf, st), "cudaFreeAsync");
  return s ? s : s2;
}
