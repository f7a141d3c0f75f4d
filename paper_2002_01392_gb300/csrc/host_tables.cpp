// Host-side tables in binary128 arithmetic (double-binary128 where the FC
// fits need more than 34 digits).
//
// FC-Gram tables follow App. B of the paper: Gram basis from the QR
// factorisation of the Vandermonde matrix of the d matching points (the basis
// orthonormal for the discrete inner product over those points), and
// blend-to-zero continuations of every Gram polynomial obtained as
// oversampled least-squares trigonometric fits with periodicity interval
// [1 - delta_r, 2b - (1 - delta_r)] (2(d + C) grid spacings).  The right-end
// matrix is M_r = A_r Q_r^T (App. B, eq. Af).
#include "host_tables.hpp"

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

namespace fcns {

typedef _Float128 q;

static q q_abs(q x) { return x < 0 ? -x : x; }

static q q_sqrt(q x) {
  if (x <= 0) return 0;
  q y = (q)std::sqrt((double)x);
  for (int i = 0; i < 4; ++i) y = (y + x / y) / 2;
  return y;
}

// atan(1/x) by its alternating series
static q q_atan_inv(int x) {
  q x2 = (q)x * (q)x, term = (q)1 / (q)x, sum = term;
  const q tiny = (q)1e-40;
  for (int k = 1; k < 400; ++k) {
    term /= x2;
    q t = term / (q)(2 * k + 1);
    sum += (k & 1) ? -t : t;
    if (t < tiny) break;
  }
  return sum;
}

static q q_pi() {
  static const q pi = 16 * q_atan_inv(5) - 4 * q_atan_inv(239);  // Machin's formula
  return pi;
}

static q taylor_sin(q x) {
  q x2 = x * x, term = x, sum = x;
  for (int n = 1; n < 30; ++n) { term *= -x2 / (q)((2 * n) * (2 * n + 1)); sum += term; }
  return sum;
}
static q taylor_cos(q x) {
  q x2 = x * x, term = 1, sum = 1;
  for (int n = 1; n < 30; ++n) { term *= -x2 / (q)((2 * n - 1) * (2 * n)); sum += term; }
  return sum;
}

// cos, sin of 2 pi num/den: exact reduction to the nearest quarter turn
static void q_sincos2pi(long long num, long long den, q* c, q* s) {
  long long r = ((num % den) + den) % den;
  long long m4 = (8 * r + den) / (2 * den);
  long long resid = 4 * r - m4 * den;
  int m = int(m4 & 3);
  q psi = 2 * q_pi() * ((q)resid / (q)(4 * den));
  q cs = taylor_cos(psi), sn = taylor_sin(psi);
  switch (m) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
  }
}

void sincos2pi(long long num, long long den, double* c, double* s) {
  q cq, sq;
  q_sincos2pi(num, den, &cq, &sq);
  *c = (double)cq;
  *s = (double)sq;
}

// ---------------------------------------------------------------------------
// Double-binary128 ("qq") arithmetic: a value is hi + lo, |lo| <= ulp(hi)/2,
// about 226 significant bits (67 digits).  The FC tables need it for d >= 6:
// the least-squares continuation fits for (d, C) = (7, 33), M = 26 are so
// ill-conditioned that binary128 (34 digits) leaves ~1e-12 relative error in
// M_r, while 45 digits reproduce it to double precision.  Built from the
// error-free transformations of Knuth (two-sum) and Dekker (two-product with
// the 2^57 + 1 splitter for the 113-bit binary128 significand).
// ---------------------------------------------------------------------------
struct qq {
  q hi = 0, lo = 0;
  qq() = default;
  qq(q h) : hi(h) {}
  qq(q h, q l) : hi(h), lo(l) {}
  qq(int i) : hi((q)i) {}
  qq(long long i) : hi((q)i) {}
  explicit operator double() const { return (double)hi + (double)lo; }
};
static inline qq quick_two_sum(q a, q b) {
  const q s = a + b;
  return qq(s, b - (s - a));
}
static inline qq two_sum(q a, q b) {
  const q s = a + b, bb = s - a;
  return qq(s, (a - (s - bb)) + (b - bb));
}
static inline void dekker_split(q a, q* h, q* l) {
  const q t = (q)144115188075855873LL * a;  // (2^57 + 1) a
  *h = t - (t - a);
  *l = a - *h;
}
static inline qq two_prod(q a, q b) {
  const q p = a * b;
  q ah, al, bh, bl;
  dekker_split(a, &ah, &al);
  dekker_split(b, &bh, &bl);
  return qq(p, ((ah * bh - p) + ah * bl + al * bh) + al * bl);
}
static inline qq operator+(qq a, qq b) {
  qq s = two_sum(a.hi, b.hi);
  const qq t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline qq operator-(qq a) { return qq(-a.hi, -a.lo); }
static inline qq operator-(qq a, qq b) { return a + (-b); }
static inline qq operator*(qq a, qq b) {
  qq p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static inline qq operator/(qq a, qq b) {
  const q q1 = a.hi / b.hi;
  qq r = a - b * qq(q1);
  const q q2 = r.hi / b.hi;
  r = r - b * qq(q2);
  const q q3 = r.hi / b.hi;
  return quick_two_sum(q1, q2) + qq(q3);
}
static inline qq& operator+=(qq& a, qq b) { return a = a + b; }
static inline qq& operator-=(qq& a, qq b) { return a = a - b; }
static inline qq& operator*=(qq& a, qq b) { return a = a * b; }
static inline qq& operator/=(qq& a, qq b) { return a = a / b; }
static inline bool operator<(qq a, qq b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
static inline bool operator>(qq a, qq b) { return b < a; }
static inline bool operator<=(qq a, qq b) { return !(b < a); }
static inline bool operator==(qq a, qq b) { return a.hi == b.hi && a.lo == b.lo; }

// scalar traits used by the generic table construction below
template <class S> struct Sc;
template <> struct Sc<q> {
  static q sqrt(q x) { return q_sqrt(x); }
  static q tiny() { return (q)1e-40; }
};
template <> struct Sc<qq> {
  static qq sqrt(qq x) {
    if (x.hi <= 0) return qq(0);
    const qq y(q_sqrt(x.hi));
    return y + (x - y * y) / (qq(2) * y);  // one Newton step doubles the 113 bits
  }
  static qq tiny() { return qq((q)1e-75); }
};

// atan(1/x) by its alternating series, pi by Machin's formula
template <class S>
static S g_atan_inv(int x) {
  const S x2 = S(x) * S(x);
  S term = S(1) / S(x), sum = term;
  for (int k = 1; k < 800; ++k) {
    term /= x2;
    const S t = term / S(2 * k + 1);
    sum += (k & 1) ? -t : t;
    if (t < Sc<S>::tiny()) break;
  }
  return sum;
}
template <class S>
static S g_pi() {
  static const S pi = S(16) * g_atan_inv<S>(5) - S(4) * g_atan_inv<S>(239);
  return pi;
}
template <class S>
static void g_sincos2pi(long long num, long long den, S* c, S* s) {
  long long r = ((num % den) + den) % den;
  long long m4 = (8 * r + den) / (2 * den);
  long long resid = 4 * r - m4 * den;
  int m = int(m4 & 3);
  const S psi = S(2) * g_pi<S>() * (S(resid) / S(4 * den));
  // Taylor series, |psi| <= pi/4: 40 terms reach 1e-100
  const S x2 = psi * psi;
  S ts = psi, tc = S(1), sn = psi, cs = S(1);
  for (int n = 1; n < 40; ++n) {
    ts *= -x2 / S((2 * n) * (2 * n + 1));
    tc *= -x2 / S((2 * n - 1) * (2 * n));
    sn += ts;
    cs += tc;
  }
  switch (m) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
  }
}

// Householder QR least squares: minimise |A x - b| for A (m x n, m >= n),
// several right-hand sides.  A is overwritten.
template <class S>
static void lsq_solve(std::vector<S>& A, int m, int n, std::vector<std::vector<S>>& rhs,
                      std::vector<std::vector<S>>* sol) {
  std::vector<S> v(m);
  for (int k = 0; k < n; ++k) {
    S norm = 0;
    for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
    norm = Sc<S>::sqrt(norm);
    S alpha = A[k * n + k] > S(0) ? -norm : norm;
    for (int i = 0; i < m; ++i) v[i] = 0;
    v[k] = A[k * n + k] - alpha;
    for (int i = k + 1; i < m; ++i) v[i] = A[i * n + k];
    S vnorm2 = 0;
    for (int i = k; i < m; ++i) vnorm2 += v[i] * v[i];
    if (vnorm2 == S(0)) continue;
    for (int j = k; j < n; ++j) {
      S dot = 0;
      for (int i = k; i < m; ++i) dot += v[i] * A[i * n + j];
      S f = S(2) * dot / vnorm2;
      for (int i = k; i < m; ++i) A[i * n + j] -= f * v[i];
    }
    for (auto& b : rhs) {
      S dot = 0;
      for (int i = k; i < m; ++i) dot += v[i] * b[i];
      S f = S(2) * dot / vnorm2;
      for (int i = k; i < m; ++i) b[i] -= f * v[i];
    }
  }
  sol->assign(rhs.size(), std::vector<S>(n));
  for (size_t r = 0; r < rhs.size(); ++r) {
    auto& x = (*sol)[r];
    for (int k = n - 1; k >= 0; --k) {
      S s = rhs[r][k];
      for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
      x[k] = s / A[k * n + k];
    }
  }
}

template <class S>
static bool build_fc_tables_in(int d, int C, int M, int n_os, FcTables* out) {
  const int P = 2 * (d + C);  // Fourier period in grid units
  // --- Gram basis: orthonormalise the Vandermonde columns V[i][p] = t_i^p, t_i = i
  std::vector<S> V(d * d);
  for (int i = 0; i < d; ++i) {
    S tp = 1;
    for (int p = 0; p < d; ++p) { V[i * d + p] = tp; tp *= S(i); }
  }
  // modified Gram-Schmidt on the columns gives Q (d x d) and R
  std::vector<S> Qm(d * d), R(d * d, S(0));
  for (int k = 0; k < d; ++k) {
    std::vector<S> col(d);
    for (int i = 0; i < d; ++i) col[i] = V[i * d + k];
    for (int pass = 0; pass < 2; ++pass)  // re-orthogonalise once
      for (int j = 0; j < k; ++j) {
        S dot = 0;
        for (int i = 0; i < d; ++i) dot += Qm[i * d + j] * col[i];
        R[j * d + k] += dot;
        for (int i = 0; i < d; ++i) col[i] -= dot * Qm[i * d + j];
      }
    S nrm = 0;
    for (int i = 0; i < d; ++i) nrm += col[i] * col[i];
    nrm = Sc<S>::sqrt(nrm);
    R[k * d + k] = nrm;
    for (int i = 0; i < d; ++i) Qm[i * d + k] = col[i] / nrm;
  }
  // polynomial coefficients of Gram polynomial k: Q = V R^{-1}, so c_k = column k of R^{-1}
  std::vector<S> Rinv(d * d, S(0));
  for (int k = 0; k < d; ++k) {
    for (int i = d - 1; i >= 0; --i) {  // solve R x = e_k
      S s = (i == k) ? S(1) : S(0);
      for (int j = i + 1; j < d; ++j) s -= R[i * d + j] * Rinv[j * d + k];
      Rinv[i * d + k] = s / R[i * d + i];
    }
  }
  auto gram_val = [&](int k, S t) {
    S s = 0, tp = 1;
    for (int p = 0; p < d; ++p) { s += Rinv[p * d + k] * tp; tp *= t; }
    return s;
  };
  // --- least-squares system: points t = i/n_os on [0, d-1] and d+C + i/n_os
  const int npt = (d - 1) * n_os + 1;
  const int m = 2 * npt, n = 2 * M + 1;
  if (m < n) return false;
  std::vector<S> A(m * n);
  std::vector<long long> tnum(m);  // t = tnum / n_os
  for (int i = 0; i < npt; ++i) { tnum[i] = i; tnum[npt + i] = (long long)(d + C) * n_os + i; }
  for (int r = 0; r < m; ++r) {
    A[r * n] = 1;
    for (int mm = 1; mm <= M; ++mm) {
      S c, s;
      g_sincos2pi<S>((long long)mm * tnum[r], (long long)P * n_os, &c, &s);
      A[r * n + 2 * mm - 1] = c;
      A[r * n + 2 * mm] = s;
    }
  }
  std::vector<S> Acopy = A;
  std::vector<std::vector<S>> rhs(d, std::vector<S>(m, S(0)));
  for (int k = 0; k < d; ++k)
    for (int i = 0; i < npt; ++i) rhs[k][i] = gram_val(k, S(tnum[i]) / S(n_os));
  std::vector<std::vector<S>> rhs0 = rhs, sol;
  lsq_solve<S>(A, m, n, rhs, &sol);
  // residuals
  double worst = 0;
  for (int k = 0; k < d; ++k) {
    S rr = 0, bb = 0;
    for (int r = 0; r < m; ++r) {
      S s = 0;
      for (int j = 0; j < n; ++j) s += Acopy[r * n + j] * sol[k][j];
      S e = s - rhs0[k][r];
      rr += e * e;
      bb += rhs0[k][r] * rhs0[k][r];
    }
    const double rel = (double)Sc<S>::sqrt(rr / bb);
    if (rel > worst) worst = rel;
  }
  // --- evaluate the continuations at t = d + j and form M_r = A_r Q^T
  std::vector<S> Ar(C * d);
  for (int j = 0; j < C; ++j) {
    std::vector<S> row(n);
    row[0] = 1;
    for (int mm = 1; mm <= M; ++mm) {
      S c, s;
      g_sincos2pi<S>((long long)mm * (d + j), P, &c, &s);
      row[2 * mm - 1] = c;
      row[2 * mm] = s;
    }
    for (int k = 0; k < d; ++k) {
      S s = 0;
      for (int jj = 0; jj < n; ++jj) s += row[jj] * sol[k][jj];
      Ar[j * d + k] = s;
    }
  }
  out->d = d; out->C = C; out->M = M; out->n_os = n_os;
  out->ls_residual = worst;
  out->Mr.assign(C * d, 0.0);
  for (int j = 0; j < C; ++j)
    for (int i = 0; i < d; ++i) {
      S s = 0;
      for (int k = 0; k < d; ++k) s += Ar[j * d + k] * Qm[i * d + k];
      out->Mr[j * d + i] = (double)s;
    }
  return true;
}

bool build_fc_tables(int d, int C, int M, int n_os, FcTables* out) {
  if (d < 2 || d > 10 || C < d || C > 64 || M < 1 || n_os < 1) return false;
  // Double-binary128 arithmetic (~67 digits) for every (d, C): binary128
  // alone leaves the (5, 25) fits ~17 correct digits, so about two thirds of
  // the entries round to the neighbouring double, and the continuation's
  // cancellation (row sums up to 1.2e4) turns those ulps into 1e-12 of the
  // continued values.  With ~67 digits every entry is the correctly rounded
  // double.  The tables of a (d, C, M, n_os) are built once per process.
  static std::mutex mtx;
  static std::map<std::tuple<int, int, int, int>, FcTables> cache;
  const auto key = std::make_tuple(d, C, M, n_os);
  {
    std::lock_guard<std::mutex> lk(mtx);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return true;
    }
  }
  FcTables T;
  if (!build_fc_tables_in<qq>(d, C, M, n_os, &T)) return false;
  std::lock_guard<std::mutex> lk(mtx);
  cache.emplace(key, T);
  *out = T;
  return true;
}

// direct DFT helpers on binary128 with a root table
struct Roots {
  int N;
  std::vector<q> c, s;  // exp(2 pi i m / N) = c[m] + i s[m]
  explicit Roots(int N_) : N(N_), c(N_), s(N_) {
    for (int m = 0; m < N; ++m) q_sincos2pi(m, N, &c[m], &s[m]);
  }
};

// spectrum of a real kernel h(j), j in [-(Np-1), Nz-1], placed circularly on L
static void kernel_spectrum(const std::vector<q>& h, int jlo, int L, std::vector<std::complex<double>>* H) {
  Roots rl(L);
  const int jhi = jlo + (int)h.size() - 1;
  H->assign(L, std::complex<double>(0, 0));
  for (int kk = 0; kk < L; ++kk) {
    q re = 0, im = 0;
    for (int j = jlo; j <= jhi; ++j) {
      long long mm = (((long long)j % L) + L) % L;
      long long e = (mm * kk) % L;
      re += h[j - jlo] * rl.c[e];
      im -= h[j - jlo] * rl.s[e];
    }
    (*H)[kk] = std::complex<double>((double)(re / (q)L), (double)(im / (q)L));
  }
}

void deriv_conv_spectra(int Nz, int Np, int L, std::vector<std::complex<double>>* H1,
                        std::vector<std::complex<double>>* H2) {
  if (L == Np) {
    // circular convolution of length N' itself: the spectra are the derivative
    // multipliers i k (Nyquist zeroed) and -k^2 of the N'-periodic unit grid, / N'
    H1->assign(L, 0);
    H2->assign(L, 0);
    const q twopi = 2 * q_pi();
    for (int l = 0; l < Np; ++l) {
      const int ls = (l <= (Np - 1) / 2) ? l : l - Np;
      const q k = twopi * (q)ls / (q)Np;
      const bool nyq = (Np % 2 == 0) && (l == Np / 2);
      (*H1)[l] = std::complex<double>(0.0, nyq ? 0.0 : (double)(k / (q)Np));
      (*H2)[l] = std::complex<double>((double)(-k * k / (q)Np), 0.0);
    }
    return;
  }
  Roots rn(Np);
  const q twopi = 2 * q_pi();
  // With L >= 2 N' - 1 the kernels are placed on the whole window
  // |j| <= N' - 1 (zeros between): d1 is odd and d2 even on it, so their
  // spectra are purely imaginary and purely real.  The outputs n < Nz only
  // use j in [-(N'-1), Nz-1], so they are the same either way.
  const bool sym = conv_symmetric(Np, L);
  const int jlo = -(Np - 1), jhi = sym ? Np - 1 : Nz - 1;
  std::vector<q> d1(jhi - jlo + 1), d2(jhi - jlo + 1);
  for (int j = jlo; j <= jhi; ++j) {
    q s1 = 0, s2 = 0;
    for (int l = 0; l < Np; ++l) {
      int ls = (l <= (Np - 1) / 2) ? l : l - Np;
      q k = twopi * (q)ls / (q)Np;
      long long m = ((long long)l * j) % Np;
      if (m < 0) m += Np;
      bool nyq = (Np % 2 == 0) && (l == Np / 2);
      if (!nyq) s1 += -k * rn.s[m];
      s2 += -k * k * rn.c[m];
    }
    d1[j - jlo] = s1 / (q)Np;
    d2[j - jlo] = s2 / (q)Np;
  }
  kernel_spectrum(d1, jlo, L, H1);
  kernel_spectrum(d2, jlo, L, H2);
  if (sym)
    for (int k = 0; k < L; ++k) {
      (*H1)[k] = std::complex<double>(0.0, (*H1)[k].imag());
      (*H2)[k] = std::complex<double>((*H2)[k].real(), 0.0);
    }
}

void filter_conv_spectrum(int Nz, int Np, int L, double beta, double two_p,
                          std::vector<std::complex<double>>* Hf) {
  Roots rn(Np);
  std::vector<q> fz(Np);
  for (int l = 0; l < Np; ++l) {
    int ls = (l <= (Np - 1) / 2) ? l : l - Np;
    if (Np % 2 == 0 && l == Np / 2) ls = -Np / 2;
    const double x = std::fabs((double)ls) / (Np / 2.0);
    fz[l] = (q)std::exp(-beta * std::pow(x, two_p));
  }
  if (L == Np) {  // circular convolution of length N' itself: the filter factors, / N'
    Hf->assign(L, 0);
    for (int l = 0; l < Np; ++l) (*Hf)[l] = std::complex<double>((double)(fz[l] / (q)Np), 0.0);
    return;
  }
  // symmetric placement as in deriv_conv_spectra: the kernel is even, its
  // spectrum real
  const bool sym = conv_symmetric(Np, L);
  const int jlo = -(Np - 1), jhi = sym ? Np - 1 : Nz - 1;
  std::vector<q> h(jhi - jlo + 1);
  for (int j = jlo; j <= jhi; ++j) {
    q s = 0;
    for (int l = 0; l < Np; ++l) {
      long long m = ((long long)l * j) % Np;
      if (m < 0) m += Np;
      s += fz[l] * rn.c[m];  // fz is even in l, so the kernel is real
    }
    h[j - jlo] = s / (q)Np;
  }
  kernel_spectrum(h, jlo, L, Hf);
  if (sym)
    for (int k = 0; k < L; ++k) (*Hf)[k] = std::complex<double>((*Hf)[k].real(), 0.0);
}

void z_kernels_real(int Nz, int Np, double beta, double two_p, std::vector<double>* d2, std::vector<double>* hf) {
  Roots rn(Np);
  const q twopi = 2 * q_pi();
  const int jlo = -(Np - 1), jhi = Nz - 1;
  std::vector<q> fz(Np);
  for (int l = 0; l < Np; ++l) {
    int ls = (l <= (Np - 1) / 2) ? l : l - Np;
    if (Np % 2 == 0 && l == Np / 2) ls = -Np / 2;
    fz[l] = (q)std::exp(-beta * std::pow(std::fabs((double)ls) / (Np / 2.0), two_p));
  }
  d2->assign(jhi - jlo + 1, 0.0);
  hf->assign(jhi - jlo + 1, 0.0);
  for (int j = jlo; j <= jhi; ++j) {
    q s2 = 0, sf = 0;
    for (int l = 0; l < Np; ++l) {
      const int ls = (l <= (Np - 1) / 2) ? l : l - Np;
      const q k = twopi * (q)ls / (q)Np;
      long long m = ((long long)l * j) % Np;
      if (m < 0) m += Np;
      s2 += -k * k * rn.c[m];
      sf += fz[l] * rn.c[m];
    }
    (*d2)[j - jlo] = (double)(s2 / (q)Np);
    (*hf)[j - jlo] = (double)(sf / (q)Np);
  }
}

void bluestein_tables(int Np, int L, std::vector<std::complex<double>>* chirp,
                      std::vector<std::complex<double>>* Hfwd, std::vector<std::complex<double>>* Hinv) {
  Roots rl(L);
  std::vector<q> wc(Np), ws(Np);  // chirp w_n = exp(-i pi n^2/Np) = exp(-2 pi i n^2 / (2 Np))
  for (int nn = 0; nn < Np; ++nn) {
    long long num = ((long long)nn * nn) % (2LL * Np);
    q c, s;
    q_sincos2pi(num, 2LL * Np, &c, &s);
    wc[nn] = c;
    ws[nn] = -s;
  }
  chirp->resize(Np);
  for (int nn = 0; nn < Np; ++nn) (*chirp)[nn] = std::complex<double>((double)wc[nn], (double)ws[nn]);
  // b[m mod L] = conj(w_|m|) for |m| < Np (forward); binv = w_|m|
  Hfwd->assign(L, 0);
  Hinv->assign(L, 0);
  for (int kk = 0; kk < L; ++kk) {
    q fr = 0, fi = 0, ir = 0, ii = 0;
    for (int m = -(Np - 1); m <= Np - 1; ++m) {
      int a = m < 0 ? -m : m;
      long long mm = (((long long)m % L) + L) % L;
      long long e = (mm * kk) % L;
      q c = rl.c[e], s = -rl.s[e];  // e^{-2 pi i mm kk / L}
      q br = wc[a], bi = -ws[a];   // conj(w)
      fr += br * c - bi * s;
      fi += br * s + bi * c;
      q vr = wc[a], vi = ws[a];    // w
      ir += vr * c - vi * s;
      ii += vr * s + vi * c;
    }
    (*Hfwd)[kk] = std::complex<double>((double)(fr / (q)L), (double)(fi / (q)L));
    (*Hinv)[kk] = std::complex<double>((double)(ir / (q)L), (double)(ii / (q)L));
  }
}

void split_twiddles(int N, std::vector<std::complex<double>>* tw) {
  tw->resize(N / 2 + 1);
  for (int k = 0; k <= N / 2; ++k) {
    q c, s;
    q_sincos2pi(k, N, &c, &s);
    (*tw)[k] = std::complex<double>((double)c, (double)-s);
  }
}

void engine_twiddles(int L1, int L2, std::vector<std::complex<double>>* tw) {
  const int L = L1 * L2;
  tw->resize(2 * L);
  for (int n2 = 0; n2 < L2; ++n2)
    for (int k1 = 0; k1 < L1; ++k1) {
      q c, s;
      q_sincos2pi((long long)n2 * k1, L, &c, &s);
      const std::complex<double> w((double)c, (double)-s);
      (*tw)[n2 * L1 + k1] = w;          // read by the k1-threads (B side)
      (*tw)[L + k1 * L2 + n2] = w;      // read by the n2-threads (A side)
    }
}

}  // namespace fcns
