// Register-resident small DFTs with compile-time twiddles.
//
// A length N with coprime factors N = A B (A a power of 2 or 3, B the rest) is
// split by the prime-factor (Good-Thomas) index maps, which need no twiddle
// factors at all: the maps are compile-time register renamings.  A prime-power
// length R1 R2 ... Rm is done as m Stockham autosort passes over a register
// array (all indices compile-time constants after template expansion, so the
// arrays stay in registers).  Twiddle factors are evaluated at compile time by
// kcos2pi/ksin2pi (octant reduction + Taylor series written out below), so
// they become immediates; powers of i become swaps and sign changes.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

namespace fcns {

template <class T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };
template <class T> using cx = typename V2<T>::t;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <class C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// float complex add / subtract / real scaling as one packed 2 x fp32 instruction
// (sm_100 family), rounded to nearest like the scalar forms
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
#endif
template <class C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <class C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <class C, class S> __host__ __device__ __forceinline__ C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
template <> __device__ __forceinline__ float2 cscale<float2, float>(float2 a, float s) {
  return __fmul2_rn(a, make_float2(s, s));
}
#endif
// multiply by sign * i
template <int SIGN, class C> __host__ __device__ __forceinline__ C mul_si(C a) {
  C r;
  if (SIGN > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
// a * s + c for complex a, c and real s: one fused multiply-add per component
// (one packed 2 x fp32 instruction on sm_100 family parts)
template <class C, class S> __host__ __device__ __forceinline__ C cfma_s(C a, S s, C c) {
  C r; r.x = a.x * s + c.x; r.y = a.y * s + c.y; return r;
}
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
template <> __device__ __forceinline__ float2 cfma_s<float2, float>(float2 a, float s, float2 c) {
  return __ffma2_rn(a, make_float2(s, s), c);
}
#endif
// t + SIGN i s d for complex t, d and real s, as two scalar fused
// multiply-adds (the rotation by i swaps the components, which a packed
// instruction cannot do without extra moves)
template <int SIGN, class C, class S> __host__ __device__ __forceinline__ C add_rot(C t, C d, S s) {
  C r;
#if defined(__CUDA_ARCH__)
  if constexpr (sizeof(S) == 4) {
    r.x = __fmaf_rn(S(-SIGN) * s, d.y, t.x);
    r.y = __fmaf_rn(S(SIGN) * s, d.x, t.y);
  } else {
    r.x = fma(S(-SIGN) * s, d.y, t.x);
    r.y = fma(S(SIGN) * s, d.x, t.y);
  }
#else
  r.x = t.x + S(-SIGN) * s * d.y;
  r.y = t.y + S(SIGN) * s * d.x;
#endif
  return r;
}
// t + SIGN i d (no scaling): two scalar adds
template <int SIGN, class C> __host__ __device__ __forceinline__ C add_i(C t, C d) {
  C r;
  if (SIGN > 0) { r.x = t.x - d.y; r.y = t.y + d.x; } else { r.x = t.x + d.y; r.y = t.y - d.x; }
  return r;
}

// ---------------------------------------------------------------------------
// compile-time cos / sin of 2 pi num / den
// ---------------------------------------------------------------------------
constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr double taylor_sin(double x) {  // |x| <= pi/4
  double x2 = x * x, term = x, sum = x;
  for (int n = 1; n < 14; ++n) { term *= -x2 / double((2 * n) * (2 * n + 1)); sum += term; }
  return sum;
}
constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int n = 1; n < 14; ++n) { term *= -x2 / double((2 * n - 1) * (2 * n)); sum += term; }
  return sum;
}
// Nearest quarter turn m, residual fraction rho in [-1/8, 1/8] of a turn.
constexpr void quarter_reduce(long long num, long long den, int& m, double& psi) {
  long long r = ((num % den) + den) % den;       // [0, den)
  long long m4 = (4 * r * 2 + den) / (2 * den);  // round(4 r / den)
  long long resid = 4 * r - m4 * den;            // in [-den/2, den/2]
  m = int(m4 & 3);
  psi = kTwoPi * (double(resid) / double(4 * den));
}
constexpr double kcos2pi(long long num, long long den) {
  int m = 0; double psi = 0;
  quarter_reduce(num, den, m, psi);
  return m == 0 ? taylor_cos(psi) : m == 1 ? -taylor_sin(psi) : m == 2 ? -taylor_cos(psi) : taylor_sin(psi);
}
constexpr double ksin2pi(long long num, long long den) {
  int m = 0; double psi = 0;
  quarter_reduce(num, den, m, psi);
  return m == 0 ? taylor_sin(psi) : m == 1 ? taylor_cos(psi) : m == 2 ? -taylor_sin(psi) : -taylor_cos(psi);
}

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------
template <int I, int E> struct SFor {
  template <class F> __host__ __device__ __forceinline__ static void run(F&& f) {
    if constexpr (I < E) {
      f(std::integral_constant<int, I>{});
      SFor<I + 1, E>::run(f);
    }
  }
};

// ---------------------------------------------------------------------------
// radix butterflies (natural order in / out), SIGN = -1 forward, +1 inverse
// ---------------------------------------------------------------------------
template <int R, int SIGN, class T> struct Radix;

template <int SIGN, class T> struct Radix<2, SIGN, T> {
  __host__ __device__ __forceinline__ static void run(cx<T>* v) {
    cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};
template <int SIGN, class T> struct Radix<3, SIGN, T> {
  __host__ __device__ __forceinline__ static void run(cx<T>* v) {
    constexpr T s = T(0.86602540378443864676372317075294);  // sin(2 pi / 3)
    cx<T> a = v[0], b = v[1], c = v[2];
    cx<T> t1 = cadd(b, c);
    cx<T> dd = csub(b, c);
    cx<T> t2 = cfma_s(t1, T(-0.5), a);   // a - t1 / 2
    v[0] = cadd(a, t1);
    v[1] = add_rot<SIGN>(t2, dd, s);      // t2 + SIGN i s (b - c)
    v[2] = add_rot<-SIGN>(t2, dd, s);
  }
};
template <int SIGN, class T> struct Radix<4, SIGN, T> {
  __host__ __device__ __forceinline__ static void run(cx<T>* v) {
    cx<T> a = v[0], b = v[1], c = v[2], d = v[3];
    cx<T> s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = mul_si<SIGN>(csub(b, d));
    v[0] = cadd(s0, s1); v[2] = csub(s0, s1);
    v[1] = cadd(d0, d1); v[3] = csub(d0, d1);
  }
};
template <int SIGN, class T> struct Radix<5, SIGN, T> {
  __host__ __device__ __forceinline__ static void run(cx<T>* v) {
    constexpr T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi/5)
    constexpr T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi/5)
    constexpr T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi/5)
    constexpr T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi/5)
    cx<T> a0 = v[0];
    cx<T> p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    cx<T> p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    cx<T> r1 = cfma_s(p2, c2, cfma_s(p1, c1, a0));      // a0 + c1 p1 + c2 p2
    cx<T> r2 = cfma_s(p2, c1, cfma_s(p1, c2, a0));      // a0 + c2 p1 + c1 p2
    cx<T> i1 = cfma_s(m2, s2, cscale(m1, s1));          // s1 m1 + s2 m2
    cx<T> i2 = cfma_s(m2, -s1, cscale(m1, s2));         // s2 m1 - s1 m2
    v[0] = cadd(a0, cadd(p1, p2));
    v[1] = add_i<SIGN>(r1, i1); v[4] = add_i<-SIGN>(r1, i1);
    v[2] = add_i<SIGN>(r2, i2); v[3] = add_i<-SIGN>(r2, i2);
  }
};

// ---------------------------------------------------------------------------
// radix schedule: prefer 4, then 2, 3, 5
// ---------------------------------------------------------------------------
constexpr int first_radix(int n) {
  return (n % 4 == 0 && n != 8) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : n;
}
constexpr bool smooth235(int n) {
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

// One Stockham pass with radix R at stage Ns over arrays in -> out (length N).
template <int N, int R, int NS, int SIGN, class T>
__host__ __device__ __forceinline__ void stockham_pass(const cx<T>* in, cx<T>* out) {
  SFor<0, N / R>::run([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    cx<T> v[R];
    SFor<0, R>::run([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      v[r] = in[j + r * (N / R)];
      if constexpr (NS > 1 && r > 0 && ((j % NS) * r) != 0) {
        constexpr long long num = (long long)r * (j % NS);
        constexpr long long den = (long long)NS * R;
        if constexpr ((4 * num) % den == 0) {
          // e^{SIGN 2 pi i q / 4} = (SIGN i)^q
          constexpr int q = int(((4 * num) / den) % 4);
          if constexpr (q == 1) v[r] = mul_si<SIGN>(v[r]);
          else if constexpr (q == 2) v[r] = mk<T>(-v[r].x, -v[r].y);
          else if constexpr (q == 3) v[r] = mul_si<-SIGN>(v[r]);
        } else {
          constexpr T c = T(kcos2pi(num, den));
          constexpr T s = T(SIGN * ksin2pi(num, den));
          v[r] = cmul(v[r], mk<T>(c, s));
        }
      }
    });
    Radix<R, SIGN, T>::run(v);
    constexpr int idxD = (j / NS) * NS * R + (j % NS);
    SFor<0, R>::run([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      out[idxD + r * NS] = v[r];
    });
  });
}

template <int N, int REM, int NS, int SIGN, class T>
__host__ __device__ __forceinline__ void stockham_all(cx<T>* a) {
  if constexpr (REM > 1) {
    constexpr int R = first_radix(REM);
    static_assert(R == 2 || R == 3 || R == 4 || R == 5, "length must be 2^a 3^b 5^c");
    cx<T> tmp[N];
    stockham_pass<N, R, NS, SIGN, T>(a, tmp);
    SFor<0, N>::run([&](auto ic) { constexpr int i = decltype(ic)::value; a[i] = tmp[i]; });
    stockham_all<N, REM / R, NS * R, SIGN, T>(a);
  }
}

// Coprime split for the prime-factor algorithm: A = the 2-part of N, else
// its 3-part; 0 when N is a prime power (no split).
constexpr int prime_part(int n, int p) {
  int r = 1;
  while (n % p == 0) { n /= p; r *= p; }
  return r;
}
constexpr int pfa_split(int n) {
  const int a2 = prime_part(n, 2), a3 = prime_part(n, 3), a5 = prime_part(n, 5);
  const int parts = (a2 > 1) + (a3 > 1) + (a5 > 1);
  return parts < 2 ? 0 : (a2 > 1 ? a2 : a3);
}
// a^{-1} mod m for coprime a, m (m >= 2)
constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 0;
}

template <int N, int SIGN, class T>
__host__ __device__ __forceinline__ void dft_reg(cx<T> (&a)[N]);

// Good-Thomas: n = (ia B + ib A) mod N, k = the residue pair (k mod A, k mod B),
// so e^{-2 pi i nk/N} = e^{-2 pi i ia ka/A} e^{-2 pi i ib kb/B} and the
// transform is a plain A x B two-dimensional DFT.
template <int N, int A, int SIGN, class T>
__host__ __device__ __forceinline__ void pfa_reg(cx<T> (&a)[N]) {
  constexpr int B = N / A;
  cx<T> t[B][A];
  SFor<0, B>::run([&](auto bc) {
    constexpr int ib = decltype(bc)::value;
    SFor<0, A>::run([&](auto ac) {
      constexpr int ia = decltype(ac)::value;
      t[ib][ia] = a[(ia * B + ib * A) % N];
    });
    dft_reg<A, SIGN, T>(t[ib]);
  });
  constexpr int eA = B * inv_mod(B % A, A), eB = A * inv_mod(A % B, B);  // CRT idempotents
  SFor<0, A>::run([&](auto ac) {
    constexpr int ka = decltype(ac)::value;
    cx<T> u[B];
    SFor<0, B>::run([&](auto bc) {
      constexpr int ib = decltype(bc)::value;
      u[ib] = t[ib][ka];
    });
    dft_reg<B, SIGN, T>(u);
    SFor<0, B>::run([&](auto bc) {
      constexpr int kb = decltype(bc)::value;
      a[(ka * eA + kb * eB) % N] = u[kb];
    });
  });
}

// In-place DFT of length N on a register array, natural order in and out.
// SIGN = -1: X_k = sum x_n e^{-2 pi i nk/N};  SIGN = +1: unnormalised inverse.
template <int N, int SIGN, class T>
__host__ __device__ __forceinline__ void dft_reg(cx<T> (&a)[N]) {
  static_assert(smooth235(N), "register DFT needs a 2/3/5-smooth length");
  constexpr int A = pfa_split(N);
  if constexpr (A > 1) pfa_reg<N, A, SIGN, T>(a);
  else stockham_all<N, N, 1, SIGN, T>(a);
}

}  // namespace fcns

namespace fcns {

// ---------------------------------------------------------------------------
// compensated ("float-float") dot products: a value is hi + lo with |lo| <=
// ulp(hi)/2.  Used where a float32 path needs float64-level accuracy (the
// FC continuation product, whose weights reach 4e3 and cancel) without the
// float64 pipe, which is slow on this part.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

// s += (mhi + mlo) * x, exactly up to float-float rounding.  On the device
// every operation of the error-free product / sum is an explicitly rounded
// intrinsic: the compiler must not contract p into the following sum (an
// FMA there would make t differ from s.hi + p and the correction term
// meaningless).
__host__ __device__ __forceinline__ void ff_fma(ff& s, float mhi, float mlo, float x) {
#if defined(__CUDA_ARCH__)
  const float p = __fmul_rn(mhi, x);
  const float e = __fmaf_rn(mhi, x, -p);
  const float t = __fadd_rn(s.hi, p);
  const float z = __fsub_rn(t, s.hi);
  const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(__fadd_rn(err, e), __fmul_rn(mlo, x)));
#else
  const float p = mhi * x;
  const float e = (float)((double)mhi * (double)x - (double)p);  // exact: 48-bit product
  const float t = s.hi + p;
  const float z = t - s.hi;
  const float err = (s.hi - (t - z)) + (p - z);
  s.hi = t;
  s.lo += err + e + mlo * x;
#endif
}

__host__ __device__ __forceinline__ float ff_round(const ff& s) { return s.hi + s.lo; }

// The same compensated sum in double (a "double-double" accumulator): the
// float64 path's continuation product, whose weights reach 4e3 and cancel, so
// that plain double sums would put ~1e-12 |f| of rounding into the continued
// values, which the second derivative amplifies near the walls.
struct dd {
  double hi, lo;
};
__host__ __device__ __forceinline__ void dd_fma(dd& s, double m, double x) {
#if defined(__CUDA_ARCH__)
  const double p = __dmul_rn(m, x);
  const double e = __fma_rn(m, x, -p);
  const double t = __dadd_rn(s.hi, p);
  const double z = __dsub_rn(t, s.hi);
  const double err = __dadd_rn(__dsub_rn(s.hi, __dsub_rn(t, z)), __dsub_rn(p, z));
  s.hi = t;
  s.lo = __dadd_rn(s.lo, __dadd_rn(err, e));
#else
  const double p = m * x;
  const double e = fma(m, x, -p);
  const double t = s.hi + p;
  const double z = t - s.hi;
  const double err = (s.hi - (t - z)) + (p - z);
  s.hi = t;
  s.lo += err + e;
#endif
}
__host__ __device__ __forceinline__ double dd_round(const dd& s) { return s.hi + s.lo; }

}  // namespace fcns
