// Host-side table construction in binary128 (_Float128).
#pragma once
#include <complex>
#include <vector>

namespace fcns {

struct FcTables {
  int d = 0, C = 0, M = 0, n_os = 0;
  std::vector<double> Mr;  // C x d row-major, right-end continuation matrix
  double ls_residual = 0;  // largest relative least-squares residual
};

// Gram-basis FC tables (App. B): QR of the Vandermonde on the d matching
// points, oversampled trigonometric least squares per Gram polynomial,
// M_r = A_r Q_r^T.  Returns false on invalid sizes.
bool build_fc_tables(int d, int C, int M, int n_os, FcTables* out);

// Whether the circular kernels of the z operators can be placed on the whole
// symmetric window |j| <= N' - 1 (L >= 2 N' - 1) or are the multipliers of
// length N' itself (L = N'): then the spectra of the derivative kernels are
// purely imaginary (d/dz) and purely real (d2/dz2, the filter).
inline bool conv_symmetric(int Np, int L) { return L == Np || L >= 2 * Np - 1; }

// Spectra (length L, with 1/L) of the circular kernels of d/dz and d2/dz2 on
// the N'-periodic unit grid (first Nz outputs valid).  L >= N' + Nz - 1
// (padded circular convolution) or L = N' (the multipliers i k, -k^2 / N').
// When conv_symmetric(N', L), H1 has zero real parts and H2 zero imaginary
// parts.
void deriv_conv_spectra(int Nz, int Np, int L, std::vector<std::complex<double>>* H1,
                        std::vector<std::complex<double>>* H2);

// Spectrum (length L, with 1/L) of the circular kernel of the z filter
// fz(l) = exp(-beta (|l_s| / (N'/2))^{2p}) on the N'-periodic grid (real
// when conv_symmetric(N', L)).
void filter_conv_spectrum(int Nz, int Np, int L, double beta, double two_p,
                          std::vector<std::complex<double>>* Hf);

// Real-space kernels on the N'-periodic unit grid, indexed by j + N' - 1 for
// j in [-(N'-1), Nz-1]: d2 (second derivative) and hf (the z filter), so that
// (K * x)[n] = sum_m K(n - m) x[m] for n < Nz, m < N'.
void z_kernels_real(int Nz, int Np, double beta, double two_p, std::vector<double>* d2, std::vector<double>* hf);

// Bluestein tables for a length-Np DFT done with length-L transforms:
// chirp[n] = exp(-i pi n^2 / Np) (n < Np) and the spectrum (with 1/L) of the
// circular kernel b[m mod L] = conj(chirp[|m|]), |m| < Np.  For the inverse
// DFT use conj(chirp) and the spectrum of chirp[|m|] (Hinv).
void bluestein_tables(int Np, int L, std::vector<std::complex<double>>* chirp,
                      std::vector<std::complex<double>>* Hfwd, std::vector<std::complex<double>>* Hinv);

// Twiddles exp(-2 pi i n2 k1 / L), L = L1 L2, stored twice: tw[n2 * L1 + k1]
// and tw[L + k1 * L2 + n2], so that both thread roles read them contiguously.
void engine_twiddles(int L1, int L2, std::vector<std::complex<double>>* tw);
// e^{-2 pi i k / N}, k = 0 .. N/2 (computed in binary128, rounded to double)
void split_twiddles(int N, std::vector<std::complex<double>>* tw);

// cos / sin of 2 pi num / den, correctly rounded to double from binary128.
void sincos2pi(long long num, long long den, double* c, double* s);

}  // namespace fcns
