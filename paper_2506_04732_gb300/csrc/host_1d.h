// Host-side FP64 construction of the per-dimension collocation matrices.
#pragma once
#include <complex>
#include <functional>
#include <vector>

namespace t2s2 {

struct Dim1D {
  int n = 0;                 // GLL nodes (polynomial degree n-1); m = n-2 interior unknowns (n-1 for time)
  std::vector<double> x;     // n GLL points
  std::vector<double> eta;   // m collocation points
  std::vector<double> Rt;    // m x m: l_i(eta_j), interior i
  std::vector<double> Lt;    // m x m: beta l_i'(eta_j) - eps l_i''(eta_j)
  std::vector<double> Rinv;  // Rt^{-1}
  std::vector<double> B;     // Rt^{-1} Lt
  std::vector<double> Tr, Ti;  // complex Schur form of B: B = Z T Z^H, T upper triangular
  std::vector<double> Zr, Zi;  // unitary Schur basis
  std::vector<double> R0, L0;  // time dimension only: the columns of the initial node s = -1
  std::vector<double> Rf, Lf;  // space dimensions: m x n, every GLL node a column (boundary data)
};

void gll_points(int N, double* x);
void gauss_points(int N, double* g);
void collocation_points(int N, double eps, double beta, int plain, double* eta);
void lagrange_matrices(int N, const double* x, int npts, const double* t, double* R, double* D,
                       double* D2);
bool invert(int m, double* A);
void hessenberg(int m, double* B, double* W);
bool complex_schur(int m, const double* A, std::complex<double>* T, std::complex<double>* Z);
bool build_dimension(int n, double eps, double beta, int plain, Dim1D* out);
// As build_dimension with variable coefficients: the collocation points are
// those of the reference speed beta_ref; at collocation point eta_j the rows
// of D are scaled by beta_at(eta_j) (empty: beta_ref) and rho_at(eta_j) Rt
// (empty: zero) is added, Lt = diag(beta(eta)) D - eps D2 + diag(rho(eta)) Rt.
// False if a coefficient is not finite.
bool build_dimension_coef(int n, double eps, double beta_ref, int plain, const std::function<double(double)>& beta_at,
                          const std::function<double(double)>& rho_at, Dim1D* out);
// The time dimension of the space-time form: m = n-1 unknowns (all GLL nodes
// but s = -1), collocation at the n-1 Gauss points, Lt = scale * D.
bool build_time_dimension(int n, double scale, Dim1D* out);

}  // namespace t2s2
