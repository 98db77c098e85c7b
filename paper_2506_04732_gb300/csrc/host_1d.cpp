// Host-side FP64 construction of the 1D pieces of the collocation operator.
//
// Overview (i): Lagrange basis on the n = N+1 Gauss-Lobatto-Legendre (GLL)
// points (N-1 zeros of P_N' plus +-1).  Overview (ii) / Fig. 1: the equation is
// collocated on separate points that move from the zeros of P_N' (diffusion
// dominated) to N-1 of the zeros of P_N (convection dominated) as eps/|beta|
// falls.  The paper does not print the rule; this library takes the roots in
// (-1,1) of q(x) = eps P_N'(x) - beta P_N(x), which is the 1D operator
// beta d/dx - eps d^2/dx^2 applied to the GLL nodal polynomial (1-x^2) P_N'
// (up to a factor), so collocation there is exact on degree N+1.  For beta > 0
// the kept roots are bracketed one per interval (g_j, x_j) between the j-th
// Gauss point and the j-th interior GLL point; the N-th root, near the outflow
// end x = +1, is dropped.  beta < 0 is the mirror image.
#include "host_1d.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

namespace t2s2 {

// P_N(x), P_N'(x), P_N''(x) by the three-term recurrence.
static void legendre3(int N, double x, double* p, double* dp, double* ddp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, s0 = 0.0, s1 = 0.0;
  if (N == 0) { *p = 1.0; *dp = 0.0; *ddp = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    double s2 = s0 + (2.0 * k + 1.0) * d1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
  }
  *p = p1; *dp = d1; *ddp = s1;
}

void gll_points(int N, double* x) {
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre3(N, t, &p, &dp, &ddp);
      double step = dp / ddp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[j] = t;
  }
  // enforce exact symmetry
  for (int j = 0; j <= N / 2; ++j) {
    double a = 0.5 * (x[N - j] - x[j]);
    x[j] = -a;
    x[N - j] = a;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
}

void gauss_points(int N, double* g) {
  for (int j = 0; j < N; ++j) {
    double t = -std::cos(M_PI * (j + 0.5) / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre3(N, t, &p, &dp, &ddp);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    g[j] = t;
  }
}

// Root of q = eps P' - beta P in the bracket [lo, hi] (q(lo) q(hi) <= 0):
// Newton steps kept inside the bracket, bisection otherwise.
static double bracketed_root(int N, double eps, double beta, double lo, double hi) {
  auto q = [&](double t, double* dq) {
    double p, dp, ddp;
    legendre3(N, t, &p, &dp, &ddp);
    *dq = eps * ddp - beta * dp;
    return eps * dp - beta * p;
  };
  double dq;
  double qlo = q(lo, &dq), qhi = q(hi, &dq);
  if (qlo == 0.0) return lo;
  if (qhi == 0.0) return hi;
  double t = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double qt = q(t, &dq);
    if (qt == 0.0) return t;
    if ((qt < 0) == (qlo < 0)) { lo = t; qlo = qt; } else { hi = t; qhi = qt; }
    double tn = (dq != 0.0) ? t - qt / dq : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (std::fabs(tn - t) <= 4e-16 * std::max(1.0, std::fabs(t)) || hi - lo < 1e-16) return tn;
    t = tn;
  }
  return t;
}

void collocation_points(int N, double eps, double beta, int plain, double* eta) {
  double* x = new double[N + 1];
  gll_points(N, x);
  if (plain || beta == 0.0) {
    for (int j = 1; j < N; ++j) eta[j - 1] = x[j];
    delete[] x;
    return;
  }
  double* g = new double[N];
  gauss_points(N, g);
  double b = std::fabs(beta);
  // beta > 0: root j in (g_j, x_j), j = 1..N-1 (1-based GLL interior index).
  for (int j = 1; j < N; ++j) eta[j - 1] = bracketed_root(N, eps, b, g[j - 1], x[j]);
  if (beta < 0) {  // mirror: eta(-beta) = -reverse(eta(beta))
    for (int j = 0; j < (N - 1) / 2; ++j) std::swap(eta[j], eta[N - 2 - j]);
    for (int j = 0; j < N - 1; ++j) eta[j] = -eta[j];
  }
  delete[] g;
  delete[] x;
}

// l_i(t), l_i'(t), l_i''(t) for all i at one point t.  With f_m = t - x_m, the
// numerator prod_{m != i} f_m and its first two derivatives are accumulated
// factor by factor: e2 <- e2 f + e1, e1 <- e1 f + e0, e0 <- e0 f, so that
// prod' = e1 and prod'' = 2 e2; no division by t - x_m (exact at the nodes).
static void lagrange_at(int N, const double* x, const double* den, double t, double* l,
                        double* l1, double* l2) {
  for (int i = 0; i <= N; ++i) {
    double e0 = 1.0, e1 = 0.0, e2 = 0.0;
    for (int m = 0; m <= N; ++m) {
      if (m == i) continue;
      double f = t - x[m];
      e2 = e2 * f + e1;
      e1 = e1 * f + e0;
      e0 = e0 * f;
    }
    l[i] = e0 / den[i];
    l1[i] = e1 / den[i];
    l2[i] = 2.0 * e2 / den[i];
  }
}

void lagrange_matrices(int N, const double* x, int npts, const double* t, double* R, double* D,
                       double* D2) {
  double* den = new double[N + 1];
  for (int i = 0; i <= N; ++i) {
    double p = 1.0;
    for (int m = 0; m <= N; ++m)
      if (m != i) p *= (x[i] - x[m]);
    den[i] = p;
  }
  for (int j = 0; j < npts; ++j)
    lagrange_at(N, x, den, t[j], R + (size_t)j * (N + 1), D + (size_t)j * (N + 1),
                D2 + (size_t)j * (N + 1));
  delete[] den;
}

// In-place inverse of an m x m row-major matrix by Gauss-Jordan with partial
// pivoting.  Returns false if a pivot vanishes.
bool invert(int m, double* A) {
  int* perm = new int[m];
  double* W = new double[(size_t)m * 2 * m];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      W[(size_t)i * 2 * m + j] = A[(size_t)i * m + j];
      W[(size_t)i * 2 * m + m + j] = (i == j) ? 1.0 : 0.0;
    }
    perm[i] = i;
  }
  bool ok = true;
  for (int c = 0; c < m && ok; ++c) {
    int piv = c;
    for (int i = c + 1; i < m; ++i)
      if (std::fabs(W[(size_t)i * 2 * m + c]) > std::fabs(W[(size_t)piv * 2 * m + c])) piv = i;
    if (W[(size_t)piv * 2 * m + c] == 0.0) { ok = false; break; }
    if (piv != c)
      for (int j = 0; j < 2 * m; ++j) std::swap(W[(size_t)c * 2 * m + j], W[(size_t)piv * 2 * m + j]);
    double inv = 1.0 / W[(size_t)c * 2 * m + c];
    for (int j = 0; j < 2 * m; ++j) W[(size_t)c * 2 * m + j] *= inv;
    for (int i = 0; i < m; ++i) {
      if (i == c) continue;
      double f = W[(size_t)i * 2 * m + c];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * m; ++j) W[(size_t)i * 2 * m + j] -= f * W[(size_t)c * 2 * m + j];
    }
  }
  if (ok)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = W[(size_t)i * 2 * m + m + j];
  delete[] W;
  delete[] perm;
  return ok;
}

// Householder reduction to upper Hessenberg form: H = W^T B W, W orthogonal.
// B (m x m row-major) is overwritten by H; W is returned row-major.
void hessenberg(int m, double* B, double* W) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) W[(size_t)i * m + j] = (i == j) ? 1.0 : 0.0;
  double* v = new double[m];
  for (int k = 0; k + 2 < m; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < m; ++i) alpha += B[(size_t)i * m + k] * B[(size_t)i * m + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    double x0 = B[(size_t)(k + 1) * m + k];
    double s = (x0 >= 0) ? -alpha : alpha;  // reflect x to s e_1
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    v[k + 1] = x0 - s;
    for (int i = k + 2; i < m; ++i) v[i] = B[(size_t)i * m + k];
    double vn = 0.0;
    for (int i = k + 1; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    double tau = 2.0 / vn;
    // B <- P B P with P = I - tau v v^T (rows then columns); W <- W P
    for (int j = 0; j < m; ++j) {
      double s2 = 0.0;
      for (int i = k + 1; i < m; ++i) s2 += v[i] * B[(size_t)i * m + j];
      s2 *= tau;
      for (int i = k + 1; i < m; ++i) B[(size_t)i * m + j] -= s2 * v[i];
    }
    for (int i = 0; i < m; ++i) {
      double s2 = 0.0;
      for (int j = k + 1; j < m; ++j) s2 += B[(size_t)i * m + j] * v[j];
      s2 *= tau;
      for (int j = k + 1; j < m; ++j) B[(size_t)i * m + j] -= s2 * v[j];
    }
    for (int i = 0; i < m; ++i) {
      double s2 = 0.0;
      for (int j = k + 1; j < m; ++j) s2 += W[(size_t)i * m + j] * v[j];
      s2 *= tau;
      for (int j = k + 1; j < m; ++j) W[(size_t)i * m + j] -= s2 * v[j];
    }
    for (int i = k + 2; i < m; ++i) B[(size_t)i * m + k] = 0.0;
  }
  delete[] v;
}

// Complex Schur form A = Z T Z^H (T upper triangular, Z unitary) of a real
// m x m matrix: Householder reduction to Hessenberg form, then single-shift
// QR sweeps (bulge chasing with Givens rotations) with Wilkinson shifts and
// deflation of negligible subdiagonal entries.  Unitary transformations only,
// so the form is backward stable however non-normal A is.
bool complex_schur(int m, const double* A, std::complex<double>* T, std::complex<double>* Z) {
  typedef std::complex<double> C;
  std::vector<double> H(A, A + (size_t)m * m), W((size_t)m * m);
  hessenberg(m, H.data(), W.data());
  for (size_t e = 0; e < (size_t)m * m; ++e) {
    T[e] = C(H[e], 0.0);
    Z[e] = C(W[e], 0.0);
  }
  auto t = [&](int i, int j) -> C& { return T[(size_t)i * m + j]; };
  auto z = [&](int i, int j) -> C& { return Z[(size_t)i * m + j]; };
  const double eps = 2.220446049250313e-16;
  int hi = m - 1, iter = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double sub = std::abs(t(l, l - 1));
      double diag = std::abs(t(l - 1, l - 1)) + std::abs(t(l, l));
      if (sub <= eps * (diag > 0 ? diag : 1.0)) {
        t(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // 1 x 1 block converged
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 100 * m) return false;
    ++iter;
    C mu;
    if (iter % 11 == 0) {  // exceptional shift
      mu = t(hi, hi) + C(0.75 * std::abs(t(hi, hi - 1)), 0.0);
    } else {
      C a = t(hi - 1, hi - 1), b = t(hi - 1, hi), c = t(hi, hi - 1), d = t(hi, hi);
      C half = 0.5 * (a - d);
      C disc = std::sqrt(half * half + b * c);
      C l1 = 0.5 * (a + d) + disc, l2 = 0.5 * (a + d) - disc;
      mu = (std::abs(l1 - d) < std::abs(l2 - d)) ? l1 : l2;
    }
    C x = t(l, l) - mu, y = t(l + 1, l);
    for (int k = l; k < hi; ++k) {
      double ax = std::abs(x), ay = std::abs(y);
      double r = std::hypot(ax, ay);
      double c;
      C s;
      if (r == 0.0) {
        c = 1.0;
        s = 0.0;
      } else if (ax == 0.0) {
        c = 0.0;
        s = std::conj(y) / ay;
      } else {
        c = ax / r;
        s = (x / ax) * std::conj(y) / r;
      }
      // rows k, k+1 from column max(l, k-1): G = [[c, s], [-conj(s), c]]
      for (int j = std::max(l, k - 1); j < m; ++j) {
        C u = t(k, j), v = t(k + 1, j);
        t(k, j) = c * u + s * v;
        t(k + 1, j) = -std::conj(s) * u + c * v;
      }
      // columns k, k+1 (right multiplication by G^H), rows up to min(k+2, hi)
      int rmax = std::min(k + 2, hi);
      for (int i = 0; i <= rmax; ++i) {
        C u = t(i, k), v = t(i, k + 1);
        t(i, k) = c * u + std::conj(s) * v;
        t(i, k + 1) = -s * u + c * v;
      }
      for (int i = 0; i < m; ++i) {
        C u = z(i, k), v = z(i, k + 1);
        z(i, k) = c * u + std::conj(s) * v;
        z(i, k + 1) = -s * u + c * v;
      }
      if (k + 2 <= hi) {
        x = t(k + 1, k);
        y = t(k + 2, k);
      }
    }
  }
  for (int i = 1; i < m; ++i)
    for (int j = 0; j < i; ++j) t(i, j) = 0.0;
  return true;
}

// Interpolation inverse, B = Rt^{-1} Lt and B's complex Schur form, from the
// m x m matrices Rt and Lt already in *out.
static bool finish_dimension(int m, Dim1D* out) {
  out->Rinv = out->Rt;
  if (!invert(m, out->Rinv.data())) return false;
  out->B.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int l = 0; l < m; ++l) s += out->Rinv[(size_t)i * m + l] * out->Lt[(size_t)l * m + j];
      out->B[(size_t)i * m + j] = s;
    }
  std::vector<std::complex<double>> T((size_t)m * m), Z((size_t)m * m);
  if (!complex_schur(m, out->B.data(), T.data(), Z.data())) return false;
  out->Tr.resize((size_t)m * m);
  out->Ti.resize((size_t)m * m);
  out->Zr.resize((size_t)m * m);
  out->Zi.resize((size_t)m * m);
  for (size_t e = 0; e < (size_t)m * m; ++e) {
    out->Tr[e] = T[e].real();
    out->Ti[e] = T[e].imag();
    out->Zr[e] = Z[e].real();
    out->Zi[e] = Z[e].imag();
  }
  return true;
}

bool build_dimension(int n, double eps, double beta, int plain, Dim1D* out) {
  return build_dimension_coef(n, eps, beta, plain, {}, {}, out);
}

bool build_dimension_coef(int n, double eps, double beta_ref, int plain, const std::function<double(double)>& beta_at,
                          const std::function<double(double)>& rho_at, Dim1D* out) {
  const int N = n - 1, m = n - 2;
  out->n = n;
  out->x.assign(n, 0.0);
  out->eta.assign(m, 0.0);
  gll_points(N, out->x.data());
  collocation_points(N, eps, beta_ref, plain, out->eta.data());
  std::vector<double> R((size_t)m * n), D((size_t)m * n), D2((size_t)m * n);
  lagrange_matrices(N, out->x.data(), m, out->eta.data(), R.data(), D.data(), D2.data());
  out->Rt.assign((size_t)m * m, 0.0);
  out->Lt.assign((size_t)m * m, 0.0);
  out->Rf.assign((size_t)m * n, 0.0);
  out->Lf.assign((size_t)m * n, 0.0);
  for (int j = 0; j < m; ++j) {
    const double bj = beta_at ? beta_at(out->eta[j]) : beta_ref;
    const double rj = rho_at ? rho_at(out->eta[j]) : 0.0;
    if (!std::isfinite(bj) || !std::isfinite(rj)) return false;
    for (int i = 0; i < n; ++i) {
      const size_t e = (size_t)j * n + i;
      out->Rf[e] = R[e];
      out->Lf[e] = bj * D[e] - eps * D2[e] + rj * R[e];
    }
    for (int i = 0; i < m; ++i) {
      out->Rt[(size_t)j * m + i] = out->Rf[(size_t)j * n + i + 1];
      out->Lt[(size_t)j * m + i] = out->Lf[(size_t)j * n + i + 1];
    }
  }
  return finish_dimension(m, out);
}

bool build_time_dimension(int n, double scale, Dim1D* out) {
  const int N = n - 1, m = n - 1;
  out->n = n;
  out->x.assign(n, 0.0);
  out->eta.assign(m, 0.0);
  gll_points(N, out->x.data());
  gauss_points(N, out->eta.data());
  std::vector<double> R((size_t)m * n), D((size_t)m * n), D2((size_t)m * n);
  lagrange_matrices(N, out->x.data(), m, out->eta.data(), R.data(), D.data(), D2.data());
  out->Rt.assign((size_t)m * m, 0.0);
  out->Lt.assign((size_t)m * m, 0.0);
  out->R0.assign(m, 0.0);
  out->L0.assign(m, 0.0);
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) {
      out->Rt[(size_t)j * m + i] = R[(size_t)j * n + i + 1];
      out->Lt[(size_t)j * m + i] = scale * D[(size_t)j * n + i + 1];
    }
    out->R0[j] = R[(size_t)j * n];
    out->L0[j] = scale * D[(size_t)j * n];
  }
  return finish_dimension(m, out);
}

}  // namespace t2s2
