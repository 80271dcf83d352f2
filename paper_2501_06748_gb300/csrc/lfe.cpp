// The low-frequency expansion of the reduced element equation (Section 3.2), the
// paper's comparison method: with the density constant along every radial line the
// coefficient matrices E0, E1, E2, M0 do not depend on xi, and the element's dynamic
// stiffness is expanded as S ~ K - omega^2 M with
//
//   K from the algebraic Riccati equation (K - E1) E0^-1 (K - E1^T) - E2 = 0, and
//   M from the Lyapunov equation (K - E1) E0^-1 M + M E0^-1 (K - E1^T) + 2 M - M0 = 0.
//
// Riccati: with q = xi E0 u_xi + E1^T u (Eq. (internal)) the static equation is
// xi d/dxi [u; q] = -Z [u; q], Z = [[E0^-1 E1^T, -E0^-1], [-E2 + E1 E0^-1 E1^T, -E1 E0^-1]];
// the solutions bounded at the scaling centre span the invariant subspace of Z's
// eigenvalues with negative real part plus the constant mode u = 1, q = 0 (its double
// zero eigenvalue is exact because E1^T 1 = E2 1 = 0), and K = Q_q Q_u^-1 for a basis
// [Q_u; Q_q] of it.  The stable subspace is found without eigenvectors, as the range of
// (I - sign(Z + sigma I)) / 2 with the matrix sign function by the scaled Newton
// iteration X <- (c X + (c X)^-1) / 2 (Roberts' method); the shift sigma = 1/2 moves the
// zero pair to the right half-plane while the stable eigenvalues, whose real parts are
// at most -1 for these operators (the linear fields u ~ xi x, xi y give -1), stay left.
// The projector's rank must be n_b - 1 (the stable eigenvalues, the constant mode's pair
// being shifted to the right): its trace and the pivoted Gram-Schmidt basis are checked,
// and an element whose spectrum does not split that way is refused (SBFWI_ESINGULAR)
// rather than given a wrong subspace.
// Lyapunov: with F = (K - E1) E0^-1 + I and G = E0^-1 (K - E1^T) + I the equation reads
// F M + M G = M0.  G's eigenvalues are 1 + the exponents lambda >= 0 of the bounded modes
// u ~ xi^lambda (G u = (1 + lambda) u, since xi u_xi = E0^-1 (K - E1^T) u on them), and F
// shares them, so both spectra lie at or right of 1 and M = C_inf / 2 from the coupled
// Newton sign iteration F <- (F + F^-1)/2, G <- (G + G^-1)/2, C <- (C + F^-1 C G^-1)/2
// (Roberts' method for Sylvester equations), O(n_b^3) per step.  Host code, FP64: this is
// per-model set-up of the comparison method, not part of the time loop.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace sbfwi {
namespace {

// LU with partial pivoting of the n x n row-major A (in place); false if singular
bool lu_factor(std::vector<double>& A, std::vector<int>& piv, int n) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + k]) > best) { best = std::fabs(A[(size_t)r * n + k]); p = r; }
    if (!(best > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int c = 0; c < n; ++c) std::swap(A[(size_t)k * n + c], A[(size_t)p * n + c]);
    const double inv = 1.0 / A[(size_t)k * n + k];
    for (int r = k + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + k] * inv;
      A[(size_t)r * n + k] = f;
      if (f != 0.0)
        for (int c = k + 1; c < n; ++c) A[(size_t)r * n + c] -= f * A[(size_t)k * n + c];
    }
  }
  return true;
}

void lu_solve(const std::vector<double>& LU, const std::vector<int>& piv, int n, double* b) {
  for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
  for (int r = 1; r < n; ++r) {
    double s = b[r];
    for (int c = 0; c < r; ++c) s -= LU[(size_t)r * n + c] * b[c];
    b[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < n; ++c) s -= LU[(size_t)r * n + c] * b[c];
    b[r] = s / LU[(size_t)r * n + r];
  }
}

bool inverse(const std::vector<double>& A, std::vector<double>& inv, int n, double* logdet = nullptr) {
  std::vector<double> LU(A);
  std::vector<int> piv;
  if (!lu_factor(LU, piv, n)) return false;
  if (logdet) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += std::log(std::fabs(LU[(size_t)k * n + k]));
    *logdet = s;
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    std::fill(col.begin(), col.end(), 0.0);
    col[c] = 1.0;
    lu_solve(LU, piv, n, col.data());
    for (int r = 0; r < n; ++r) inv[(size_t)r * n + c] = col[r];
  }
  return true;
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int n, int k, int m) {
  std::vector<double> C((size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[(size_t)i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < m; ++j) C[(size_t)i * m + j] += a * B[(size_t)l * m + j];
    }
  return C;
}

}  // namespace

int lfe_element(const double* E0, const double* E1, const double* E2, const double* M0, int nb, double* Kout,
                double* Mout) {
  const int n = nb, n2 = 2 * nb;
  std::vector<double> e0(E0, E0 + (size_t)n * n), e1(E1, E1 + (size_t)n * n), e2(E2, E2 + (size_t)n * n);
  std::vector<double> e1t((size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) e1t[(size_t)r * n + c] = e1[(size_t)c * n + r];
  std::vector<double> e0i;
  if (!inverse(e0, e0i, n)) return fail(SBFWI_ESINGULAR, "E0 of an element is singular");
  const std::vector<double> a11 = matmul(e0i, e1t, n, n, n);           // E0^-1 E1^T
  const std::vector<double> e1e0i = matmul(e1, e0i, n, n, n);          // E1 E0^-1
  const std::vector<double> e1e0ie1t = matmul(e1e0i, e1t, n, n, n);
  // X0 = Z + sigma I
  const double sigma = 0.5;
  std::vector<double> X((size_t)n2 * n2, 0.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      X[(size_t)r * n2 + c] = a11[(size_t)r * n + c];
      X[(size_t)r * n2 + n + c] = -e0i[(size_t)r * n + c];
      X[(size_t)(n + r) * n2 + c] = -e2[(size_t)r * n + c] + e1e0ie1t[(size_t)r * n + c];
      X[(size_t)(n + r) * n2 + n + c] = -e1e0i[(size_t)r * n + c];
    }
  for (int k = 0; k < n2; ++k) X[(size_t)k * n2 + k] += sigma;
  // sign(X) by the determinant-scaled Newton iteration
  std::vector<double> Xi;
  bool converged = false;
  for (int it = 0; it < 100; ++it) {
    double logdet = 0.0;
    if (!inverse(X, Xi, n2, &logdet)) return fail(SBFWI_ESINGULAR, "the sign iteration of an element's Riccati equation met a singular matrix");
    const double cs = it < 8 ? std::exp(-logdet / n2) : 1.0;     // scaling only while far from convergence
    double diff = 0.0, norm = 0.0;
    for (size_t t = 0; t < X.size(); ++t) {
      const double nx = 0.5 * (cs * X[t] + Xi[t] / cs);
      diff = std::max(diff, std::fabs(nx - X[t]));
      norm = std::max(norm, std::fabs(nx));
      X[t] = nx;
    }
    if (diff <= 1e-14 * norm) { converged = true; break; }
  }
  if (!converged) return fail(SBFWI_ESINGULAR, "the sign iteration of an element's Riccati equation did not converge");
  // projector on the stable subspace, P = (I - sign) / 2; basis of its range (rank n - 1)
  // by Gram-Schmidt with column pivoting, then the constant mode [1; 0]
  std::vector<double> P((size_t)n2 * n2);
  for (int r = 0; r < n2; ++r)
    for (int c = 0; c < n2; ++c) P[(size_t)r * n2 + c] = 0.5 * ((r == c ? 1.0 : 0.0) - X[(size_t)r * n2 + c]);
  double trace = 0.0;
  for (int k = 0; k < n2; ++k) trace += P[(size_t)k * n2 + k];
  if (std::fabs(trace - (n - 1)) > 0.25)
    return fail(SBFWI_ESINGULAR, "an element's stable subspace has dimension " + std::to_string(trace) +
                                     " instead of n_b - 1 = " + std::to_string(n - 1));
  std::vector<std::vector<double>> cols(n2, std::vector<double>(n2));
  for (int c = 0; c < n2; ++c)
    for (int r = 0; r < n2; ++r) cols[c][r] = P[(size_t)r * n2 + c];
  std::vector<std::vector<double>> basis;
  std::vector<bool> used(n2, false);
  double first = 0.0;
  for (int k = 0; k < n; ++k) {
    int best = -1;
    double bn = 0.0;
    for (int c = 0; c < n2; ++c) {
      if (used[c]) continue;
      double s = 0.0;
      for (int r = 0; r < n2; ++r) s += cols[c][r] * cols[c][r];
      if (s > bn) { bn = s; best = c; }
    }
    if (k == n - 1) {
      // every column is now orthogonal to a basis of the whole range: what remains is rounding
      if (bn > 1e-16 * first) return fail(SBFWI_ESINGULAR, "an element's stable subspace is not of rank n_b - 1");
      break;
    }
    if (best < 0 || !(bn > 1e-16 * first)) return fail(SBFWI_ESINGULAR, "an element's stable subspace is degenerate");
    if (k == 0) first = bn;
    used[best] = true;
    std::vector<double> q = cols[best];
    const double inv = 1.0 / std::sqrt(bn);
    for (double& v : q) v *= inv;
    for (int c = 0; c < n2; ++c) {
      if (used[c]) continue;
      double d = 0.0;
      for (int r = 0; r < n2; ++r) d += q[r] * cols[c][r];
      for (int r = 0; r < n2; ++r) cols[c][r] -= d * q[r];
    }
    basis.push_back(q);
  }
  std::vector<double> Qu((size_t)n * n), Qq((size_t)n * n);
  for (int k = 0; k < n; ++k)
    for (int r = 0; r < n; ++r) {
      Qu[(size_t)r * n + k] = k < n - 1 ? basis[k][r] : 1.0;
      Qq[(size_t)r * n + k] = k < n - 1 ? basis[k][n + r] : 0.0;
    }
  std::vector<double> Qui;
  if (!inverse(Qu, Qui, n)) return fail(SBFWI_ESINGULAR, "an element's Riccati basis is singular");
  const std::vector<double> K = matmul(Qq, Qui, n, n, n);
  // Lyapunov: F M + M G = M0 with F = (K - E1) E0^-1 + I, G = E0^-1 (K - E1^T) + I
  std::vector<double> kme1((size_t)n * n), kme1t((size_t)n * n);
  for (size_t t = 0; t < kme1.size(); ++t) { kme1[t] = K[t] - e1[t]; kme1t[t] = K[t] - e1t[t]; }
  std::vector<double> F = matmul(kme1, e0i, n, n, n);
  std::vector<double> G = matmul(e0i, kme1t, n, n, n);
  for (int k = 0; k < n; ++k) { F[(size_t)k * n + k] += 1.0; G[(size_t)k * n + k] += 1.0; }
  std::vector<double> C(M0, M0 + (size_t)n * n), Fi, Gi;
  converged = false;
  for (int it = 0; it < 100; ++it) {
    double logdet = 0.0;
    if (!inverse(F, Fi, n, &logdet) || !inverse(G, Gi, n))
      return fail(SBFWI_ESINGULAR, "the sign iteration of an element's Lyapunov equation met a singular matrix");
    const double cs = it < 8 ? std::exp(-logdet / n) : 1.0;
    const std::vector<double> FCG = matmul(matmul(Fi, C, n, n, n), Gi, n, n, n);
    double diff = 0.0, norm = 0.0;
    for (size_t t = 0; t < F.size(); ++t) {
      const double nf = 0.5 * (cs * F[t] + Fi[t] / cs);
      diff = std::max(diff, std::fabs(nf - F[t]));
      norm = std::max(norm, std::fabs(nf));
      F[t] = nf;
      G[t] = 0.5 * (cs * G[t] + Gi[t] / cs);
      C[t] = 0.5 * (cs * C[t] + FCG[t] / cs);
    }
    if (diff <= 1e-14 * norm) { converged = true; break; }
  }
  if (!converged) return fail(SBFWI_ESINGULAR, "the sign iteration of an element's Lyapunov equation did not converge");
  std::copy(K.begin(), K.end(), Kout);
  for (size_t t = 0; t < C.size(); ++t) Mout[t] = 0.5 * C[t];
  return SBFWI_OK;
}

}  // namespace sbfwi

extern "C" int sbfwi_lfe_element_matrices(const double* E0, const double* E1, const double* E2, const double* M0,
                                          int32_t n_b, double* K, double* M) {
  using namespace sbfwi;
  if (!E0 || !E1 || !E2 || !M0 || !K || !M) return fail(SBFWI_EINVAL, "NULL argument");
  if (n_b < 2 || n_b > kMaxBoundaryNodes) return fail(SBFWI_EINVAL, "n_b must be in 2..40");
  return lfe_element(E0, E1, E2, M0, n_b, K, M);
}
