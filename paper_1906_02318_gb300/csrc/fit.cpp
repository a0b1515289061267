// fit_model: least-squares fit of the lifted operator (Sec. IV-A).
//
// K = argmin sum_m || Psi(x_{m+1}, u_m) - K Psi(x_m, u_m) ||^2.  With the lifted
// snapshots as rows of X (m x n) and Y (m x n) this is X K^T ~= Y, solved by
// Householder QR of X in float64 (no normal equations, so the conditioning of X
// is not squared).  The fit runs once per model, offline, on the host.
#include <math.h>

#include <string>
#include <vector>

#include "basis.h"
#include "internal.h"

namespace mpmi {

static void lift_row(int kind, int n, const double* x, const double* u, double* out) {
  double p[kMaxP] = {0, 0, 0};
  monomials64(kind, u, p);
  const int ai = angle_index(kind);
  const double s = ai >= 0 ? sin(x[ai]) : 0.0, c = ai >= 0 ? cos(x[ai]) : 0.0;
  for (int j = 0; j < n; ++j) {
    double a, b[kMaxP];
    feature_split<double>(kind, j, x, s, c, &a, b);
    double v = a;
    for (int k = 0; k < kMaxP; ++k)
      if (b[k] != 0.0) v += p[k] * b[k];
    out[j] = v;
  }
}

int fit_householder(int kind, const double* x, const double* u, const double* xn,
                    int64_t m, std::vector<double>* K, double* residual, std::string* err) {
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m < n) {
    *err = "fit_model: need at least n transitions";
    return MPMI_E_INVALID_ARG;
  }
  // column-major copies: A = X, B = Y
  std::vector<double> A((size_t)m * n), B((size_t)m * n), row(n);
  for (int64_t i = 0; i < m; ++i) {
    lift_row(kind, n, x + i * nx, u + i * nu, row.data());
    for (int j = 0; j < n; ++j) A[(size_t)j * m + i] = row[j];
    lift_row(kind, n, xn + i * nx, u + i * nu, row.data());
    for (int j = 0; j < n; ++j) B[(size_t)j * m + i] = row[j];
  }
  const std::vector<double> A0 = A, B0 = B;
  std::vector<double> rdiag(n);
  double rmax = 0.0;
  for (int k = 0; k < n; ++k) {
    double* ak = &A[(size_t)k * m];
    double norm2 = 0.0;
    for (int64_t i = k; i < m; ++i) norm2 += ak[i] * ak[i];
    const double norm = sqrt(norm2);
    if (!(norm > 0.0)) {
      *err = "fit_model: lifted data is rank deficient";
      return MPMI_E_INVALID_ARG;
    }
    const double alpha = ak[k] > 0 ? -norm : norm;
    // v = ak[k:] - alpha e_k, stored in place; v^T v = 2 (norm2 - alpha ak[k])
    const double vtv = 2.0 * (norm2 - alpha * ak[k]);
    ak[k] -= alpha;
    auto reflect = [&](double* col) {
      double dot = 0.0;
      for (int64_t i = k; i < m; ++i) dot += ak[i] * col[i];
      const double f = 2.0 * dot / vtv;
      for (int64_t i = k; i < m; ++i) col[i] -= f * ak[i];
    };
    for (int c = k + 1; c < n; ++c) reflect(&A[(size_t)c * m]);
    for (int c = 0; c < n; ++c) reflect(&B[(size_t)c * m]);
    rdiag[k] = alpha;
    rmax = fmax(rmax, fabs(alpha));
  }
  for (int k = 0; k < n; ++k) {
    if (fabs(rdiag[k]) <= 1e-13 * rmax) {
      *err = "fit_model: lifted data is rank deficient";
      return MPMI_E_INVALID_ARG;
    }
  }
  // back substitution R X = (Q^T Y)[0:n]; R's strict upper part is in A, its
  // diagonal in rdiag.  Column c of X holds row c of K.
  K->assign((size_t)n * n, 0.0);
  std::vector<double> xs(n);
  for (int c = 0; c < n; ++c) {
    const double* bc = &B[(size_t)c * m];
    for (int i = n - 1; i >= 0; --i) {
      double s = bc[i];
      for (int j = i + 1; j < n; ++j) s -= A[(size_t)j * m + i] * xs[j];
      xs[i] = s / rdiag[i];
    }
    for (int k = 0; k < n; ++k) (*K)[(size_t)c * n + k] = xs[k];
  }
  // held input features: the exact solution of their rows is the unit row, which
  // the back substitution returns up to rounding
  for (int c = 0; c < n; ++c)
    if (held_feature(kind, c))
      for (int k = 0; k < n; ++k) (*K)[(size_t)c * n + k] = k == c ? 1.0 : 0.0;
  if (residual) {
    double num = 0.0, den = 0.0;
    for (int c = 0; c < n; ++c) {
      const double* kc = &(*K)[(size_t)c * n];
      for (int64_t i = 0; i < m; ++i) {
        double pred = 0.0;
        for (int k = 0; k < n; ++k) pred += A0[(size_t)k * m + i] * kc[k];
        const double y = B0[(size_t)c * m + i];
        num += (pred - y) * (pred - y);
        den += y * y;
      }
    }
    *residual = den > 0 ? sqrt(num / den) : 0.0;
  }
  return MPMI_OK;
}

}  // namespace mpmi
