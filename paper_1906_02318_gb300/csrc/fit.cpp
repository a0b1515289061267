// fit_model: least-squares fit of the lifted operator (Sec. IV-A), and the
// sparsity-promoting selection of its basis (Sec. IV-A, V-C.3).
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

// Column-major lifted snapshots: X[j * m + i] = Psi_j(x_i, u_i), Y likewise for
// (x_next_i, u_i).
static void lift_pairs(int kind, int n, int nx, int nu, const double* x, const double* u,
                       const double* xn, int64_t m, std::vector<double>* X,
                       std::vector<double>* Y) {
  X->assign((size_t)m * n, 0.0);
  Y->assign((size_t)m * n, 0.0);
  std::vector<double> row(n);
  for (int64_t i = 0; i < m; ++i) {
    lift_row(kind, n, x + i * nx, u + i * nu, row.data());
    for (int j = 0; j < n; ++j) (*X)[(size_t)j * m + i] = row[j];
    lift_row(kind, n, xn + i * nx, u + i * nu, row.data());
    for (int j = 0; j < n; ++j) (*Y)[(size_t)j * m + i] = row[j];
  }
}

// Least squares A W ~= B by Householder QR.  A: m x p column-major, B: m x q
// column-major; W (p x q) returned row-major (W[r * q + c]).
static int qr_lstsq(std::vector<double> A, std::vector<double> B, int64_t m, int p, int q,
                    std::vector<double>* W, std::string* err) {
  std::vector<double> rdiag(p);
  double rmax = 0.0;
  for (int k = 0; k < p; ++k) {
    double* ak = &A[(size_t)k * m];
    double norm2 = 0.0;
    for (int64_t i = k; i < m; ++i) norm2 += ak[i] * ak[i];
    const double norm = sqrt(norm2);
    if (!(norm > 0.0)) {
      *err = "fit: lifted data is rank deficient";
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
    for (int c = k + 1; c < p; ++c) reflect(&A[(size_t)c * m]);
    for (int c = 0; c < q; ++c) reflect(&B[(size_t)c * m]);
    rdiag[k] = alpha;
    rmax = fmax(rmax, fabs(alpha));
  }
  for (int k = 0; k < p; ++k) {
    if (fabs(rdiag[k]) <= 1e-13 * rmax) {
      *err = "fit: lifted data is rank deficient";
      return MPMI_E_INVALID_ARG;
    }
  }
  // back substitution R W = (Q^T B)[0:p]; R's strict upper part is in A, its
  // diagonal in rdiag
  W->assign((size_t)p * q, 0.0);
  std::vector<double> xs(p);
  for (int c = 0; c < q; ++c) {
    const double* bc = &B[(size_t)c * m];
    for (int i = p - 1; i >= 0; --i) {
      double s = bc[i];
      for (int j = i + 1; j < p; ++j) s -= A[(size_t)j * m + i] * xs[j];
      xs[i] = s / rdiag[i];
    }
    for (int r = 0; r < p; ++r) (*W)[(size_t)r * q + c] = xs[r];
  }
  return MPMI_OK;
}

// Held input features: the exact least-squares solution of their rows is the
// unit row (their target column is their regressor column), which the solver
// returns up to rounding; set it exactly.
static void set_held_rows(int kind, int n, std::vector<double>* K) {
  for (int c = 0; c < n; ++c)
    if (held_feature(kind, c))
      for (int k = 0; k < n; ++k) (*K)[(size_t)c * n + k] = k == c ? 1.0 : 0.0;
}

// ||X K^T - Y||_F / ||Y||_F over the predicted features `rows` (all if empty).
static double fit_residual(const std::vector<double>& X, const std::vector<double>& Y,
                           const std::vector<double>& K, int64_t m, int n,
                           const std::vector<unsigned char>& keep) {
  double num = 0.0, den = 0.0;
  for (int c = 0; c < n; ++c) {
    if (!keep.empty() && !keep[c]) continue;
    const double* kc = &K[(size_t)c * n];
    for (int64_t i = 0; i < m; ++i) {
      double pred = 0.0;
      for (int k = 0; k < n; ++k) pred += X[(size_t)k * m + i] * kc[k];
      const double y = Y[(size_t)c * m + i];
      num += (pred - y) * (pred - y);
      den += y * y;
    }
  }
  return den > 0 ? sqrt(num / den) : 0.0;
}

int fit_householder(int kind, const double* x, const double* u, const double* xn,
                    int64_t m, std::vector<double>* K, double* residual, std::string* err) {
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m < n) {
    *err = "fit_model: need at least n transitions";
    return MPMI_E_INVALID_ARG;
  }
  std::vector<double> X, Y, W;
  lift_pairs(kind, n, nx, nu, x, u, xn, m, &X, &Y);
  const int rc = qr_lstsq(X, Y, m, n, n, &W, err);
  if (rc != MPMI_OK) return rc;
  // W = K^T
  K->assign((size_t)n * n, 0.0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) (*K)[(size_t)c * n + r] = W[(size_t)r * n + c];
  set_held_rows(kind, n, K);
  if (residual) *residual = fit_residual(X, Y, *K, m, n, {});
  return MPMI_OK;
}

// ---- sparsity-promoting basis selection -----------------------------------
// Sparsity-promoting DMD (Jovanovic, Schmid & Nichols 2014) has two stages: an
// l1-type penalised least squares solved by ADMM, then an unpenalised refit
// ("polishing") on the surviving terms.  Applied here to the lifted regression
// X W ~= Y (W = K^T) with one group per candidate feature j (row W[j, :], its
// influence on every predicted feature), on unit-RMS scaled A = X D^-1 and
// B = Y E^-1:
//   minimise (1/m) ||A V - B||_F^2 + gamma sum_{j in C} ||V[j, :]||_2
// ADMM (split V = Z, penalty rho, scaled dual U):
//   V <- (2/m A^T A + rho I)^-1 (2/m A^T B + rho (Z - U))   (Cholesky, once)
//   Z[j] <- max(0, 1 - (gamma/rho) / ||(V + U)[j]||) (V + U)[j]  for j in C,
//   Z[j] <- (V + U)[j] otherwise;   U <- U + V - Z.
// Candidates C: every feature but the state and the held ones.  The support is
// {j : Z[j] != 0} plus every feature outside C; polishing refits on its columns.
static int cholesky(std::vector<double>* G, int n) {
  for (int j = 0; j < n; ++j) {
    double d = (*G)[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= (*G)[(size_t)j * n + k] * (*G)[(size_t)j * n + k];
    if (!(d > 0.0)) return MPMI_E_INVALID_ARG;
    const double l = sqrt(d);
    (*G)[(size_t)j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double s = (*G)[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= (*G)[(size_t)i * n + k] * (*G)[(size_t)j * n + k];
      (*G)[(size_t)i * n + j] = s / l;
    }
  }
  return MPMI_OK;
}

// Solves L L^T v = b in place (L lower, row-major n x n).
static void chol_solve(const std::vector<double>& L, int n, double* b) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
    b[i] = s / L[(size_t)i * n + i];
  }
}

int fit_sparse(int kind, const double* x, const double* u, const double* xn, int64_t m,
               double gamma, double rho, int iters, std::vector<double>* K,
               std::vector<unsigned char>* support, double* residual, std::string* err) {
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m < n) {
    *err = "fit_sparse: need at least n transitions";
    return MPMI_E_INVALID_ARG;
  }
  std::vector<double> X, Y;
  lift_pairs(kind, n, nx, nu, x, u, xn, m, &X, &Y);
  // unit-RMS scaling of regressors and targets
  std::vector<double> A = X, B = Y;
  for (int j = 0; j < n; ++j) {
    for (std::vector<double>* M : {&A, &B}) {
      double* col = &(*M)[(size_t)j * m];
      double ss = 0.0;
      for (int64_t i = 0; i < m; ++i) ss += col[i] * col[i];
      double s = sqrt(ss / (double)m);
      if (s == 0.0) s = 1.0;
      for (int64_t i = 0; i < m; ++i) col[i] /= s;
    }
  }
  std::vector<unsigned char> cand(n, 0);
  for (int j = nx; j < n; ++j) cand[j] = held_feature(kind, j) ? 0 : 1;
  // G = 2/m A^T A + rho I (row-major), AtB = 2/m A^T B (row-major, n x n)
  std::vector<double> G((size_t)n * n), AtB((size_t)n * n);
  for (int a = 0; a < n; ++a) {
    for (int b = 0; b < n; ++b) {
      double g = 0.0, h = 0.0;
      const double* ca = &A[(size_t)a * m];
      const double* cb = &A[(size_t)b * m];
      const double* yb = &B[(size_t)b * m];
      for (int64_t i = 0; i < m; ++i) {
        g += ca[i] * cb[i];
        h += ca[i] * yb[i];
      }
      G[(size_t)a * n + b] = 2.0 / (double)m * g + (a == b ? rho : 0.0);
      AtB[(size_t)a * n + b] = 2.0 / (double)m * h;
    }
  }
  if (cholesky(&G, n) != MPMI_OK) {
    *err = "fit_sparse: normal matrix not positive definite";
    return MPMI_E_INVALID_ARG;
  }
  std::vector<double> Z((size_t)n * n, 0.0), U((size_t)n * n, 0.0), V((size_t)n * n),
      col(n);
  for (int it = 0; it < iters; ++it) {
    // V = G^-1 (AtB + rho (Z - U)), one right-hand side per target column
    for (int c = 0; c < n; ++c) {
      for (int r = 0; r < n; ++r)
        col[r] = AtB[(size_t)r * n + c] + rho * (Z[(size_t)r * n + c] - U[(size_t)r * n + c]);
      chol_solve(G, n, col.data());
      for (int r = 0; r < n; ++r) V[(size_t)r * n + c] = col[r];
    }
    for (int r = 0; r < n; ++r) {
      double nrm2 = 0.0;
      for (int c = 0; c < n; ++c) {
        const double pv = V[(size_t)r * n + c] + U[(size_t)r * n + c];
        nrm2 += pv * pv;
      }
      const double nrm = sqrt(nrm2);
      double f = 1.0;
      if (cand[r]) {
        f = nrm > 0.0 ? 1.0 - (gamma / rho) / nrm : 0.0;
        if (f < 0.0) f = 0.0;
      }
      for (int c = 0; c < n; ++c) {
        const double pv = V[(size_t)r * n + c] + U[(size_t)r * n + c];
        Z[(size_t)r * n + c] = f * pv;
      }
    }
    for (size_t i = 0; i < U.size(); ++i) U[i] += V[i] - Z[i];
  }
  support->assign(n, 1);
  std::vector<int> cols;
  for (int r = 0; r < n; ++r) {
    if (cand[r]) {
      bool nz = false;
      for (int c = 0; c < n; ++c) nz = nz || Z[(size_t)r * n + c] != 0.0;
      (*support)[r] = nz ? 1 : 0;
    }
    if ((*support)[r]) cols.push_back(r);
  }
  // polishing: least squares on the support's columns of X
  const int p = (int)cols.size();
  std::vector<double> Xs((size_t)m * p), W;
  for (int a = 0; a < p; ++a)
    for (int64_t i = 0; i < m; ++i) Xs[(size_t)a * m + i] = X[(size_t)cols[a] * m + i];
  const int rc = qr_lstsq(Xs, Y, m, p, n, &W, err);
  if (rc != MPMI_OK) return rc;
  K->assign((size_t)n * n, 0.0);
  for (int a = 0; a < p; ++a)
    for (int c = 0; c < n; ++c) (*K)[(size_t)c * n + cols[a]] = W[(size_t)a * n + c];
  for (int r = 0; r < n; ++r)
    if (!(*support)[r])
      for (int c = 0; c < n; ++c) (*K)[(size_t)r * n + c] = 0.0;
  set_held_rows(kind, n, K);
  if (residual) *residual = fit_residual(X, Y, *K, m, n, *support);
  return MPMI_OK;
}

}  // namespace mpmi
