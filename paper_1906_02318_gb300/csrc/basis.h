// Lifted bases of the learned linear model (Sec. IV-A), in split form.
//
// Every feature of Psi(x, u) used here is a(x) + sum_k p_k(u) b_k(x): a state
// part plus input monomials p_k times state coefficients.  Because the input is
// held over the horizon (Sec. VII-B), a tick lifts all N candidates of the same
// x_t: the state parts need one sine/cosine per tick and each candidate adds P
// products per feature.  The host fit (float64) and the tick kernel (float32)
// use this one definition.
//
//   balance bot (n = 12, P = 1, p = {u}):
//     theta, theta_dot, x, x_dot, u, sin th, cos th, thd^2, thd u,
//     thd^2 sin th, u cos th, 1
//   race car (n = 32, P = 3, p = {delta, a, delta^2}):
//     px, py, psi, vx, vy, om, delta, a, sin, cos, vx cos, vx sin, vy cos, vy sin,
//     om vx, om vy, vx^2, vy^2, om^2, delta vx, delta vy, delta om, a vx,
//     delta cos, delta sin, a cos, a sin, om cos, om sin, vx vy, delta^2, 1
//   linear (n = nx + nu, P = nu, p_k = u_k): x, u
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define MPMI_HD __host__ __device__ __forceinline__
#else
#define MPMI_HD inline
#endif

namespace mpmi {

enum BasisKind : int { kBot = 0, kCar = 1, kLin11 = 2, kLin22 = 3, kLin41 = 4 };

template <int KIND>
struct BasisTraits;
template <>
struct BasisTraits<kBot> {
  static constexpr int N = 12, NX = 4, NU = 1, NP = 1;
  static constexpr bool TRACK = false;
};
template <>
struct BasisTraits<kCar> {
  static constexpr int N = 32, NX = 6, NU = 2, NP = 3;
  static constexpr bool TRACK = true;
};
template <>
struct BasisTraits<kLin11> {
  static constexpr int N = 2, NX = 1, NU = 1, NP = 1;
  static constexpr bool TRACK = false;
};
template <>
struct BasisTraits<kLin22> {
  static constexpr int N = 4, NX = 2, NU = 2, NP = 2;
  static constexpr bool TRACK = false;
};
template <>
struct BasisTraits<kLin41> {
  static constexpr int N = 5, NX = 4, NU = 1, NP = 1;
  static constexpr bool TRACK = false;
};

constexpr int kMaxP = 3;

// Split coefficients of feature j at state x: *a and b[0..P).  s, c are the
// sine and cosine of the basis angle (bot: theta = x[0]; car: psi = x[2]),
// computed once by the caller.  T is double on the host fit, float per tick.
template <class T>
MPMI_HD void feature_split(int kind, int j, const T* x, T s, T c, T* a, T* b) {
  for (int k = 0; k < kMaxP; ++k) b[k] = T(0);
  *a = T(0);
  if (kind == kBot) {
    const T thd = x[1];
    switch (j) {
      case 0: *a = x[0]; break;
      case 1: *a = thd; break;
      case 2: *a = x[2]; break;
      case 3: *a = x[3]; break;
      case 4: b[0] = T(1); break;
      case 5: *a = s; break;
      case 6: *a = c; break;
      case 7: *a = thd * thd; break;
      case 8: b[0] = thd; break;
      case 9: *a = thd * thd * s; break;
      case 10: b[0] = c; break;
      default: *a = T(1); break;  // 11
    }
    return;
  }
  if (kind == kCar) {
    const T vx = x[3], vy = x[4], om = x[5];
    switch (j) {
      case 0: *a = x[0]; break;
      case 1: *a = x[1]; break;
      case 2: *a = x[2]; break;
      case 3: *a = vx; break;
      case 4: *a = vy; break;
      case 5: *a = om; break;
      case 6: b[0] = T(1); break;
      case 7: b[1] = T(1); break;
      case 8: *a = s; break;
      case 9: *a = c; break;
      case 10: *a = vx * c; break;
      case 11: *a = vx * s; break;
      case 12: *a = vy * c; break;
      case 13: *a = vy * s; break;
      case 14: *a = om * vx; break;
      case 15: *a = om * vy; break;
      case 16: *a = vx * vx; break;
      case 17: *a = vy * vy; break;
      case 18: *a = om * om; break;
      case 19: b[0] = vx; break;
      case 20: b[0] = vy; break;
      case 21: b[0] = om; break;
      case 22: b[1] = vx; break;
      case 23: b[0] = c; break;
      case 24: b[0] = s; break;
      case 25: b[1] = c; break;
      case 26: b[1] = s; break;
      case 27: *a = om * c; break;
      case 28: *a = om * s; break;
      case 29: *a = vx * vy; break;
      case 30: b[2] = T(1); break;
      default: *a = T(1); break;  // 31
    }
    return;
  }
  // linear bases: z = (x, u)
  const int nx = kind == kLin11 ? 1 : kind == kLin22 ? 2 : 4;
  if (j < nx) {
    *a = x[j];
  } else {
    b[j - nx] = T(1);
  }
}

// Features that depend on the input alone (and the constant).  With the input
// held over the horizon (Sec. VII-B) a prediction step leaves them unchanged:
// their column of the fit target equals their regressor column, so their rows
// of K are exact unit rows (the fit sets them; operators from callers are
// checked), and a rollout need not recompute them.
MPMI_HD constexpr bool held_feature(int kind, int j) {
  return kind == kBot   ? (j == 4 || j == 11)
         : kind == kCar ? (j == 6 || j == 7 || j == 30 || j == 31)
                        : j >= (kind == kLin11 ? 1 : (kind == kLin22 ? 2 : 4));
}

// Index of the state coordinate whose sine/cosine the basis uses (-1: none).
MPMI_HD int angle_index(int kind) { return kind == kBot ? 0 : (kind == kCar ? 2 : -1); }

// Input monomials p_k(u) in float64 (host fit).
MPMI_HD void monomials64(int kind, const double* u, double* p) {
  if (kind == kBot) {
    p[0] = u[0];
  } else if (kind == kCar) {
    p[0] = u[0];
    p[1] = u[1];
    p[2] = u[0] * u[0];
  } else {
    const int nu = kind == kLin22 ? 2 : 1;
    for (int k = 0; k < nu; ++k) p[k] = u[k];
  }
}

inline int basis_kind(int basis, int nx, int nu) {
  if (basis == 0) return (nx == 4 && nu == 1) ? kBot : -1;
  if (basis == 1) return (nx == 6 && nu == 2) ? kCar : -1;
  if (basis == 2) {
    if (nx == 1 && nu == 1) return kLin11;
    if (nx == 2 && nu == 2) return kLin22;
    if (nx == 4 && nu == 1) return kLin41;
  }
  return -1;
}

inline void kind_dims(int kind, int* n, int* nx, int* nu, int* np) {
  switch (kind) {
    case kBot: *n = 12; *nx = 4; *nu = 1; *np = 1; break;
    case kCar: *n = 32; *nx = 6; *nu = 2; *np = 3; break;
    case kLin11: *n = 2; *nx = 1; *nu = 1; *np = 1; break;
    case kLin22: *n = 4; *nx = 2; *nu = 2; *np = 2; break;
    default: *n = 5; *nx = 4; *nu = 1; *np = 1; break;
  }
}

}  // namespace mpmi
