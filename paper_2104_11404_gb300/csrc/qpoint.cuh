// Quadrature-point physics of the Lagrangian step, templated on the compute
// type T (double for the FP64 path, float for the mixed path).
//
// Per point (Section 2, eq:EOS, eq:adaptive-timestep, and the artificial
// viscosity sigma_a of eq:euler in the form of Dobrev, Kolev, Rieben 2012):
//   rho   = rho0|J0| / |J|                 (mass conservation, density eliminated)
//   p     = (gamma - 1) rho e               (ideal gas)
//   c_s   = sqrt(max(0, gamma (gamma - 1) e))
//   h_min = sigma_min(J) / k
//   grad v = grad_ref v J^{-1},  eps = sym(grad v),  (lambda, s) its smallest eigenpair
//   if lambda < 0:  l = l_0 |J J0^{-1} s|,  mu = rho (q2 l^2 |lambda| + q1 l c_s),
//                   sigma = -p I + mu eps;   else sigma = -p I, mu = 0
//   tau   = cfl / (c_s / h_min + cfl_mu mu / (rho h_min^2))
#pragma once

#include <math.h>

#include "lagh_impl.cuh"

namespace lagh {

// Square root, quotient and hypotenuse in the working precision: correctly
// rounded in FP64.  In FP32 the 2D point physics issues a dozen of them per
// point, so these take the single hardware approximations (reciprocal and
// reciprocal square root, about one unit in the last place) with products
// that are never fused: every template instance then computes the same bits,
// whatever launch shape it is compiled for.
__device__ __forceinline__ float rcp_approx(float a) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float a) {
  float r;
  asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
template <typename T> __device__ __forceinline__ T t_sqrt(T a);
template <> __device__ __forceinline__ double t_sqrt<double>(double a) { return sqrt(a); }
// a rsqrt(a) for finite a > 0; 0, +inf (and NaN) map to themselves
template <> __device__ __forceinline__ float t_sqrt<float>(float a) {
  return (a > 0.0f && a < __int_as_float(0x7f800000)) ? __fmul_rn(a, rsqrt_approx(a)) : a;
}
template <typename T> __device__ __forceinline__ T t_div(T a, T b);
template <> __device__ __forceinline__ double t_div<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float t_div<float>(float a, float b) {
  return __fmul_rn(a, rcp_approx(b));
}
template <typename T> __device__ __forceinline__ T t_hypot(T a, T b);
template <> __device__ __forceinline__ double t_hypot<double>(double a, double b) { return hypot(a, b); }
// FP32: |(a, b)| without rescaling (the mixed path's gradients and strain
// rates are far from the FP32 overflow range; squares below the underflow
// range stand for a vanishing vector)
template <> __device__ __forceinline__ float t_hypot<float>(float a, float b) {
  return t_sqrt<float>(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)));
}

// The point physics takes the approximate FP32 forms in 2D.  In 3D it keeps
// correctly rounded quotients and square roots: there the mixed path's
// velocity after a whole 3D blast run sits close to its 1e-4 bound against
// the FP64 run, and the approximations (measured) carry it past the bound.
template <typename T> __device__ __forceinline__ T ieee_sqrt(T a);
template <> __device__ __forceinline__ double ieee_sqrt<double>(double a) { return sqrt(a); }
template <> __device__ __forceinline__ float ieee_sqrt<float>(float a) { return sqrtf(a); }
template <typename T, int DIM> __device__ __forceinline__ T q_sqrt(T a) {
  if constexpr (DIM == 2) return t_sqrt<T>(a);
  else return ieee_sqrt<T>(a);
}
template <typename T, int DIM> __device__ __forceinline__ T q_div(T a, T b) {
  if constexpr (DIM == 2) return t_div<T>(a, b);
  else return a / b;
}
template <typename T> __device__ __forceinline__ T t_abs(T a) { return a < T(0) ? -a : a; }
template <typename T> __device__ __forceinline__ T t_inf();
template <> __device__ __forceinline__ double t_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }
template <> __device__ __forceinline__ float t_inf<float>() { return __int_as_float(0x7f800000); }

template <typename T, int DIM>
__device__ __forceinline__ T det_of(const T (&J)[DIM][DIM]) {
  if constexpr (DIM == 2) {
    return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  } else {
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  }
}

// adj(J) with adj(J) J = det(J) I
template <typename T, int DIM>
__device__ __forceinline__ void adj_of(const T (&J)[DIM][DIM], T (&A)[DIM][DIM]) {
  if constexpr (DIM == 2) {
    A[0][0] = J[1][1];  A[0][1] = -J[0][1];
    A[1][0] = -J[1][0]; A[1][1] = J[0][0];
  } else {
    A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  }
}

// Cyclic Jacobi rotations on a symmetric 3x3 matrix S (in place); the columns
// of V collect the rotations.  Pairs (0,1), (0,2), (1,2) in that order, at
// most 12 sweeps.  The sweeps stop once the off-diagonal part is at the
// rounding level of the diagonal (sum of squares below (8 eps)^2 times the
// diagonal's): there the rotations only move rounding errors (an exactly
// zero off-diagonal is never reached in floating point, the iteration would
// run to its cap).
template <typename T>
__device__ __forceinline__ void jacobi_sym3(T (&S)[3][3], T (&V)[3][3]) {
  constexpr T eps8 = sizeof(T) == 8 ? T(8.0 * 2.220446049250313e-16) : T(8.0 * 1.1920929e-07);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const T off = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2];
    const T dia = S[0][0] * S[0][0] + S[1][1] * S[1][1] + S[2][2] * S[2][2];
    if (off <= eps8 * eps8 * dia) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0;
      const int q = r == 0 ? 1 : 2;
      T spq = S[p][q];
      if (spq == T(0)) continue;
      // a correctly rounded quotient here: spq may be subnormal with an exactly
      // zero numerator (theta = 0, a 45 degree rotation)
      T theta = (S[q][q] - S[p][p]) / (T(2) * spq);
      T t = (theta >= T(0) ? T(1) : T(-1)) / (t_abs(theta) + ieee_sqrt(theta * theta + T(1)));
      T cs = T(1) / ieee_sqrt(t * t + T(1));
      T sn = t * cs;
      for (int j = 0; j < 3; ++j) {  // rows p, q
        T a = S[p][j], b = S[q][j];
        S[p][j] = cs * a - sn * b;
        S[q][j] = sn * a + cs * b;
      }
      for (int j = 0; j < 3; ++j) {  // columns p, q
        T a = S[j][p], b = S[j][q];
        S[j][p] = cs * a - sn * b;
        S[j][q] = sn * a + cs * b;
      }
      for (int j = 0; j < 3; ++j) {
        T a = V[j][p], b = V[j][q];
        V[j][p] = cs * a - sn * b;
        V[j][q] = sn * a + cs * b;
      }
    }
  }
}

// Smallest eigenvalue and a unit eigenvector of the symmetric matrix E.
template <typename T, int DIM>
__device__ __forceinline__ void min_eigenpair(const T (&E)[DIM][DIM], T& lam, T (&s)[DIM]) {
  if constexpr (DIM == 2) {
    T a = E[0][0], b = E[0][1], d = E[1][1];
    T r = t_hypot(T(0.5) * (a - d), b);
    lam = T(0.5) * (a + d) - r;
    if (r == T(0)) { s[0] = T(1); s[1] = T(0); return; }
    // null vectors (b, lam - a) and (lam - d, b) of E - lam I: keep the longer
    T u0 = b, u1 = lam - a, w0 = lam - d, w1 = b;
    T nu = t_hypot(u0, u1), nw = t_hypot(w0, w1);
    if (nu >= nw) { s[0] = t_div(u0, nu); s[1] = t_div(u1, nu); }
    else { s[0] = t_div(w0, nw); s[1] = t_div(w1, nw); }
  } else {
    T S[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[i][j] = E[i][j];
    jacobi_sym3(S, V);
    int im = 0;
    if (S[1][1] < S[im][im]) im = 1;
    if (S[2][2] < S[im][im]) im = 2;
    lam = S[im][im];
    for (int j = 0; j < 3; ++j) s[j] = V[j][im];
  }
}

// Smallest singular value of J.
template <typename T, int DIM>
__device__ __forceinline__ T sigma_min_of(const T (&J)[DIM][DIM], T detJ) {
  if constexpr (DIM == 2) {
    // sigma_max = (|(a+d, c-b)| + |(a-d, b+c)|) / 2 and sigma_min = |det| / sigma_max
    T s1 = t_hypot(J[0][0] + J[1][1], J[1][0] - J[0][1]);
    T s2 = t_hypot(J[0][0] - J[1][1], J[0][1] + J[1][0]);
    return t_div(T(2) * t_abs(detJ), s1 + s2);
  } else {
    T S[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T acc = T(0);
        for (int c = 0; c < 3; ++c) acc += J[c][i] * J[c][j];
        S[i][j] = acc;
      }
    jacobi_sym3(S, V);
    T m = S[0][0];
    if (S[1][1] < m) m = S[1][1];
    if (S[2][2] < m) m = S[2][2];
    return ieee_sqrt(m > T(0) ? m : T(0));
  }
}

// A physical constant in the working precision: the FP64 value, or its FP32
// copy rounded once on the host (no conversion per point).
template <typename T>
__device__ __forceinline__ T pconst(double d, float f);
template <>
__device__ __forceinline__ double pconst<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pconst<float>(double, float f) { return f; }

// Stress and time-step estimate at one point.  J, Gv: reference gradients
// (row = component, column = reference direction).  p_ref: a constant
// reference pressure taken out of the returned stress (sigma + p_ref I is
// returned; the caller accounts for -p_ref I separately).  gam: the adiabatic
// index of the element (eq:EOS).  Returns the flags kDevTangled /
// kDevNonFinite (then sigma = 0 and tau = 0).
template <typename T, int DIM>
__device__ __forceinline__ int qpoint_physics(const T (&J)[DIM][DIM], const T (&Gv)[DIM][DIM],
                                              T e_q, T rho0K, T gam, const Phys& ph,
                                              const T (&J0inv)[DIM], T ell0, T kinv, T p_ref,
                                              T (&sigma)[DIM][DIM], T& tau) {
  T detJ = det_of<T, DIM>(J);
  for (int c = 0; c < DIM; ++c)
    for (int n = 0; n < DIM; ++n) sigma[c][n] = T(0);
  if (!isfinite(detJ) || !isfinite(e_q)) { tau = T(0); return kDevNonFinite; }
  if (!(detJ > T(0))) { tau = T(0); return kDevTangled; }
  T rho = q_div<T, DIM>(rho0K, detJ);
  T p = (gam - T(1)) * rho * e_q;
  T cs2 = gam * (gam - T(1)) * e_q;
  T cs = q_sqrt<T, DIM>(cs2 > T(0) ? cs2 : T(0));
  for (int c = 0; c < DIM; ++c) sigma[c][c] = p_ref - p;
  T hmin = sigma_min_of<T, DIM>(J, detJ) * kinv;
  T mu = T(0);
  if (ph.visc) {
    T A[DIM][DIM], eps[DIM][DIM], gv[DIM][DIM];
    adj_of<T, DIM>(J, A);
    T idet = q_div<T, DIM>(T(1), detJ);
    for (int c = 0; c < DIM; ++c)
      for (int n = 0; n < DIM; ++n) {
        T acc = T(0);
        for (int m = 0; m < DIM; ++m) acc += Gv[c][m] * A[m][n];
        gv[c][n] = acc * idet;
      }
    for (int c = 0; c < DIM; ++c)
      for (int n = 0; n < DIM; ++n) eps[c][n] = T(0.5) * (gv[c][n] + gv[n][c]);
    T lam, s[DIM];
    min_eigenpair<T, DIM>(eps, lam, s);
    // compression only above a floor of 1e-5 (|eps|_F + c_s / h_min): below it
    // the sign of the smallest strain rate is rounding noise (a vanishing
    // strain rate: z-invariant flow in 3D, gas at rest) and would switch on
    // the linear term
    T frob = T(0);
    for (int c = 0; c < DIM; ++c)
      for (int n = 0; n < DIM; ++n) frob += eps[c][n] * eps[c][n];
    frob = q_sqrt<T, DIM>(frob);
    if (lam < -T(1e-5) * (frob + q_div<T, DIM>(cs, hmin))) {
      T n2 = T(0);
      for (int c = 0; c < DIM; ++c) {
        T dc = T(0);
        for (int m = 0; m < DIM; ++m) dc += J[c][m] * J0inv[m] * s[m];
        n2 += dc * dc;
      }
      T ell = ell0 * q_sqrt<T, DIM>(n2);
      mu = rho * (pconst<T>(ph.q2, ph.q2f) * ell * ell * (-lam) + pconst<T>(ph.q1, ph.q1f) * ell * cs);
      for (int c = 0; c < DIM; ++c)
        for (int n = 0; n < DIM; ++n) sigma[c][n] += mu * eps[c][n];
    }
  }
  T inv = q_div<T, DIM>(cs, hmin) + q_div<T, DIM>(pconst<T>(ph.cfl_mu, ph.cfl_muf) * mu, rho * hmin * hmin);
  tau = inv > T(0) ? q_div<T, DIM>(pconst<T>(ph.cfl, ph.cflf), inv) : t_inf<T>();
  return 0;
}

}  // namespace lagh
