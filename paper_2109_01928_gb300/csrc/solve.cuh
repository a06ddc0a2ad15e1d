// FP64 per-candidate linear algebra of the damped least-squares step.
//
// With G = A^T A, h = A^T b (from the Gram pass) and Marquardt scaling
// D = diag(sqrt(G_ii)), the damped normal matrix M = G + lam diag(G) is
// D (C + lam I) D with C = D^-1 G D^-1 (unit diagonal). The factor L of
// (C + lam I) = L L^T (Cholesky, FP64) gives every solve needed here:
//   M^-1 v   = D^-1 (L L^T)^-1 D^-1 v
//   M v      = D L (L^T (D v))
//   v^T M v  = || L^T (D v) ||^2
#pragma once
#include "common.cuh"

namespace debyefit {

// L (packed lower, n x n) in place: Cholesky of the scaled damped matrix.
// Returns false if a pivot is not positive or not finite.
__device__ __forceinline__ bool cholesky_packed(double* L, int n) {
  for (int j = 0; j < n; ++j) {
    double s = L[pk(j, j)];
    for (int k = 0; k < j; ++k) s = fma(-L[pk(j, k)], L[pk(j, k)], s);
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double ljj = sqrt(s);
    L[pk(j, j)] = ljj;
    const double inv = 1.0 / ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = L[pk(i, j)];
      for (int k = 0; k < j; ++k) v = fma(-L[pk(i, k)], L[pk(j, k)], v);
      L[pk(i, j)] = v * inv;
    }
  }
  return true;
}

// v <- (L L^T)^-1 v
__device__ __forceinline__ void llt_solve(const double* L, double* v, int n) {
  for (int i = 0; i < n; ++i) {
    double s = v[i];
    for (int k = 0; k < i; ++k) s = fma(-L[pk(i, k)], v[k], s);
    v[i] = s / L[pk(i, i)];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = v[i];
    for (int k = i + 1; k < n; ++k) s = fma(-L[pk(k, i)], v[k], s);
    v[i] = s / L[pk(i, i)];
  }
}

// out <- L^T v
__device__ __forceinline__ void lt_mul(const double* L, const double* v, double* out, int n) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = i; k < n; ++k) s = fma(L[pk(k, i)], v[k], s);
    out[i] = s;
  }
}

// out <- L v
__device__ __forceinline__ void l_mul(const double* L, const double* v, double* out, int n) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s = fma(L[pk(i, k)], v[k], s);
    out[i] = s;
  }
}

}  // namespace debyefit
