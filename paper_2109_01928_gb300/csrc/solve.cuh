// Per-candidate linear algebra of the damped least-squares step.
//
// With G = A^T A, h = A^T b (from the Gram pass) and Marquardt scaling
// D = diag(sqrt(G_ii)), the damped normal matrix M = G + lam diag(G) is
// D (C + lam I) D with C = D^-1 G D^-1 (unit diagonal). The factor L of
// (C + lam I) = L L^T (Cholesky) gives every solve needed here:
//   M^-1 v   = D^-1 (L L^T)^-1 D^-1 v
//   M v      = D L (L^T (D v))
//   v^T M v  = || L^T (D v) ||^2
// The factor and the products with it are computed in type T (the FP64 path
// instantiates double; the mixed path solves its systems in k_solve_sums, with
// an FP32 copy of the factor refined in float-float).
#pragma once
#include "common.cuh"

namespace debyefit {

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float sqrt_t(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_t(double a) { return sqrt(a); }

// L (packed lower, n x n) in place: Cholesky of the scaled damped matrix.
// Returns false if a pivot is not positive or not finite.
template <typename T>
__device__ __forceinline__ bool cholesky_packed(T* L, int n) {
  for (int j = 0; j < n; ++j) {
    T s = L[pk(j, j)];
    for (int k = 0; k < j; ++k) s = fma_t(-L[pk(j, k)], L[pk(j, k)], s);
    if (!(s > T(0)) || !isfinite(s)) return false;
    const T ljj = sqrt_t(s);
    L[pk(j, j)] = ljj;
    const T inv = T(1) / ljj;
    for (int i = j + 1; i < n; ++i) {
      T v = L[pk(i, j)];
      for (int k = 0; k < j; ++k) v = fma_t(-L[pk(i, k)], L[pk(j, k)], v);
      L[pk(i, j)] = v * inv;
    }
  }
  return true;
}

// v <- (L L^T)^-1 v
template <typename T>
__device__ __forceinline__ void llt_solve(const T* L, T* v, int n) {
  for (int i = 0; i < n; ++i) {
    T s = v[i];
    for (int k = 0; k < i; ++k) s = fma_t(-L[pk(i, k)], v[k], s);
    v[i] = s / L[pk(i, i)];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = v[i];
    for (int k = i + 1; k < n; ++k) s = fma_t(-L[pk(k, i)], v[k], s);
    v[i] = s / L[pk(i, i)];
  }
}

// out <- L^T v
template <typename T>
__device__ __forceinline__ void lt_mul(const T* L, const T* v, T* out, int n) {
  for (int i = 0; i < n; ++i) {
    T s = T(0);
    for (int k = i; k < n; ++k) s = fma_t(L[pk(k, i)], v[k], s);
    out[i] = s;
  }
}

// out <- L v
template <typename T>
__device__ __forceinline__ void l_mul(const T* L, const T* v, T* out, int n) {
  for (int i = 0; i < n; ++i) {
    T s = T(0);
    for (int k = 0; k <= i; ++k) s = fma_t(L[pk(i, k)], v[k], s);
    out[i] = s;
  }
}

// Candidate q's stored factor (element e at e * Q + q in the scratch, of type T).
template <typename T>
__device__ __forceinline__ const T* factor_base(const Scratch& sc) {
  return reinterpret_cast<const T*>(sc.L);
}
template <typename T>
__device__ __forceinline__ T* factor_base_w(const Scratch& sc) {
  return reinterpret_cast<T*>(sc.L);
}

}  // namespace debyefit
