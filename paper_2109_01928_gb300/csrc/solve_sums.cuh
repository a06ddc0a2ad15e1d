// Mixed-precision weights, cost and gradient from the column sums (one thread per
// candidate), shared by the general kernel (kernels.cu) and the per-pole-count
// kernels launched after each bucket's column-sum pass (pass_b*.cu).
#pragma once
#include "common.cuh"

namespace debyefit {

// ------------------------------------------------------------------ cost from column sums (mixed)
// For the Debye columns c_i = 1/(1 + j w tau_i), partial fractions give
//   Re(c_i conj c_j) = (tau_i Re c_i + tau_j Re c_j) / (tau_i + tau_j),
// so the pole block of the Gram follows from the column sums S_i = sum_k re_i(k):
//   G_ij = (tau_i S_i + tau_j S_j) / (tau_i + tau_j),  G_ii = S_i  (re^2 + im^2 = re),
// and G_0i = S_i, G_00 = K for the eps_inf column. With h = A^T b and b^T b, the
// damped weights solve M x = h (M = G + lam diag G), and for the flipped x_hat
//   cost(x_hat) = b^T b - 2 x_hat^T h + x_hat^T M x_hat
// exactly. M, h, b^T b and the products with M are float-float (the subtraction
// loses the digits of b^T b / cost, about 4: float-float keeps ~9 of the ~13
// digits it carries); x comes from an FP32 Cholesky factor of the scaled M and
// refinement steps with the float-float residual h - M x.
constexpr int SUMS_REFINE = 2;       // refinement steps with the gradient (x and the adjoint w)
// Cost-only evaluations take one step: the scaled damped matrix C + lam I has unit
// diagonal, so kappa <= (n + lam) / lam (2e4 at n = 21, lam = 1e-3) and after one
// step the weights carry about (kappa 2^-24)^2 = 1.4e-6 relative error, which
// reaches a flipped candidate's cost at first order; two steps are ~2e-9.
constexpr int SUMS_REFINE_COST = 1;

// The packed FP32 factor L of one candidate: a per-thread array (float*), or a
// column of a block-wide shared array (SmemL: entry e of thread t at p[e * stride],
// stride = threads per block, so that a warp's accesses hit 32 consecutive words).
struct SmemL {
  float* p;
  int stride;
  __device__ __forceinline__ float& operator[](int e) const { return p[e * stride]; }
};
extern __shared__ float solve_l_smem[];
// Pole counts from which the per-N kernels keep L in shared memory: the compiler
// keeps a per-thread array of up to about 21 floats in registers, not a larger one.
constexpr int SOLVE_L_SMEM_FROM = 6;
__host__ __device__ constexpr int solve_npk(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr size_t solve_smem_per_thread(int N) {
  return N >= SOLVE_L_SMEM_FROM ? sizeof(float) * (size_t)solve_npk(N) : 0;
}

__device__ __forceinline__ ff gram_ff(int i, int j, const ff* tau, const ff* S, ff kk) {
  if (i == 0 && j == 0) return kk;
  if (i == 0) return S[j - 1];
  if (j == 0 || i == j) return S[i - 1];
  const ff num = ff_sum(ff_prod(tau[i - 1], S[i - 1]), ff_prod(tau[j - 1], S[j - 1]));
  return ff_quot(num, ff_sum(tau[i - 1], tau[j - 1]));
}

// Sources of the float-float Gram entries (i >= j): formed where they are used
// (the per-N kernels, whose compiler keeps what fits), or read from a per-thread
// packed table filled once (the general kernel, whose arrays are in local memory
// anyway).
struct GramRecompute {
  const ff* tau;
  const ff* S;
  ff kk;
  __device__ __forceinline__ ff operator()(int i, int j) const { return gram_ff(i, j, tau, S, kk); }
};
struct GramTable {
  const ff* g;   // packed lower triangle, entry (i, j) at pk(i, j)
  __device__ __forceinline__ ff operator()(int i, int j) const { return g[pk(i, j)]; }
};

// (M v)_i in float-float, M = G + lam diag G; each entry serves both of its rows.
template <class GA>
__device__ __forceinline__ void mvec_ff(int n, const GA& G, ff one_lam, const ff* v, ff* out) {
#pragma unroll
  for (int i = 0; i < n; ++i) out[i] = ff{0.f, 0.f};
#pragma unroll
  for (int i = 0; i < n; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const ff g = G(i, j);
      out[i] = ff_sum(out[i], ff_prod(g, v[j]));
      out[j] = ff_sum(out[j], ff_prod(g, v[i]));
    }
    out[i] = ff_sum(out[i], ff_prod(ff_prod(G(i, i), one_lam), v[i]));
  }
}

// FP32 Cholesky L L^T of the scaled damped matrix, with 1 / L_jj stored on the
// diagonal so that the solves multiply instead of dividing.
template <class LA>
__device__ __forceinline__ bool cholesky_rdiag(LA L, int n) {
#pragma unroll
  for (int j = 0; j < n; ++j) {
    float s = L[pk(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) s = __fmaf_rn(-L[pk(j, k)], L[pk(j, k)], s);
    if (!(s > 0.f) || !isfinite(s)) return false;
    const float inv = __frsqrt_rn(s);
    L[pk(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < n; ++i) {
      float v = L[pk(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v = __fmaf_rn(-L[pk(i, k)], L[pk(j, k)], v);
      L[pk(i, j)] = __fmul_rn(v, inv);
    }
  }
  return true;
}

// v <- (L L^T)^-1 v for the factor of cholesky_rdiag
template <class LA>
__device__ __forceinline__ void llt_solve_rdiag(LA L, float* v, int n) {
#pragma unroll
  for (int i = 0; i < n; ++i) {
    float s = v[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = __fmaf_rn(-L[pk(i, k)], v[k], s);
    v[i] = __fmul_rn(s, L[pk(i, i)]);
  }
#pragma unroll
  for (int i = n - 1; i >= 0; --i) {
    float s = v[i];
#pragma unroll
    for (int k = i + 1; k < n; ++k) s = __fmaf_rn(-L[pk(k, i)], v[k], s);
    v[i] = __fmul_rn(s, L[pk(i, i)]);
  }
}

// M^-1 rhs through the FP32 factor L of the scaled M (scaling dinv = diag(G)^-1/2),
// refined `steps` times against the float-float M.
template <class LA, class GA>
__device__ __forceinline__ bool refined_solve(int n, LA L, const float* dinv, const GA& G, ff one_lam,
                                              const ff* rhs, ff* x, ff* r, float* v, int steps) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < n; ++i) x[i] = ff{0.f, 0.f};
#pragma unroll
  for (int it = 0; it <= steps && ok; ++it) {
    // r = rhs - M x (the first step has x = 0), dx = M^-1 r through the FP32 factor
    if (it == 0) {
#pragma unroll
      for (int i = 0; i < n; ++i) r[i] = rhs[i];
    } else {
      mvec_ff(n, G, one_lam, x, r);
#pragma unroll
      for (int i = 0; i < n; ++i) r[i] = ff_sum(rhs[i], ff_neg(r[i]));
    }
#pragma unroll
    for (int i = 0; i < n; ++i) v[i] = __fmul_rn(r[i].h, dinv[i]);
    llt_solve_rdiag(L, v, n);
#pragma unroll
    for (int i = 0; i < n; ++i) {
      x[i] = ff_sum(x[i], ff{__fmul_rn(v[i], dinv[i]), 0.f});
      ok = ok && isfinite(x[i].h);
    }
  }
  return ok;
}

// Cost (and, with grad, its derivative in theta) from the column sums. The
// gradient of cost(x_hat) = b^T b - 2 x_hat^T h + x_hat^T M x_hat, x_hat = s * x*
// (s the signs of the flip), x* = M^-1 h, is (variable projection with an
// adjoint for the flip)
//   d cost / d theta_i = -2 x_hat_i E_i + x_hat^T M_i x_hat + 2 (w_i E_i - w^T M_i x*),
//   w = M^-1 (s * (M x_hat - h)),
// with M_i = dM / d theta_i nonzero in row and column i only:
//   (M_i)_{i0} = D_i,  (M_i)_{ii} = (1 + lam) D_i,
//   (M_i)_{ij} = tau_i D_i / (tau_i + tau_j) + ln10 tau_i tau_j (S_i - S_j) / (tau_i + tau_j)^2
// (the derivative of G_ij = (tau_i S_i + tau_j S_j)/(tau_i + tau_j), d tau_i = ln10 tau_i).
//
// NT = 0: any pole count (u.N at run time); the small systems live in per-thread
// local memory. NT > 0: every unit has NT poles (one launch per pole bucket), the
// loops have constant trip counts, unroll, and the systems stay in registers.
// GRAD (0 or 1) fixes whether the gradient is computed.
// From N = 9 the per-N kernels are held to about 170 registers (3 resident blocks of
// 128): with spills to L1 the extra resident warps hide more of the dependent chains
// (measured on whole table-mode mixed_1024 fits: 136.4 -> 132.2 ms; 128 registers:
// 130.7 ms, but 0.6 % slower in the direct mode, where the solve overlaps the passes).
template <int NT, int GRAD>
__global__ void __launch_bounds__(128, (NT >= 9 ? 3 : 1)) k_solve_sums_t(EvalArgs a, double* cost, double* weights,
                                                                      double* grad) {
  const int64_t Q = a.sc.Q;
  const int nmax = a.sc.nmax, nm1 = nmax + 1;
  const bool with_grad = GRAD < 0 ? grad != nullptr : GRAD > 0;
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int q = u.q0 + (int)threadIdx.x;
    if (q >= u.q1 || (a.active && !a.active[q])) continue;
    if (NT > 0 && u.N != NT) {
      set_status(a.status, DEBYE_EBOUNDS);
      continue;
    }
    const int N = NT > 0 ? NT : u.N, n = N + 1;
    // arrays sized for the compile-time pole count (NT > 0) so that they can live in registers
    constexpr int AN = NT > 0 ? NT : NMAX, AN1 = AN + 1, APK = AN1 * (AN1 + 1) / 2;
    constexpr bool L_SMEM = NT >= SOLVE_L_SMEM_FROM;
    ff tau[AN], S[AN], hv[AN1], x[AN1], r[AN1];
    float Lreg[L_SMEM ? 1 : APK], dinv[AN1], v[AN1];
    const auto L = [&] {
      if constexpr (L_SMEM) return SmemL{solve_l_smem + threadIdx.x, (int)blockDim.x};
      else return (float*)Lreg;
    }();
#pragma unroll
    for (int i = 0; i < N; ++i) {
      tau[i] = ff_of(a.sc.x[(int64_t)i * Q + q]);   // 10^theta_i from the column-sum pass
      S[i] = ff_of(a.sc.G[(int64_t)i * Q + q]);
      hv[i + 1] = ff_of(a.sc.G[(int64_t)(N + i) * Q + q]);
    }
    hv[0] = ff_of(a.h0[u.s]);
    const ff kk = ff_of((double)(u.k1 - u.k0));
    const ff one_lam = ff_of(1.0 + a.lam);
    // the general kernel's gradient variant keeps the entries in a table: its five
    // products with M outweigh the table's local-memory traffic (measured on N = 20:
    // cost and gradient 40.6 -> 35.5 ms; cost only, two products, 6.0 -> 7.5 ms)
    constexpr bool G_TABLE = NT == 0 && GRAD > 0;
    ff gtab[G_TABLE ? NPACK_MAX : 1];
    const auto G = [&] {
      if constexpr (!G_TABLE) {
        return GramRecompute{tau, S, kk};
      } else {
        for (int i = 0; i < n; ++i)
          for (int j = 0; j <= i; ++j) gtab[pk(i, j)] = gram_ff(i, j, tau, S, kk);
        return GramTable{gtab};
      }
    }();
    // FP32 Cholesky of the Marquardt-scaled damped matrix (unit diagonal + lam)
#pragma unroll
    for (int i = 0; i < n; ++i) dinv[i] = __frsqrt_rn(G(i, i).h);   // diag(G)^-1/2
#pragma unroll
    for (int i = 0; i < n; ++i) {
#pragma unroll
      for (int j = 0; j < i; ++j) L[pk(i, j)] = __fmul_rn(__fmul_rn(G(i, j).h, dinv[i]), dinv[j]);
      L[pk(i, i)] = (float)(1.0 + a.lam);
    }
    bool ok = cholesky_rdiag(L, n);
    if (ok) ok = refined_solve(n, L, dinv, G, one_lam, hv, x, r, v, with_grad ? SUMS_REFINE : SUMS_REFINE_COST);
    record_fail(a, q, u.s, ok);
    if (!ok) {
      if (cost) cost[q] = INFINITY;
      if (weights)
        for (int j = 0; j < nm1; ++j) weights[(int64_t)q * nm1 + j] = 0.0;
      if (with_grad)
        for (int j = 0; j < nmax; ++j) grad[(int64_t)q * nmax + j] = 0.0;
      continue;
    }
    // sign flip of negative d_eps (Sec. III-B), then the exact quadratic cost
    float sgn[AN1];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      sgn[i] = (i > 0 && x[i].h < 0.f) ? -1.f : 1.f;
      if (sgn[i] < 0.f) x[i] = ff_neg(x[i]);
    }
    mvec_ff(n, G, one_lam, x, r);   // r = M x_hat
    ff c = ff_of(a.bb[u.s]);
#pragma unroll
    for (int i = 0; i < n; ++i) {
      c = ff_sum(c, ff_neg(ff_prod(ff{__fmul_rn(2.f, x[i].h), __fmul_rn(2.f, x[i].l)}, hv[i])));
      c = ff_sum(c, ff_prod(x[i], r[i]));
    }
    double cv = ff_dbl(c);
    if (!isfinite(cv)) cv = INFINITY;
    if (cv < 0.0) cv = 0.0;
    if (cost) cost[q] = cv;
    if (weights) {
#pragma unroll
      for (int j = 0; j < n; ++j) weights[(int64_t)q * nm1 + j] = ff_dbl(x[j]);
      for (int j = n; j < nm1; ++j) weights[(int64_t)q * nm1 + j] = 0.0;
    }
    if (!with_grad) continue;
    // adjoint w = M^-1 (s * (M x_hat - h)); r becomes its right-hand side
    ff w[AN1], rw[AN1];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      r[i] = ff_sum(r[i], ff_neg(hv[i]));
      if (sgn[i] < 0.f) r[i] = ff_neg(r[i]);
    }
    if (!refined_solve(n, L, dinv, G, one_lam, r, w, rw, v, SUMS_REFINE)) {
      for (int j = 0; j < nmax; ++j) grad[(int64_t)q * nmax + j] = 0.0;
      continue;
    }
    const ff ln10 = ff_of(2.302585092994046);
    for (int i = N; i < nmax; ++i) grad[(int64_t)q * nmax + i] = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int I = i + 1;
      const ff Di = ff_of(a.sc.G[(int64_t)(2 * N + i) * Q + q]);
      const ff Ei = ff_of(a.sc.G[(int64_t)(3 * N + i) * Q + q]);
      // row i of M_i against x_hat, w and x* (x*_j = s_j x_hat_j), off the diagonal
      ff ax = ff_prod(Di, x[0]), aw = ff_prod(Di, w[0]), as = ax;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const ff rr = ff_quot(ff{1.f, 0.f}, ff_sum(tau[i], tau[j]));
        const ff t1 = ff_prod(ff_prod(tau[i], Di), rr);
        const ff t2 = ff_prod(ff_prod(ff_prod(ln10, ff_prod(tau[i], tau[j])), ff_sum(S[i], ff_neg(S[j]))),
                              ff_prod(rr, rr));
        const ff row = ff_sum(t1, t2);
        const ff xs = sgn[j + 1] < 0.f ? ff_neg(x[j + 1]) : x[j + 1];
        ax = ff_sum(ax, ff_prod(row, x[j + 1]));
        aw = ff_sum(aw, ff_prod(row, w[j + 1]));
        as = ff_sum(as, ff_prod(row, xs));
      }
      const ff diag = ff_prod(Di, one_lam);
      const ff xhI = x[I], wI = w[I];
      const ff xsI = sgn[I] < 0.f ? ff_neg(xhI) : xhI;
      // x_hat^T M_i x_hat = 2 x_hat_i ax + diag x_hat_i^2;  w^T M_i x* = w_i as + x*_i aw + diag w_i x*_i
      ff gsum = ff_neg(ff_prod(ff{__fmul_rn(2.f, xhI.h), __fmul_rn(2.f, xhI.l)}, Ei));
      gsum = ff_sum(gsum, ff_prod(ff{__fmul_rn(2.f, xhI.h), __fmul_rn(2.f, xhI.l)}, ax));
      gsum = ff_sum(gsum, ff_prod(diag, ff_prod(xhI, xhI)));
      ff adj = ff_prod(wI, Ei);
      adj = ff_sum(adj, ff_neg(ff_prod(wI, as)));
      adj = ff_sum(adj, ff_neg(ff_prod(xsI, aw)));
      adj = ff_sum(adj, ff_neg(ff_prod(diag, ff_prod(wI, xsI))));
      gsum = ff_sum(gsum, ff{__fmul_rn(2.f, adj.h), __fmul_rn(2.f, adj.l)});
      grad[(int64_t)q * nmax + i] = ff_dbl(gsum);
    }
  }
}

}  // namespace debyefit
