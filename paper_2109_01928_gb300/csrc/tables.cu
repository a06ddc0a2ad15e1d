// Column-sum tables of the mixed precision's table variant (DEBYE_PREC_MIXED_TABLE).
//
// The Gram identity of Debye columns (G_ij = (tau_i S_i + tau_j S_j) / (tau_i + tau_j))
// leaves, per pole, the column sums S(theta) = sum_k re_k and h(theta) = a^T b (and
// their theta derivatives for the gradient): four functions of one variable per
// spectrum, whatever the candidate. They are tabulated once per call as piecewise
// Chebyshev interpolants over the spectrum's log10(tau) box (stored as polynomials in
// the segment's coordinate), and every candidate's sums are then read off by
// float-float Horner steps: O(TAB_NC) per pole instead of O(K).
//
// Accuracy: with s = ln tau^2, each term 1 / (1 + w_k^2 e^s) has its poles at
// Im s = +-pi, so every column sum is analytic in the strip |Im s| < pi and bounded
// there by 1 / sin(Im s) times the sum of |terms|. On a segment of TAB_W = 0.2
// decades (0.92 in s) the Chebyshev coefficients then decay by about 20 per degree
// (Bernstein-ellipse bound), and 12 coefficients reach ~1e-14 relative: measured on
// the mixed and tabulated workloads in FP64 (worst 1e-14 for S and h, 8e-14 for the
// derivatives), below the float-float node sums' own rounding (~1e-12).
#include <cmath>

#include "common.cuh"
#include "launch.h"

namespace debyefit {

// Chebyshev points of the first kind, the matching discrete cosine transform, and the
// monomial coefficients of the Chebyshev polynomials (integers, exact in FP64).
struct ChebConst {
  double xm[TAB_NC];            // x_m = cos(pi (m + 1/2) / NC)
  double dct[TAB_NC][TAB_NC];   // (2 / NC) cos(pi k (m + 1/2) / NC), row 0 halved
  double mono[TAB_NC][TAB_NC];  // T_j(x) = sum_k mono[j][k] x^k
};

static const ChebConst& cheb_const() {
  static ChebConst c = [] {
    ChebConst r{};
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < TAB_NC; ++m) r.xm[m] = std::cos(pi * (m + 0.5) / TAB_NC);
    for (int k = 0; k < TAB_NC; ++k)
      for (int m = 0; m < TAB_NC; ++m)
        r.dct[k][m] = (k == 0 ? 1.0 : 2.0) / TAB_NC * std::cos(pi * k * (m + 0.5) / TAB_NC);
    // T_0 = 1, T_1 = x, T_{j+1} = 2 x T_j - T_{j-1}
    r.mono[0][0] = 1.0;
    if (TAB_NC > 1) r.mono[1][1] = 1.0;
    for (int j = 1; j + 1 < TAB_NC; ++j)
      for (int k = 0; k < TAB_NC; ++k)
        r.mono[j + 1][k] = (k > 0 ? 2.0 * r.mono[j][k - 1] : 0.0) - r.mono[j - 1][k];
    return r;
  }();
  return c;
}

// Node thetas, pseudo-candidate-major: spectrum s owns rows qn0[s] .. qn0[s+1]-1 of
// theta_n[.][TAB_NODE_N]; node n = g NC + m (segment g, point m) sits at slot n of the
// spectrum's rows, theta = lo + TAB_W (g + 1/2 + x_m / 2); slots past the last node
// repeat it.
__global__ void k_tab_nodes(int64_t S, const int32_t* qn0, const int32_t* nseg, const double* lo,
                            ChebConst cc, double* theta_n) {
  for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
    const int64_t base = (int64_t)qn0[s] * TAB_NODE_N;
    const int slots = (qn0[s + 1] - qn0[s]) * TAB_NODE_N;
    const int nodes = nseg[s] * TAB_NC;
    const double l = lo[s];
    for (int n = threadIdx.x; n < slots; n += blockDim.x) {
      const int nn = n < nodes ? n : nodes - 1;
      const int g = nn / TAB_NC, m = nn % TAB_NC;
      theta_n[base + n] = l + TAB_W * ((double)g + 0.5 + 0.5 * cc.xm[m]);
    }
  }
}

// Coefficients of segment g and function f of spectrum s from the node pass's output:
// for node n, pseudo-candidate q = qn0[s] + n / TAB_NODE_N and pole i = n % TAB_NODE_N,
// the column-sum pass wrote S, h, dS, dh at G[(r TAB_NODE_N + i) Qn + q], r = 0..3, and
// tau at X[i Qn + q].
__global__ void k_tab_coef(int64_t S, const int32_t* qn0, const int32_t* nseg, const int64_t* seg0,
                           ChebConst cc, const double* G, const double* X, int64_t Qn, float2* coef) {
  for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
    const int items = nseg[s] * TAB_NF;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int g = it / TAB_NF, f = it % TAB_NF;
      double v[TAB_NC];
#pragma unroll
      for (int m = 0; m < TAB_NC; ++m) {
        const int n = g * TAB_NC + m;
        const int64_t q = qn0[s] + n / TAB_NODE_N;
        const int i = n % TAB_NODE_N;
        v[m] = f == 2 ? X[(int64_t)i * Qn + q] : G[(int64_t)((f < 2 ? f : f - 1) * TAB_NODE_N + i) * Qn + q];
      }
      double c[TAB_NC];
#pragma unroll
      for (int k = 0; k < TAB_NC; ++k) {
        c[k] = 0.0;
#pragma unroll
        for (int m = 0; m < TAB_NC; ++m) c[k] = fma(cc.dct[k][m], v[m], c[k]);
      }
      // monomial coefficients in x (the series' coefficients fall by ~20 a degree, the
      // Chebyshev polynomials' monomial coefficients grow by at most 1 + sqrt 2: the
      // monomial form is as well conditioned on [-1, 1])
      float2* out = coef + ((seg0[s] + g) * TAB_NF + f) * TAB_NC;
#pragma unroll
      for (int k = 0; k < TAB_NC; ++k) {
        double a = 0.0;
#pragma unroll
        for (int j = k; j < TAB_NC; ++j) a = fma(cc.mono[j][k], c[j], a);
        const float hi = __double2float_rn(a);
        out[k] = make_float2(hi, __double2float_rn(a - (double)hi));
      }
    }
  }
}

// f(x) = sum_k a_k x^k for x in [-1, 1] by Horner's rule in float-float. The
// coefficients are read two at a time (16-byte loads: every function's TAB_NC
// coefficients start on a multiple of TAB_NC * 8 = 96 bytes from the allocation),
// halving the load instructions, which bound this kernel on the L1 pipe.
static_assert(TAB_NC % 2 == 0 && (TAB_NC * sizeof(float2)) % 16 == 0, "paired coefficient loads");
__device__ __forceinline__ ff poly_ff(const float2* __restrict__ a, ff x) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  float4 c[TAB_NC / 2];
#pragma unroll
  for (int i = 0; i < TAB_NC / 2; ++i) c[i] = __ldg(a4 + i);
  ff acc{c[TAB_NC / 2 - 1].z, c[TAB_NC / 2 - 1].w};
#pragma unroll
  for (int k = TAB_NC - 2; k >= 0; --k) {
    const float4 q = c[k / 2];
    acc = ff_sum(ff_prod(acc, x), (k & 1) ? ff{q.z, q.w} : ff{q.x, q.y});
  }
  return acc;
}

// The four column sums of one pole directly over the spectrum's samples in FP64, for a
// theta outside the table (or not finite): S, h, dS/dtheta, dh/dtheta as the
// column-sum pass defines them.
template <bool GRAD>
__device__ void direct_sums(const EvalArgs& a, const Unit& u, double tau, double* out) {
  constexpr double LN10 = 2.302585092994046;
  double S = 0.0, A = 0.0, C = 0.0, U = 0.0, V = 0.0, W = 0.0;
#pragma unroll 1
  for (int64_t k = u.k0; k < u.k1; ++k) {
    const double om = a.omega[k];
    const double x = om * tau;
    const double re = 1.0 / (1.0 + x * x);
    const double er = a.eps_re[k], wi = om * a.eps_im[k];
    S += re;
    A += re * er;
    C += re * wi;
    if (GRAD) {
      const double uu = x * x * re * re;
      U += uu;
      V += uu * er;
      W += uu * wi;
    }
  }
  out[0] = S;
  out[1] = A + tau * C;
  out[2] = -2.0 * LN10 * U;
  out[3] = LN10 * (-2.0 * V + tau * (C - 2.0 * W));
}

// Column sums of every (candidate, pole) of the units from the tables, written where
// the column-sum pass writes them (tau to sc.x row i; S, h, dS, dh to G rows i, N + i,
// 2N + i, 3N + i) for the column-sum solves. One thread per (candidate, pole).
template <bool GRAD>
__global__ void __launch_bounds__(128) k_tab_eval(EvalArgs a) {
  const int64_t Q = a.sc.Q;
  double* G = a.sc.G;
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int nc = u.q1 - u.q0, N = u.N;
    const double l = a.tab.lo[u.s];
    const int ns = a.tab.nseg[u.s];
    const float2* cs = a.tab.coef + a.tab.seg0[u.s] * (TAB_NF * TAB_NC);
    for (int p = threadIdx.x; p < nc * N; p += blockDim.x) {
      const int j = p / nc, q = u.q0 + p % nc;
      if (a.active && !a.active[q]) continue;
      const double th = a.theta[(int64_t)q * a.sc.nmax + j];
      const double d = th - l;
      const double uu = d * TAB_INV_W;
      double tau, v[4] = {0.0, 0.0, 0.0, 0.0};
      if (uu >= 0.0 && uu <= (double)ns) {
        // x = 2 (uu - g) - 1 in [-1, 1]; the FP64 work stays a handful of operations
        const int g = min((int)uu, ns - 1);
        const ff x = ff_of(fma(d, 2.0 * TAB_INV_W, -(double)(2 * g + 1)));
        const float2* c = cs + (int64_t)g * (TAB_NF * TAB_NC);
        v[0] = ff_dbl(poly_ff(c, x));
        v[1] = ff_dbl(poly_ff(c + TAB_NC, x));
        tau = ff_dbl(poly_ff(c + 2 * TAB_NC, x));
        if (GRAD) {
          v[2] = ff_dbl(poly_ff(c + 3 * TAB_NC, x));
          v[3] = ff_dbl(poly_ff(c + 4 * TAB_NC, x));
        }
      } else {
        tau = exp10(th);
        direct_sums<GRAD>(a, u, tau, v);
      }
      a.sc.x[(int64_t)j * Q + q] = tau;
      G[(int64_t)j * Q + q] = v[0];
      G[(int64_t)(N + j) * Q + q] = v[1];
      if (GRAD) {
        G[(int64_t)(2 * N + j) * Q + q] = v[2];
        G[(int64_t)(3 * N + j) * Q + q] = v[3];
      }
    }
  }
}

void launch_tab_nodes(int64_t S, const int32_t* qn0, const int32_t* nseg, const double* lo, double* theta_n,
                      int sms, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)sms * 32));
  k_tab_nodes<<<grid, 128, 0, st>>>(S, qn0, nseg, lo, cheb_const(), theta_n);
}

void launch_tab_coef(int64_t S, const int32_t* qn0, const int32_t* nseg, const int64_t* seg0, const double* G,
                     const double* X, int64_t Qn, float2* coef, int sms, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(S, (int64_t)sms * 32));
  k_tab_coef<<<grid, 128, 0, st>>>(S, qn0, nseg, seg0, cheb_const(), G, X, Qn, coef);
}

void launch_tab_eval(const EvalArgs& a, bool grad, int sms, cudaStream_t st) {
  const int grid = std::max(1, std::min(a.n_units, sms * 16));
  if (grad) k_tab_eval<true><<<grid, 128, 0, st>>>(a);
  else k_tab_eval<false><<<grid, 128, 0, st>>>(a);
}

}  // namespace debyefit
