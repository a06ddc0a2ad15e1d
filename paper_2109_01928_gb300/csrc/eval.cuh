// Per-N passes over the frequency samples of one candidate (one thread per
// candidate, all threads of a warp belong to the same spectrum, so every
// per-sample load is a warp-uniform broadcast).
//
//   gram_unit    G = A^T A (packed, (N+1)x(N+1)) and h = A^T b of the stacked
//                real basis of Eq. 7 (rows: eps' and eps'' of every sample).
//   refine_unit  r = b - A x at the current weights, rr = ||r||^2 and t = A^T r.
//   grad_unit    projections of the derivative columns needed by the
//                variable-projection gradient.
//
// MIXED = true : FP32 basis and Gram (Sec. 8a rows a2/a3 on the FP32 pipe);
//                residual in float-float, so rr carries ~2^-44 relative error.
// MIXED = false: everything in FP64.
#pragma once
#include "common.cuh"

namespace debyefit {

template <int N>
struct Acc {
  static constexpr int NP = N * (N + 1) / 2;
};

// Samples summed in registers before a mixed-precision Gram block is added to
// the shared-memory accumulators.
constexpr int GRAM_BLOCK = 64;

// Shared-memory floats per thread needed by the mixed Gram pass for N poles
// (2N + N(N+1)/2 accumulators, rounded up to an odd stride).
__host__ __device__ constexpr int gram_smem_stride(int N) { return (2 * N + N * (N + 1) / 2) | 1; }

extern __shared__ __align__(16) unsigned char dyn_smem[];

// ------------------------------------------------------------------ Gram
template <int N, bool MIXED>
__device__ __forceinline__ void gram_unit(const EvalArgs& a, const Unit& u) {
  const int q = u.q0 + (int)threadIdx.x;
  if (q >= u.q1) return;
  if (a.active && !a.active[q]) return;
  constexpr int NP = Acc<N>::NP;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  if constexpr (MIXED) {
    // Two-level FP32 accumulation: registers sum GRAM_BLOCK consecutive samples,
    // then each block is added into this thread's slice of shared memory (entry e
    // of thread t at outer[t * SA + e], SA odd and known at compile time, so every
    // access is an immediate offset). The rounding error then grows like
    // (GRAM_BLOCK + K / GRAM_BLOCK) instead of K.
    constexpr int SA = gram_smem_stride(N);
    float* outer = reinterpret_cast<float*>(dyn_smem) + threadIdx.x * SA;
    constexpr int bs = 1;
#pragma unroll
    for (int e = 0; e < SA; ++e) outer[e] = 0.f;
    float tau[N];
#pragma unroll
    for (int i = 0; i < N; ++i) tau[i] = __double2float_rn(exp10(th[i]));
    for (int64_t kb = u.k0; kb < u.k1; kb += GRAM_BLOCK) {
      const int64_t ke = min(u.k1, kb + (int64_t)GRAM_BLOCK);
      float g0[N], hv[N], gp[NP];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        g0[i] = 0.f;
        hv[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) gp[i] = 0.f;
#pragma unroll 1
      for (int64_t k = kb; k < ke; ++k) {
        const float4 v = __ldg(&a.kf32[k]);
        float re[N], im[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float x = v.x * tau[i];
          const float r = rcp_approx(fmaf(x, x, 1.0f));
          re[i] = r;
          im[i] = x * r;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          g0[i] += re[i];
          hv[i] = fmaf(re[i], v.y, fmaf(im[i], v.z, hv[i]));
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int j = 0; j <= i; ++j)
            gp[i * (i + 1) / 2 + j] = fmaf(re[i], re[j], fmaf(im[i], im[j], gp[i * (i + 1) / 2 + j]));
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        outer[i * bs] += g0[i];
        outer[(N + i) * bs] += hv[i];
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) outer[(2 * N + i) * bs] += gp[i];
    }
    double* G = a.sc.G;
    G[(int64_t)pk(0, 0) * Q + q] = (double)(u.k1 - u.k0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      G[(int64_t)pk(i + 1, 0) * Q + q] = (double)outer[i * bs];
#pragma unroll
      for (int j = 0; j <= i; ++j)
        G[(int64_t)pk(i + 1, j + 1) * Q + q] = (double)outer[(2 * N + i * (i + 1) / 2 + j) * bs];
    }
    const int hb = (a.sc.nmax + 1) * (a.sc.nmax + 2) / 2;
    G[(int64_t)hb * Q + q] = a.h0[u.s];
#pragma unroll
    for (int i = 0; i < N; ++i) G[(int64_t)(hb + 1 + i) * Q + q] = (double)outer[(N + i) * bs];
  } else {
    double tau[N], g0[N], hv[N], gp[NP];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      tau[i] = exp10(th[i]);
      g0[i] = 0.0;
      hv[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) gp[i] = 0.0;
#pragma unroll 1
    for (int64_t k = u.k0; k < u.k1; ++k) {
      const double w = __ldg(&a.omega[k]);
      const double br = __ldg(&a.eps_re[k]);
      const double bi = __ldg(&a.eps_im[k]);
      double re[N], im[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double x = w * tau[i];
        const double r = 1.0 / fma(x, x, 1.0);
        re[i] = r;
        im[i] = x * r;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        g0[i] += re[i];
        hv[i] = fma(re[i], br, fma(im[i], bi, hv[i]));
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j)
          gp[i * (i + 1) / 2 + j] = fma(re[i], re[j], fma(im[i], im[j], gp[i * (i + 1) / 2 + j]));
    }
    double* G = a.sc.G;
    G[(int64_t)pk(0, 0) * Q + q] = (double)(u.k1 - u.k0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      G[(int64_t)pk(i + 1, 0) * Q + q] = g0[i];
#pragma unroll
      for (int j = 0; j <= i; ++j) G[(int64_t)pk(i + 1, j + 1) * Q + q] = gp[i * (i + 1) / 2 + j];
    }
    const int hb = (a.sc.nmax + 1) * (a.sc.nmax + 2) / 2;
    G[(int64_t)hb * Q + q] = a.h0[u.s];
#pragma unroll
    for (int i = 0; i < N; ++i) G[(int64_t)(hb + 1 + i) * Q + q] = hv[i];
  }
}

// ------------------------------------------------------------------ residual pass
// Reads the weights x (FP64) of candidate q, writes rt[0] = ||b - A x||^2 and
// rt[1 + j] = (A^T (b - A x))_j, j = 0..N.
template <int N, bool MIXED>
__device__ __forceinline__ void refine_unit(const EvalArgs& a, const Unit& u) {
  const int q = u.q0 + (int)threadIdx.x;
  if (q >= u.q1) return;
  if (a.active && !a.active[q]) return;
  if (a.sc.fail[q]) return;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  const double* X = a.sc.x;
  if constexpr (MIXED) {
    // t = A^T r is a float-float dot product (Dot2) of the float-float basis and
    // residual: the refinement step multiplies its error by M^-1, large along
    // nearly collinear poles, and a flipped cost is first-order in the weights.
    float th_[N], tl_[N], wh[N], wl[N], th_t[N], tl_t[N];
    float w0h, w0l;
    split_double(X[q], w0h, w0l);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      split_double(exp10(th[i]), th_[i], tl_[i]);
      split_double(X[(int64_t)(i + 1) * Q + q], wh[i], wl[i]);
      th_t[i] = 0.f;
      tl_t[i] = 0.f;
    }
    float t0h = 0.f, t0l = 0.f, rrh = 0.f, rrl = 0.f;
#pragma unroll 1
    for (int64_t k = u.k0; k < u.k1; ++k) {
      const float4 vh = __ldg(&a.kf32[k]);
      const float4 vl = __ldg(&a.kff[k]);
      float reh[N], rel[N], imh[N], iml[N];
      // residual of the real row: eps' - eps_inf - sum x_i re_i
      float arh, arl, aih, ail;
      two_sum(vh.y, -w0h, arh, arl);
      arl = __fadd_rn(arl, __fsub_rn(vl.y, w0l));
      aih = vh.z;
      ail = vl.z;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float xh;
        basis_ff(vh.x, vl.x, th_[i], tl_[i], reh[i], rel[i], imh[i], iml[i], xh);
        ff_sub_prod(arh, arl, wh[i], wl[i], reh[i], rel[i]);
        ff_sub_prod(aih, ail, wh[i], wl[i], imh[i], iml[i]);
      }
      ff_norm(arh, arl);
      ff_norm(aih, ail);
      ff_add(rrh, rrl, __fmul_rn(arh, arh));
      ff_add(rrh, rrl, __fmul_rn(aih, aih));
      ff_add(t0h, t0l, arh);
      t0l = __fadd_rn(t0l, arl);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        ff_add_prod(th_t[i], tl_t[i], reh[i], rel[i], arh, arl);
        ff_add_prod(th_t[i], tl_t[i], imh[i], iml[i], aih, ail);
      }
    }
    double* R = a.sc.rt;
    R[q] = (double)rrh + (double)rrl;
    R[Q + q] = (double)t0h + (double)t0l;
#pragma unroll
    for (int i = 0; i < N; ++i) R[(int64_t)(i + 2) * Q + q] = (double)th_t[i] + (double)tl_t[i];
  } else {
    double tau[N], w[N], t[N];
    const double w0 = X[q];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      tau[i] = exp10(th[i]);
      w[i] = X[(int64_t)(i + 1) * Q + q];
      t[i] = 0.0;
    }
    double t0 = 0.0, rr = 0.0;
#pragma unroll 1
    for (int64_t k = u.k0; k < u.k1; ++k) {
      const double om = __ldg(&a.omega[k]);
      double ar = __ldg(&a.eps_re[k]) - w0;
      double ai = __ldg(&a.eps_im[k]);
      double re[N], im[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double x = om * tau[i];
        const double r = 1.0 / fma(x, x, 1.0);
        re[i] = r;
        im[i] = x * r;
        ar = fma(-w[i], re[i], ar);
        ai = fma(-w[i], im[i], ai);
      }
      rr = fma(ar, ar, fma(ai, ai, rr));
      t0 += ar;
#pragma unroll
      for (int i = 0; i < N; ++i) t[i] = fma(re[i], ar, fma(im[i], ai, t[i]));
    }
    double* R = a.sc.rt;
    R[q] = rr;
    R[Q + q] = t0;
#pragma unroll
    for (int i = 0; i < N; ++i) R[(int64_t)(i + 2) * Q + q] = t[i];
  }
}

// ------------------------------------------------------------------ gradient pass
// With x1 (unflipped, sc.x), x_hat (flipped, sc.xh) and w = M^-1 S g_hat (sc.w):
//   gt[i]        = a_i'^T r_hat,  r_hat = b - A x_hat
//   gt[N + i]    = a_i^T a_i'
//   gt[2N + i]   = a_i'^T r,      r = r_hat + A (x_hat - x1)
//   gt[3N + i]   = a_i'^T (A w)
// where a_i' = d a_i / d log10(tau_i).
template <int N, bool MIXED>
__device__ __forceinline__ void grad_unit(const EvalArgs& a, const Unit& u) {
  const int q = u.q0 + (int)threadIdx.x;
  if (q >= u.q1) return;
  if (a.active && !a.active[q]) return;
  if (a.sc.fail[q]) return;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  constexpr float LN10F = 2.302585092994046f;
  constexpr double LN10 = 2.302585092994046;
  if constexpr (MIXED) {
    // Both residuals are float-float: r_hat = b - A x_hat and r = b - A x1 (in a
    // flipped candidate r_hat is large and r small, so r is not formed as
    // r_hat + A e). The projections are summed with TwoSum.
    float th_[N], tl_[N], xhh[N], xhl[N], x1h[N], x1l[N], w[N];
    float trh_h[N], trh_l[N], taa[N], tr_h[N], tr_l[N], taw_h[N], taw_l[N];
    float x0h, x0l, x10h, x10l;
    split_double(a.sc.xh[q], x0h, x0l);
    split_double(a.sc.x[q], x10h, x10l);
    const float w0 = __double2float_rn(a.sc.w[q]);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      split_double(exp10(th[i]), th_[i], tl_[i]);
      split_double(a.sc.xh[(int64_t)(i + 1) * Q + q], xhh[i], xhl[i]);
      split_double(a.sc.x[(int64_t)(i + 1) * Q + q], x1h[i], x1l[i]);
      w[i] = __double2float_rn(a.sc.w[(int64_t)(i + 1) * Q + q]);
      trh_h[i] = trh_l[i] = taa[i] = tr_h[i] = tr_l[i] = taw_h[i] = taw_l[i] = 0.f;
    }
#pragma unroll 1
    for (int64_t k = u.k0; k < u.k1; ++k) {
      const float4 vh = __ldg(&a.kf32[k]);
      const float4 vl = __ldg(&a.kff[k]);
      float reh[N], imh[N], xv[N];
      float hrh, hrl, hih, hil, rrh, rrl, rih, ril;
      two_sum(vh.y, -x0h, hrh, hrl);
      hrl = __fadd_rn(hrl, __fsub_rn(vl.y, x0l));
      hih = vh.z;
      hil = vl.z;
      two_sum(vh.y, -x10h, rrh, rrl);
      rrl = __fadd_rn(rrl, __fsub_rn(vl.y, x10l));
      rih = vh.z;
      ril = vl.z;
      float awr = w0, awi = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float rel, iml;
        basis_ff(vh.x, vl.x, th_[i], tl_[i], reh[i], rel, imh[i], iml, xv[i]);
        ff_sub_prod(hrh, hrl, xhh[i], xhl[i], reh[i], rel);
        ff_sub_prod(hih, hil, xhh[i], xhl[i], imh[i], iml);
        ff_sub_prod(rrh, rrl, x1h[i], x1l[i], reh[i], rel);
        ff_sub_prod(rih, ril, x1h[i], x1l[i], imh[i], iml);
        awr = fmaf(w[i], reh[i], awr);
        awi = fmaf(w[i], imh[i], awi);
      }
      const float rhr = __fadd_rn(hrh, hrl), rhi = __fadd_rn(hih, hil);
      const float rr = __fadd_rn(rrh, rrl), ri = __fadd_rn(rih, ril);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float x = xv[i], re = reh[i];
        const float re2l = re * re * LN10F;
        const float dre = -2.0f * x * x * re2l;
        const float dim = x * (1.0f - x * x) * re2l;
        ff_add(trh_h[i], trh_l[i], __fmaf_rn(dim, rhi, __fmul_rn(dre, rhr)));
        taa[i] = fmaf(re, dre, fmaf(imh[i], dim, taa[i]));
        ff_add(tr_h[i], tr_l[i], __fmaf_rn(dim, ri, __fmul_rn(dre, rr)));
        ff_add(taw_h[i], taw_l[i], __fmaf_rn(dim, awi, __fmul_rn(dre, awr)));
      }
    }
    double* T = a.sc.gt;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T[(int64_t)i * Q + q] = (double)trh_h[i] + (double)trh_l[i];
      T[(int64_t)(N + i) * Q + q] = taa[i];
      T[(int64_t)(2 * N + i) * Q + q] = (double)tr_h[i] + (double)tr_l[i];
      T[(int64_t)(3 * N + i) * Q + q] = (double)taw_h[i] + (double)taw_l[i];
    }
  } else {
    double tau[N], xh[N], e[N], w[N];
    double t_rh[N], t_aa[N], t_r[N], t_aw[N];
    const double x0 = a.sc.xh[q];
    const double e0 = a.sc.xh[q] - a.sc.x[q];
    const double w0 = a.sc.w[q];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      tau[i] = exp10(th[i]);
      xh[i] = a.sc.xh[(int64_t)(i + 1) * Q + q];
      e[i] = xh[i] - a.sc.x[(int64_t)(i + 1) * Q + q];
      w[i] = a.sc.w[(int64_t)(i + 1) * Q + q];
      t_rh[i] = t_aa[i] = t_r[i] = t_aw[i] = 0.0;
    }
#pragma unroll 1
    for (int64_t k = u.k0; k < u.k1; ++k) {
      const double om = __ldg(&a.omega[k]);
      double rhr = __ldg(&a.eps_re[k]) - x0, rhi = __ldg(&a.eps_im[k]);
      double aer = e0, aei = 0.0, awr = w0, awi = 0.0;
      double re[N], im[N], xv[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double x = om * tau[i];
        const double r = 1.0 / fma(x, x, 1.0);
        xv[i] = x;
        re[i] = r;
        im[i] = x * r;
        rhr = fma(-xh[i], re[i], rhr);
        rhi = fma(-xh[i], im[i], rhi);
        aer = fma(e[i], re[i], aer);
        aei = fma(e[i], im[i], aei);
        awr = fma(w[i], re[i], awr);
        awi = fma(w[i], im[i], awi);
      }
      const double rr = rhr + aer, ri = rhi + aei;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double x = xv[i];
        const double re2l = re[i] * re[i] * LN10;
        const double dre = -2.0 * x * x * re2l;
        const double dim = x * (1.0 - x * x) * re2l;
        t_rh[i] = fma(dre, rhr, fma(dim, rhi, t_rh[i]));
        t_aa[i] = fma(re[i], dre, fma(im[i], dim, t_aa[i]));
        t_r[i] = fma(dre, rr, fma(dim, ri, t_r[i]));
        t_aw[i] = fma(dre, awr, fma(dim, awi, t_aw[i]));
      }
    }
    double* T = a.sc.gt;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T[(int64_t)i * Q + q] = t_rh[i];
      T[(int64_t)(N + i) * Q + q] = t_aa[i];
      T[(int64_t)(2 * N + i) * Q + q] = t_r[i];
      T[(int64_t)(3 * N + i) * Q + q] = t_aw[i];
    }
  }
}

// ------------------------------------------------------------------ N dispatch
template <int PH, int N, bool MIXED>
__device__ __forceinline__ void run_phase(const EvalArgs& a, const Unit& u) {
  if constexpr (PH == PH_GRAM) gram_unit<N, MIXED>(a, u);
  else if constexpr (PH == PH_REFINE) refine_unit<N, MIXED>(a, u);
  else grad_unit<N, MIXED>(a, u);
}

template <int PH, int LO, int HI, bool MIXED>
__device__ __forceinline__ void dispatch_n(const EvalArgs& a, const Unit& u) {
  if constexpr (LO <= HI) {
    if (u.N == LO) run_phase<PH, LO, MIXED>(a, u);
    else dispatch_n<PH, LO + 1, HI, MIXED>(a, u);
  }
}

// One block per unit (grid-stride over the unit list); LO..HI is the pole
// bucket compiled into this kernel.
template <int PH, int LO, int HI, bool MIXED>
__global__ void __launch_bounds__(256) k_pass(EvalArgs a) {
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    if (u.N < LO || u.N > HI) {
      if (threadIdx.x == 0) set_status(a.status, DEBYE_EBOUNDS);
      continue;
    }
    dispatch_n<PH, LO, HI, MIXED>(a, u);
  }
}

}  // namespace debyefit
