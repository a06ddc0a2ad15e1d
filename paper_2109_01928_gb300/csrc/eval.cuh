// Per-N passes over the frequency samples of one candidate.
//
// Thread mapping: a group of `ks` consecutive lanes (ks = a.ks, a power of two
// <= 32) evaluates one candidate; lane `slice` of the group sums the samples
// k0 + slice, k0 + slice + ks, ... and the group then reduces its partial sums
// with warp shuffles. All lanes of a block belong to the same spectrum. ks = 1
// (one thread per candidate, every per-sample load a warp-wide broadcast) is
// used for full populations; ks > 1 keeps warps full when a spectrum has only
// a few candidates (line-search points, one re-solve per spectrum).
//
// Mixed precision (float-float on the FP32 pipe):
//   sums_sq_unit column sums S_i = sum re_i and h = A^T b of the Debye basis (and,
//                for the gradient, the same sums over the derivative columns),
//                from which k_solve_sums forms the Gram, weights, cost and gradient.
// FP64 precision:
//   gram_unit    G = A^T A (packed, (N+1)x(N+1)) and h = A^T b of the stacked
//                real basis of Eq. 7 (rows: eps' and eps'' of every sample).
//   refine_unit  r = b - A x at the current weights, rr = ||r||^2 and t = A^T r.
//   grad_unit    projections of the derivative columns needed by the
//                variable-projection gradient.
//
// No lane returns before the group reduction: lanes without a candidate (the
// tail of a unit, masked line-search points) contribute zeros.
#pragma once
#include "common.cuh"

namespace debyefit {

template <int N>
struct Acc {
  static constexpr int NP = N * (N + 1) / 2;
};


// ------------------------------------------------------------------ group reductions
__device__ __forceinline__ float group_sum(float v, int ks) {
  for (int o = ks >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double group_sum(double v, int ks) {
  for (int o = ks >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Float-float sum over the group: leading parts by TwoSum, low parts added.
__device__ __forceinline__ void group_sum_ff(float& h, float& l, int ks) {
  for (int o = ks >> 1; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
    float s, e;
    two_sum(h, h2, s, e);
    h = s;
    l = __fadd_rn(__fadd_rn(l, l2), e);
  }
}

struct Lane {
  int q;       // candidate
  int slice;   // sample phase within the group
  int ks;      // lanes per candidate
  bool act;    // this lane's candidate is evaluated
};

__device__ __forceinline__ Lane lane_of(const EvalArgs& a, const Unit& u, bool need_ok) {
  Lane l;
  l.ks = a.ks;
  l.slice = (int)threadIdx.x & (a.ks - 1);
  l.q = u.q0 + (int)threadIdx.x / a.ks;
  l.act = l.q < u.q1;
  if (l.act && a.active) l.act = a.active[l.q] != 0;
  if (l.act && need_ok) l.act = a.sc.fail[l.q] == 0;
  return l;
}

// ------------------------------------------------------------------ Gram
template <int N>
__device__ __forceinline__ void gram_unit(const EvalArgs& a, const Unit& u) {
  const Lane ln = lane_of(a, u, false);
  const int q = ln.act ? ln.q : u.q0;
  constexpr int NP = Acc<N>::NP;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  const int64_t kbeg = u.k0 + ln.slice;
  double tau[N], g0[N], hv[N], gp[NP];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    tau[i] = ln.act ? exp10(th[i]) : 0.0;
    g0[i] = 0.0;
    hv[i] = 0.0;
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) gp[i] = 0.0;
  const int64_t kend = ln.act ? u.k1 : kbeg;
#pragma unroll 1
  for (int64_t k = kbeg; k < kend; k += ln.ks) {
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
  const bool wr = ln.act && ln.slice == 0;
  double* G = a.sc.G;
  const int hb = (a.sc.nmax + 1) * (a.sc.nmax + 2) / 2;
  if (wr) {
    G[(int64_t)pk(0, 0) * Q + q] = (double)(u.k1 - u.k0);
    G[(int64_t)hb * Q + q] = a.h0[u.s];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double g0s = group_sum(g0[i], ln.ks);
    const double hs = group_sum(hv[i], ln.ks);
    if (wr) {
      G[(int64_t)pk(i + 1, 0) * Q + q] = g0s;
      G[(int64_t)(hb + 1 + i) * Q + q] = hs;
    }
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const double v = group_sum(gp[i * (i + 1) / 2 + j], ln.ks);
      if (wr) G[(int64_t)pk(i + 1, j + 1) * Q + q] = v;
    }
  }

}

// ------------------------------------------------------------------ Gram from FP64 column sums
// The FP64 path's Gram G and h = A^T b by the partial-fraction identity of the Debye
// columns (the mixed path's algebra, in plain FP64): the pass sums, per pole,
//   S_i = sum_k re_i(k),   h_i = sum_k re_i(k) eps'_k + tau_i sum_k re_i(k) (omega_k eps''_k)
// (im = omega tau re) with re = 1/(1 + omega^2 tau^2), and writes the packed Gram
//   G_00 = K, G_i0 = G_ii = S_i, G_ij = (tau_i S_i + tau_j S_j) / (tau_i + tau_j)
// in gram_unit's layout, so the FP64 solve, residual passes and finish follow unchanged
// (the cost comes from the residual pass, free of the cancellation of b^T b - x^T h).
template <int N>
__device__ __forceinline__ void gram_sums_unit(const EvalArgs& a, const Unit& u) {
  const Lane ln = lane_of(a, u, false);
  const int q = ln.act ? ln.q : u.q0;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  const int64_t kbeg = u.k0 + ln.slice;
  const int64_t kend = ln.act ? u.k1 : kbeg;
  double tau[N], t2[N], sv[N], av[N], bv[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    tau[i] = ln.act ? exp10(th[i]) : 0.0;
    t2[i] = tau[i] * tau[i];
    sv[i] = av[i] = bv[i] = 0.0;
  }
#pragma unroll 1
  for (int64_t k = kbeg; k < kend; k += ln.ks) {
    const double w = __ldg(&a.omega[k]);
    const double er = __ldg(&a.eps_re[k]);
    const double wei = w * __ldg(&a.eps_im[k]);
    const double w2 = w * w;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double r = 1.0 / fma(w2, t2[i], 1.0);
      sv[i] += r;
      av[i] = fma(r, er, av[i]);
      bv[i] = fma(r, wei, bv[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    sv[i] = group_sum(sv[i], ln.ks);
    av[i] = group_sum(av[i], ln.ks);
    bv[i] = group_sum(bv[i], ln.ks);
  }
  if (!(ln.act && ln.slice == 0)) return;
  double* G = a.sc.G;
  const int hb = (a.sc.nmax + 1) * (a.sc.nmax + 2) / 2;
  G[(int64_t)pk(0, 0) * Q + q] = (double)(u.k1 - u.k0);
  G[(int64_t)hb * Q + q] = a.h0[u.s];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    G[(int64_t)pk(i + 1, 0) * Q + q] = sv[i];
    G[(int64_t)pk(i + 1, i + 1) * Q + q] = sv[i];
    G[(int64_t)(hb + 1 + i) * Q + q] = av[i] + tau[i] * bv[i];
#pragma unroll
    for (int j = 0; j < i; ++j)
      G[(int64_t)pk(i + 1, j + 1) * Q + q] = (tau[i] * sv[i] + tau[j] * sv[j]) / (tau[i] + tau[j]);
  }
}

// ------------------------------------------------------------------ residual pass
// Reads the weights x (FP64) of candidate q, writes rt[0] = ||b - A x||^2 and
// rt[1 + j] = (A^T (b - A x))_j, j = 0..N.
template <int N>
__device__ __forceinline__ void refine_unit(const EvalArgs& a, const Unit& u) {
  const Lane ln = lane_of(a, u, true);
  const int q = ln.act ? ln.q : u.q0;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  const double* X = a.sc.x;
  const int64_t kbeg = u.k0 + ln.slice;
  const int64_t kend = ln.act ? u.k1 : kbeg;
  const int64_t step = ln.ks;
  double tau[N], w[N], t[N];
  const double w0 = ln.act ? X[q] : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    tau[i] = ln.act ? exp10(th[i]) : 0.0;
    w[i] = ln.act ? X[(int64_t)(i + 1) * Q + q] : 0.0;
    t[i] = 0.0;
  }
  double t0 = 0.0, rr = 0.0;
#pragma unroll 1
  for (int64_t k = kbeg; k < kend; k += step) {
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
  rr = group_sum(rr, ln.ks);
  t0 = group_sum(t0, ln.ks);
#pragma unroll
  for (int i = 0; i < N; ++i) t[i] = group_sum(t[i], ln.ks);
  if (ln.act && ln.slice == 0) {
    double* R = a.sc.rt;
    R[q] = rr;
    R[Q + q] = t0;
#pragma unroll
    for (int i = 0; i < N; ++i) R[(int64_t)(i + 2) * Q + q] = t[i];
  }

}

// ------------------------------------------------------------------ sample staging (bulk copies)
// The column-sum pass reads, for every sample of a unit's spectrum, the two float4
// records {(omega 2^-30)^2, eps', omega eps''} (high and low float-float parts);
// every lane of the block reads the same samples. They are staged in shared memory
// in chunks of STAGE_SAMPLES by the Tensor Memory Accelerator (cp.async.bulk, a
// plain global -> shared copy completing on an mbarrier), double-buffered: thread 0
// issues chunk c + 1 while the block computes on chunk c. Every record is 16 bytes
// and 16-byte aligned, as the bulk copy requires.
//
// Every wait on an mbarrier is bounded (STAGE_WAIT_CYCLES of clock64): a wait that
// runs out records DEBYE_ETIMEOUT, the block agrees on it (__syncthreads_or), waits
// again, bounded, for its own copies still in flight, and leaves the kernel.
constexpr int STAGE_SAMPLES = 256;
constexpr long long STAGE_WAIT_CYCLES = 1ll << 31;   // about 1 s at the maximum SM clock

struct Stage {
  float4* hi;        // [2][STAGE_SAMPLES]
  float4* lo;        // [2][STAGE_SAMPLES]
  uint64_t* bar;     // [2] one mbarrier per buffer
  uint32_t fills0, fills1;     // completed phases of each buffer (the same in every thread)
  bool pending0, pending1;     // a copy into the buffer has been issued and not yet waited for
  __device__ __forceinline__ uint32_t& fills(int b) { return b ? fills1 : fills0; }
  __device__ __forceinline__ bool& pending(int b) { return b ? pending1 : pending0; }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void stage_init(Stage& st, float4* buf, uint64_t* bar) {
  st.hi = buf;
  st.lo = buf + 2 * STAGE_SAMPLES;
  st.bar = bar;
  st.fills0 = st.fills1 = 0;
  st.pending0 = st.pending1 = false;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar + b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Thread 0: copy samples k .. k + n - 1 of both record arrays into buffer b.
__device__ __forceinline__ void stage_issue(const EvalArgs& a, Stage& st, int b, int64_t k, int n) {
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)n * (uint32_t)sizeof(float4);
    const uint32_t bar = smem_addr(st.bar + b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier generic reads of the buffer
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2u * bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(st.hi + b * STAGE_SAMPLES)), "l"(a.kq32 + k), "r"(bytes), "r"(bar) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(st.lo + b * STAGE_SAMPLES)), "l"(a.kqff + k), "r"(bytes), "r"(bar) : "memory");
  }
  st.pending(b) = true;
}

// Wait (bounded) until buffer b's current phase has completed.
__device__ __forceinline__ bool stage_wait_one(Stage& st, int b) {
  const uint32_t bar = smem_addr(st.bar + b), parity = st.fills(b) & 1u;
  const long long t0 = clock64();
  uint32_t done = 0;
  while (true) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done || clock64() - t0 > STAGE_WAIT_CYCLES) break;
  }
  if (done) {
    st.fills(b) += 1;
    st.pending(b) = false;
  }
  return done != 0;
}

// Buffer b ready in every thread; false (the block agreeing) if a wait ran out.
__device__ __forceinline__ bool stage_wait(const EvalArgs& a, Stage& st, int b) {
  const bool ok = stage_wait_one(st, b);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) set_status(a.status, DEBYE_ETIMEOUT);
    for (int c = 0; c < 2; ++c)
      if (st.pending(c)) stage_wait_one(st, c);   // the block's own copies in flight
    return false;
  }
  return true;
}

// ------------------------------------------------------------------ column-sum pass (mixed)
// For the mixed evaluation from column sums (k_solve_sums): per candidate, in
// float-float,
//   S_i = sum_k re_i(k)                      (the pole block of the Gram follows from these)
//   h_i = sum_k re_i(k) eps'_k + im_i(k) eps''_k   (A^T b without the eps_inf row)
// and, with the gradient (GRAD), the same sums over the derivative columns
// d/d theta_i (theta = log10 tau):
//   D_i = sum_k d re_i(k),   E_i = sum_k d re_i(k) eps'_k + d im_i(k) eps''_k.
// The basis needs only x^2 = omega^2 tau^2: one float-float product of the
// per-sample omega^2 and the per-candidate tau^2 (scaled by 2^-60 and 2^60,
// exactly, to keep both far from the float range limits); 1 + x^2 by Fast2Sum on
// (max, min); re = 1/(1 + x^2) by the approximate reciprocal and one Newton step.
// With im = x re = omega tau re,
//   h_i = sum_k re_i(k) eps'_k + tau_i B_i,   B_i = sum_k re_i(k) (omega_k eps''_k),
// two Dot2 sums on the per-sample eps' and omega eps'' (k_prep_samples stores
// {omega^2, eps', omega eps''} in a.kq32 / a.kqff). With u = x^2 re^2 = re (1 - re),
// d re / d theta = -2 ln10 u and d im / d theta = ln10 x re^2 (1 - x^2)
// = ln10 omega tau (re - 2u), so
//   D_i = -2 ln10 U_i,   E_i = ln10 (-2 V_i + tau_i (B_i - 2 W_i)),
//   U = sum u,  V = sum u eps',  W = sum u (omega eps'').
// The same-sign sums S (re <= 1) and U (u <= 1/4) start from a bias of 1 so that
// Fast2Sum is exact; the bias is removed at the end. Writes tau_i = 10^theta_i to
// sc.x[i Q + q] (the FP64 power is done once per candidate here rather than again
// in the solve), sc.G[i Q + q] = S_i, sc.G[(N + i) Q + q] = h_i, and with GRAD
// sc.G[(2N + i) Q + q] = D_i, sc.G[(3N + i) Q + q] = E_i.
//
// One sweep over the samples for poles P0 .. P0 + C - 1 of an N-pole candidate:
template <int N, int P0, int C, bool GRAD>
__device__ __forceinline__ bool sums_sq_sweep(const EvalArgs& a, const Unit& u, const Lane& ln, int q, Stage& st) {
  const double* th = a.theta + (int64_t)q * a.sc.nmax + P0;
  const int64_t Q = a.sc.Q;
  constexpr int CG = GRAD ? C : 1;
  float t2h[C], t2l[C], sh[C], sl[C], ah[C], al[C], ch[C], cl[C];
  float uh[CG], ul[CG], vh_[CG], vl_[CG], wh[CG], wl[CG];
#pragma unroll
  for (int i = 0; i < C; ++i) {
    t2h[i] = t2l[i] = 0.f;
    if (ln.act) {
      const double t = exp10(th[i]);
      const double ts = t * 0x1p30;
      split_double(ts * ts, t2h[i], t2l[i]);
      if (ln.slice == 0) a.sc.x[(int64_t)(P0 + i) * Q + q] = t;   // tau for k_solve_sums and the epilogue
    }
    sh[i] = 1.f;
    sl[i] = ah[i] = al[i] = ch[i] = cl[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < CG; ++i) {
    uh[i] = 1.f;
    ul[i] = vh_[i] = vl_[i] = wh[i] = wl[i] = 0.f;
  }
  const int64_t nk = u.k1 - u.k0;
  const int nch = (int)((nk + STAGE_SAMPLES - 1) / STAGE_SAMPLES);
  auto chunk_len = [&](int64_t c0) { return (int)(nk - c0 < STAGE_SAMPLES ? nk - c0 : STAGE_SAMPLES); };
  if (nch > 0) stage_issue(a, st, 0, u.k0, chunk_len(0));
#pragma unroll 1
  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    const int64_t c0 = (int64_t)c * STAGE_SAMPLES;
    if (c + 1 < nch)   // buffer b ^ 1 was released by the barrier that ended chunk c - 1
      stage_issue(a, st, b ^ 1, u.k0 + c0 + STAGE_SAMPLES, chunk_len(c0 + STAGE_SAMPLES));
    if (!stage_wait(a, st, b)) return false;
    const int cnt = chunk_len(c0);
    const float4* bh = st.hi + b * STAGE_SAMPLES;
    const float4* bl = st.lo + b * STAGE_SAMPLES;
    const int jend = ln.act ? cnt : 0;
    float4 vhn = bh[ln.slice < jend ? ln.slice : 0], vln = bl[ln.slice < jend ? ln.slice : 0];
#pragma unroll 1
  for (int j = ln.slice; j < jend; j += ln.ks) {
    const float4 vh = vhn, vl = vln;
    if (j + ln.ks < jend) {   // next sample's records in flight during this one
      vhn = bh[j + ln.ks];
      vln = bl[j + ln.ks];
    }
#pragma unroll
    for (int i = 0; i < C; ++i) {
      // x^2 in float-float (the product of the low parts, ~2^-48, is dropped)
      const float x2h = __fmul_rn(vh.x, t2h[i]);
      float x2l = __fmaf_rn(vh.x, t2h[i], -x2h);
      x2l = __fmaf_rn(vh.x, t2l[i], __fmaf_rn(vl.x, t2h[i], x2l));
      // d = 1 + x^2: Fast2Sum of (max, min), exact
      const float big = fmaxf(1.f, x2h), small = fminf(1.f, x2h);
      const float dh = __fadd_rn(big, small);
      const float dl = __fadd_rn(__fsub_rn(small, __fsub_rn(dh, big)), x2l);
      // re = 1/d: approximate reciprocal and one Newton step on the float-float d
      const float r0 = rcp_approx(dh);
      float e = __fmaf_rn(-dh, r0, 1.0f);
      e = __fmaf_rn(-dl, r0, e);
      const float rl = __fmul_rn(r0, e);
      const float gs = __fadd_rn(sh[i], r0);                         // Fast2Sum, sh >= 1 >= re
      sl[i] = __fadd_rn(sl[i], __fadd_rn(__fsub_rn(r0, __fsub_rn(gs, sh[i])), rl));
      sh[i] = gs;
      ff_add_prod(ah[i], al[i], r0, rl, vh.y, vl.y);                 // re eps'
      ff_add_prod(ch[i], cl[i], r0, rl, vh.z, vl.z);                 // re omega eps''
      if constexpr (GRAD) {
        float r2h, r2l, qh, ql;
        ff_mul(r0, rl, r0, rl, r2h, r2l);                            // re^2
        ff_mul(x2h, x2l, r2h, r2l, qh, ql);                          // u = x^2 re^2
        const float gu = __fadd_rn(uh[i], qh);                       // Fast2Sum, uh >= 1 >= u
        ul[i] = __fadd_rn(ul[i], __fadd_rn(__fsub_rn(qh, __fsub_rn(gu, uh[i])), ql));
        uh[i] = gu;
        ff_add_prod(vh_[i], vl_[i], qh, ql, vh.y, vl.y);             // u eps'
        ff_add_prod(wh[i], wl[i], qh, ql, vh.z, vl.z);               // u omega eps''
      }
    }
  }
    __syncthreads();   // the whole block is done with buffer b
  }
#pragma unroll
  for (int i = 0; i < C; ++i) {
    group_sum_ff(sh[i], sl[i], ln.ks);
    group_sum_ff(ah[i], al[i], ln.ks);
    group_sum_ff(ch[i], cl[i], ln.ks);
  }
#pragma unroll
  for (int i = 0; i < CG; ++i) {
    if constexpr (GRAD) {
      group_sum_ff(uh[i], ul[i], ln.ks);
      group_sum_ff(vh_[i], vl_[i], ln.ks);
      group_sum_ff(wh[i], wl[i], ln.ks);
    }
  }
  if (ln.act && ln.slice == 0) {
    double* G = a.sc.G;
    constexpr double LN10 = 2.302585092994046;
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const int64_t j = P0 + i;
      const double t = a.sc.x[j * Q + q];
      const double B = (double)ch[i] + (double)cl[i];
      G[j * Q + q] = ((double)sh[i] - (double)ln.ks) + (double)sl[i];
      G[(N + j) * Q + q] = ((double)ah[i] + (double)al[i]) + t * B;
      if constexpr (GRAD) {
        const double U = ((double)uh[i] - (double)ln.ks) + (double)ul[i];
        const double V = (double)vh_[i] + (double)vl_[i];
        const double W = (double)wh[i] + (double)wl[i];
        G[(2 * N + j) * Q + q] = -2.0 * LN10 * U;
        G[(3 * N + j) * Q + q] = LN10 * (-2.0 * V + t * (B - 2.0 * W));
      }
    }
  }
  return true;
}

// With GRAD, more than SQUARED_CHUNK_GRAD poles take two sweeps of about N/2 poles
// each (14 registers per pole); the cost-only sums (8 per pole) sweep once. A unit
// without any active candidate (a masked evaluation) is skipped by the whole block.
// Returns false if a wait for staged samples ran out (the block then stops).
template <int N, bool GRAD>
__device__ __forceinline__ bool sums_sq_unit(const EvalArgs& a, const Unit& u, Stage& st) {
  const Lane ln = lane_of(a, u, false);
  if (!__syncthreads_or(ln.act)) return true;
  const int q = ln.act ? ln.q : u.q0;
  if constexpr (!GRAD || N <= SQUARED_CHUNK_GRAD) {
    return sums_sq_sweep<N, 0, N, GRAD>(a, u, ln, q, st);
  } else {
    constexpr int C1 = (N + 1) / 2;
    if (!sums_sq_sweep<N, 0, C1, GRAD>(a, u, ln, q, st)) return false;
    return sums_sq_sweep<N, C1, N - C1, GRAD>(a, u, ln, q, st);
  }
}

// ------------------------------------------------------------------ gradient pass
// With x1 (unflipped, sc.x), x_hat (flipped, sc.xh) and w = M^-1 S g_hat (sc.w):
//   gt[i]        = a_i'^T r_hat,  r_hat = b - A x_hat
//   gt[N + i]    = a_i^T a_i'
//   gt[2N + i]   = a_i'^T r,      r = b - A x1
//   gt[3N + i]   = a_i'^T (A w)
// where a_i' = d a_i / d log10(tau_i).
template <int N>
__device__ __forceinline__ void grad_unit(const EvalArgs& a, const Unit& u) {
  const Lane ln = lane_of(a, u, true);
  const int q = ln.act ? ln.q : u.q0;
  const double* th = a.theta + (int64_t)q * a.sc.nmax;
  const int64_t Q = a.sc.Q;
  const int64_t kbeg = u.k0 + ln.slice;
  const int64_t kend = ln.act ? u.k1 : kbeg;
  const int64_t step = ln.ks;
  constexpr double LN10 = 2.302585092994046;
  auto ld = [&](const double* p) { return ln.act ? *p : 0.0; };
  double tau[N], xh[N], e[N], w[N];
  double t_rh[N], t_aa[N], t_r[N], t_aw[N];
  const double x0 = ld(a.sc.xh + q);
  const double e0 = x0 - ld(a.sc.x + q);
  const double w0 = ld(a.sc.w + q);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    tau[i] = ln.act ? exp10(th[i]) : 0.0;
    xh[i] = ld(a.sc.xh + (int64_t)(i + 1) * Q + q);
    e[i] = xh[i] - ld(a.sc.x + (int64_t)(i + 1) * Q + q);
    w[i] = ld(a.sc.w + (int64_t)(i + 1) * Q + q);
    t_rh[i] = t_aa[i] = t_r[i] = t_aw[i] = 0.0;
  }
#pragma unroll 1
  for (int64_t k = kbeg; k < kend; k += step) {
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
#pragma unroll
  for (int i = 0; i < N; ++i) {
    t_rh[i] = group_sum(t_rh[i], ln.ks);
    t_aa[i] = group_sum(t_aa[i], ln.ks);
    t_r[i] = group_sum(t_r[i], ln.ks);
    t_aw[i] = group_sum(t_aw[i], ln.ks);
  }
  if (ln.act && ln.slice == 0) {
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
template <int PH, int N>
__device__ __forceinline__ void run_phase(const EvalArgs& a, const Unit& u) {
  if constexpr (PH == PH_GRAM) gram_unit<N>(a, u);
  else if constexpr (PH == PH_GRAM_SUMS) gram_sums_unit<N>(a, u);
  else if constexpr (PH == PH_REFINE) refine_unit<N>(a, u);
  else grad_unit<N>(a, u);
}

template <int PH, int LO, int HI>
__device__ __forceinline__ void dispatch_n(const EvalArgs& a, const Unit& u) {
  if constexpr (LO <= HI) {
    if (u.N == LO) run_phase<PH, LO>(a, u);
    else dispatch_n<PH, LO + 1, HI>(a, u);
  }
}

// One block per unit (grid-stride over the unit list); LO..HI is the range of
// pole counts compiled into this kernel (the library launches one N per kernel). At most MAXT threads per block; MINB
// resident blocks of that size bound the registers per thread (128 x 3: 168
// registers, 12 warps per SM with 64-thread blocks).
// The column-sum pass (PH_SUMS, PH_SUMSG) of pole count N: one block per unit
// (grid-stride over the unit list), the unit's samples staged by bulk copies.
template <int N, bool GRAD, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_pass_sums(EvalArgs a) {
  __shared__ __align__(128) float4 stage_buf[4 * STAGE_SAMPLES];
  __shared__ __align__(8) uint64_t stage_bar[2];
  Stage st;
  stage_init(st, stage_buf, stage_bar);
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    if (u.N != N) {
      if (threadIdx.x == 0) set_status(a.status, DEBYE_EBOUNDS);
      continue;
    }
    if (!sums_sq_unit<N, GRAD>(a, u, st)) return;
  }
}

template <int PH, int LO, int HI, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_pass(EvalArgs a) {
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    if (u.N < LO || u.N > HI) {
      if (threadIdx.x == 0) set_status(a.status, DEBYE_EBOUNDS);
      continue;
    }
    dispatch_n<PH, LO, HI>(a, u);
  }
}

}  // namespace debyefit
