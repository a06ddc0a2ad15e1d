// N-generic kernels of libdebyefit: input preparation, the FP64 damped solve,
// refinement/finish with the sign flip, gradient assembly, the particle swarm
// and target synthesis.
#include <cmath>

#include "launch.h"
#include "solve.cuh"
#include "solve_sums.cuh"

namespace debyefit {

// ------------------------------------------------------------------ input preparation
// Per sample: float-float split of omega, eps', eps'' for the mixed passes (the
// first n records of kf32 / kff) and of (omega 2^-30)^2, eps', omega eps'' for the
// squared-form column sums (records n .. 2n - 1), and finiteness checks; per
// spectrum: h0 = sum_k eps'_k and b^T b (FP64).
__global__ void k_prep_samples(int64_t n, const double* __restrict__ omega,
                               const double* __restrict__ er, const double* __restrict__ ei,
                               float4* __restrict__ kf32, float4* __restrict__ kff, int* status) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double w = omega[k], a = er[k], b = ei[k];
    if (!(w > 0.0) || !isfinite(w) || !isfinite(a) || !isfinite(b)) set_status(status, DEBYE_ENOTFINITE);
    float wh, wl, ah, al, bh, bl, w2h, w2l, ch, cl;
    split_double(w, wh, wl);
    split_double(a, ah, al);
    split_double(b, bh, bl);
    kf32[k] = make_float4(wh, ah, bh, 0.f);
    kff[k] = make_float4(wl, al, bl, 0.f);
    const double ws = w * 0x1p-30;
    split_double(ws * ws, w2h, w2l);
    split_double(w * b, ch, cl);
    kf32[n + k] = make_float4(w2h, ah, ch, 0.f);
    kff[n + k] = make_float4(w2l, al, cl, 0.f);
  }
}

__global__ void k_prep_spectra(int64_t S, const int64_t* __restrict__ offsets,
                               const double* __restrict__ er, const double* __restrict__ ei,
                               const double* __restrict__ lo, const double* __restrict__ hi,
                               double* __restrict__ h0, double* __restrict__ bb, int* status) {
  __shared__ double red[32], red2[32];
  for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
    const int64_t a = offsets[s], b = offsets[s + 1];
    double acc = 0.0, acc2 = 0.0;
    for (int64_t k = a + threadIdx.x; k < b; k += blockDim.x) {
      acc += er[k];
      acc2 = fma(er[k], er[k], fma(ei[k], ei[k], acc2));
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(0xffffffffu, acc, o);
      acc2 += __shfl_down_sync(0xffffffffu, acc2, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = acc;
      red2[threadIdx.x >> 5] = acc2;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
      acc2 = (threadIdx.x < (blockDim.x >> 5)) ? red2[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        acc2 += __shfl_down_sync(0xffffffffu, acc2, o);
      }
      if (threadIdx.x == 0) {
        h0[s] = acc;
        bb[s] = acc2;
        if (!(lo[s] < hi[s]) || !isfinite(lo[s]) || !isfinite(hi[s])) set_status(status, DEBYE_EBOUNDS);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ damped solve
// Scaling helpers of the factor type T: in FP64 a division by d = 1/dinv (as the
// plain method reads); in FP32 a multiplication by dinv.
template <typename T>
struct Scale {
  T dinv[NMAX1];   // 1 / sqrt(G_ii)
  double d[NMAX1]; // sqrt(G_ii)
  __device__ __forceinline__ void load(const Scratch& sc, int64_t q, int n) {
    for (int i = 0; i < n; ++i) {
      dinv[i] = (T)sc.dinv[(int64_t)i * sc.Q + q];
      if constexpr (sizeof(T) == 8) d[i] = 1.0 / sc.dinv[(int64_t)i * sc.Q + q];
      else d[i] = (double)(1.0f / dinv[i]);
    }
  }
  // D^-1 v for an FP64 vector entry, as T
  __device__ __forceinline__ T down(double v, int i) const {
    if constexpr (sizeof(T) == 8) return v / d[i];
    else return (float)v * dinv[i];
  }
  // D^-1 v for a T entry, as FP64
  __device__ __forceinline__ double up(T v, int i) const {
    if constexpr (sizeof(T) == 8) return v / d[i];
    else return (double)(v * dinv[i]);
  }
};

// x0 = M^-1 h per candidate; stores L (type T), D^-1, x0 and the failure flag.
template <typename T>
__global__ void __launch_bounds__(256) k_solve(EvalArgs a) {
  const int64_t Q = a.sc.Q;
  const int hb = (a.sc.nmax + 1) * (a.sc.nmax + 2) / 2;
  T* Lg = factor_base_w<T>(a.sc);
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int q = u.q0 + (int)threadIdx.x;
    if (q >= u.q1 || (a.active && !a.active[q])) continue;
    const int n = u.N + 1;
    T L[NPACK_MAX], dinv[NMAX1], z[NMAX1];
    for (int i = 0; i < n; ++i) dinv[i] = T(1) / sqrt_t((T)a.sc.G[(int64_t)pk(i, i) * Q + q]);
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < i; ++j) L[pk(i, j)] = (T)a.sc.G[(int64_t)pk(i, j) * Q + q] * dinv[i] * dinv[j];
      L[pk(i, i)] = (T)(1.0 + a.lam);
    }
    bool ok = cholesky_packed(L, n);
    double x0[NMAX1];
    if (ok) {
      for (int i = 0; i < n; ++i) z[i] = (T)a.sc.G[(int64_t)(hb + i) * Q + q] * dinv[i];
      llt_solve(L, z, n);
      for (int i = 0; i < n; ++i) {
        x0[i] = (double)(z[i] * dinv[i]);
        ok = ok && isfinite(x0[i]);
      }
    }
    record_fail(a, q, u.s, ok);
    if (!ok) continue;
    const int npk = n * (n + 1) / 2;
    for (int e = 0; e < npk; ++e) Lg[(int64_t)e * Q + q] = L[e];
    for (int i = 0; i < n; ++i) {
      a.sc.dinv[(int64_t)i * Q + q] = (double)dinv[i];
      a.sc.x[(int64_t)i * Q + q] = x0[i];
    }
  }
}

// ------------------------------------------------------------------ refinement / finish
// From the residual pass at x (rt: rr = ||b - A x||^2, t = A^T (b - A x)):
//   g  = t - lam diag(G) x          (minus half the cost gradient in x)
//   dx = M^-1 g,  x1 = x + dx       (one step of iterative refinement)
// final == 0: store x1 and return.
// final == 1: cost(x1) by the exact quadratic identity
//   cost(y) = cost(x) - 2 (y - x)^T g + (y - x)^T M (y - x),  cost(x) = rr + lam sum G_ii x_i^2,
// then the sign flip x_hat = x1 + e (e_i = -2 x1_i where d_eps_i < 0, Sec. III-B) and
//   cost(x_hat) = cost(x1) - 2 e^T g1 + e^T M e,  g1 = g - M dx.
// Outputs cost[q], weights[q][nmax+1] (optional); keeps x1, x_hat and g1 for the gradient.
// Sums of the cost identity are FP64; products with the factor are in its type T.
template <typename T>
__global__ void __launch_bounds__(256) k_finish(EvalArgs a, int final_step, double* cost,
                                                double* weights, double* g1_out) {
  const int64_t Q = a.sc.Q;
  const int nm1 = a.sc.nmax + 1;
  const T* Lg = factor_base<T>(a.sc);
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int q = u.q0 + (int)threadIdx.x;
    if (q >= u.q1 || (a.active && !a.active[q])) continue;
    const int n = u.N + 1;
    if (a.sc.fail[q]) {
      if (final_step) {
        if (cost) cost[q] = INFINITY;
        if (weights)
          for (int j = 0; j < nm1; ++j) weights[(int64_t)q * nm1 + j] = 0.0;
      }
      continue;
    }
    T L[NPACK_MAX], v[NMAX1], w1[NMAX1], tmp[NMAX1];
    double x[NMAX1], g[NMAX1], dx[NMAX1];
    Scale<T> sc;
    sc.load(a.sc, q, n);
    const int npk = n * (n + 1) / 2;
    for (int e = 0; e < npk; ++e) L[e] = Lg[(int64_t)e * Q + q];
    double cost0 = a.sc.rt[q];
    for (int i = 0; i < n; ++i) {
      const double gii = a.sc.G[(int64_t)pk(i, i) * Q + q];
      x[i] = a.sc.x[(int64_t)i * Q + q];
      g[i] = a.sc.rt[(int64_t)(i + 1) * Q + q] - a.lam * gii * x[i];
      cost0 += a.lam * gii * x[i] * x[i];
      v[i] = sc.down(g[i], i);
    }
    llt_solve(L, v, n);            // v = D dx
    for (int i = 0; i < n; ++i) dx[i] = sc.up(v[i], i);
    if (!final_step) {
      for (int i = 0; i < n; ++i) a.sc.x[(int64_t)i * Q + q] = x[i] + dx[i];
      continue;
    }
    lt_mul(L, v, w1, n);           // w1 = L^T D dx
    double dg = 0.0, dmd = 0.0;
    for (int i = 0; i < n; ++i) {
      dg += dx[i] * g[i];
      dmd += (double)w1[i] * (double)w1[i];
    }
    double c = cost0 - 2.0 * dg + dmd;
    // The step must not raise the damped cost, whose value at x is exact: if the
    // identity leaves [0, cost(x)] the refinement is discarded (dx = 0).
    if (!(c >= 0.0 && c <= cost0)) {
      c = cost0;
      for (int i = 0; i < n; ++i) {
        dx[i] = 0.0;
        w1[i] = T(0);
      }
    }
    l_mul(L, w1, tmp, n);          // tmp = L L^T D dx; M dx = D tmp
    bool flipped = false;
    double e[NMAX1];
    for (int i = 0; i < n; ++i) {
      const double x1 = x[i] + dx[i];
      x[i] = x1;
      g[i] -= sc.d[i] * (double)tmp[i];   // g1
      e[i] = (i > 0 && x1 < 0.0) ? -2.0 * x1 : 0.0;
      flipped |= (e[i] != 0.0);
    }
    if (flipped) {
      for (int i = 0; i < n; ++i) tmp[i] = (T)(sc.d[i] * e[i]);
      lt_mul(L, tmp, w1, n);
      double eg = 0.0, eme = 0.0;
      for (int i = 0; i < n; ++i) {
        eg += e[i] * g[i];
        eme += (double)w1[i] * (double)w1[i];
      }
      c = c - 2.0 * eg + eme;
    }
    if (!isfinite(c)) c = INFINITY;
    if (cost) cost[q] = c;
    for (int i = 0; i < n; ++i) {
      a.sc.x[(int64_t)i * Q + q] = x[i];
      a.sc.xh[(int64_t)i * Q + q] = x[i] + e[i];
      if (g1_out) g1_out[(int64_t)i * Q + q] = g[i];
    }
    if (weights) {
      for (int j = 0; j < nm1; ++j) weights[(int64_t)q * nm1 + j] = (j < n) ? x[j] + e[j] : 0.0;
    }
  }
}

// ------------------------------------------------------------------ cost from column sums, a warp per candidate
// The algebra of k_solve_sums with lane r holding row r of the (N+1)-square
// systems, so that its O(N^2) loops run across the lanes: M one row per lane,
// the factorisation one column per step (rows in parallel), the triangular
// solves one unknown per step (broadcast by shuffle), the products with M one
// row per lane and the gradient one pole per lane. It serves evaluations too
// small to fill the GPU with one thread per candidate (the polish's line-search
// and accepted points), where k_solve_sums takes the latency of one candidate's
// serial solve. Each warp keeps M (float-float) and the FP32 factor, both
// [n1][n1] with n1 = nmax + 1, and the vectors its lanes exchange in shared memory.
constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int WARP_SOLVE_MAX_WARPS = 8;     // candidates in flight per block
constexpr int WARP_SOLVE_MAX_Q_PER_SM = 256; // auto choice: at most this many candidates per SM

struct WarpSolveMem {
  ff* M;        // [n1][n1] M = G + lam diag G
  ff* tau;      // [n1] row r >= 1: tau of pole r - 1
  ff* S;        // [n1] row r >= 1: column sum S of pole r - 1
  ff* v;        // [n1] vector multiplied by M
  ff* xh;       // [n1] flipped weights x_hat
  ff* w;        // [n1] adjoint
  float* L;     // [n1][n1] FP32 factor of the scaled M, 1 / L_jj on the diagonal
  float* dinv;  // [n1] diag(G)^-1/2
  float* sgn;   // [n1] signs of the flip
};

__host__ __device__ inline size_t warp_solve_bytes(int n1) {
  const size_t b = (size_t)n1 * n1 * (sizeof(ff) + sizeof(float)) + (size_t)n1 * (5 * sizeof(ff) + 2 * sizeof(float));
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ WarpSolveMem warp_solve_mem(unsigned char* base, int n1) {
  WarpSolveMem m;
  ff* f = reinterpret_cast<ff*>(base);
  m.M = f;
  f += n1 * n1;
  m.tau = f;
  m.S = f + n1;
  m.v = f + 2 * n1;
  m.xh = f + 3 * n1;
  m.w = f + 4 * n1;
  float* g = reinterpret_cast<float*>(f + 5 * n1);
  m.L = g;
  m.dinv = g + n1 * n1;
  m.sgn = g + n1 * n1 + n1;
  return m;
}

// (M v)_r of the lane's row (zero for lanes r >= n)
__device__ __forceinline__ ff warp_mrow(const WarpSolveMem& m, int n1, int n, int r, const ff* v) {
  ff acc{0.f, 0.f};
  if (r < n)
    for (int j = 0; j < n; ++j) acc = ff_sum(acc, ff_prod(m.M[r * n1 + j], v[j]));
  return acc;
}

// L L^T = D^-1 M D^-1 in FP32 (the same operations as cholesky_rdiag): step j
// finishes column j, every row below it in its own lane.
__device__ __forceinline__ bool warp_cholesky(const WarpSolveMem& m, int n1, int n, int r) {
  for (int j = 0; j < n; ++j) {
    __syncwarp();
    float s = 0.f;
    if (r == j) {
      s = m.L[j * n1 + j];
      for (int k = 0; k < j; ++k) s = __fmaf_rn(-m.L[j * n1 + k], m.L[j * n1 + k], s);
    }
    s = __shfl_sync(FULL_MASK, s, j);
    if (!(s > 0.f) || !isfinite(s)) return false;
    const float inv = __frsqrt_rn(s);
    if (r == j) m.L[j * n1 + j] = inv;
    if (r > j && r < n) {
      float v = m.L[r * n1 + j];
      for (int k = 0; k < j; ++k) v = __fmaf_rn(-m.L[r * n1 + k], m.L[j * n1 + k], v);
      m.L[r * n1 + j] = __fmul_rn(v, inv);
    }
  }
  __syncwarp();
  return true;
}

// (L L^T)^-1 b, lane r holding b_r and receiving the solution's entry r:
// forward then backward substitution, one unknown per step.
__device__ __forceinline__ float warp_llt(const WarpSolveMem& m, int n1, int n, int r, float b) {
  const float dg = r < n ? m.L[r * n1 + r] : 0.f;
  float acc = b, y = 0.f;
  for (int j = 0; j < n; ++j) {
    const float yj = __shfl_sync(FULL_MASK, __fmul_rn(acc, dg), j);
    if (r == j) y = yj;
    if (r > j && r < n) acc = __fmaf_rn(-m.L[r * n1 + j], yj, acc);
  }
  acc = y;
  float x = 0.f;
  for (int j = n - 1; j >= 0; --j) {
    const float xj = __shfl_sync(FULL_MASK, __fmul_rn(acc, dg), j);
    if (r == j) x = xj;
    if (r < j) acc = __fmaf_rn(-m.L[j * n1 + r], xj, acc);
  }
  return x;
}

// M^-1 rhs (lane r: rhs_r in, x_r out) through the FP32 factor, refined `steps`
// times against the float-float M. Uses m.v.
__device__ __forceinline__ bool warp_refined_solve(const WarpSolveMem& m, int n1, int n, int r, ff rhs, ff& x,
                                                   int steps) {
  const float di = r < n ? m.dinv[r] : 0.f;
  x = ff{0.f, 0.f};
  bool ok = true;
  for (int it = 0; it <= steps && ok; ++it) {
    ff res = rhs;
    if (it > 0) {
      __syncwarp();
      if (r < n) m.v[r] = x;
      __syncwarp();
      res = ff_sum(rhs, ff_neg(warp_mrow(m, n1, n, r, m.v)));
    }
    const float dx = warp_llt(m, n1, n, r, __fmul_rn(res.h, di));
    x = ff_sum(x, ff{__fmul_rn(dx, di), 0.f});
    ok = __all_sync(FULL_MASK, r >= n || isfinite(x.h));
  }
  return ok;
}

__global__ void __launch_bounds__(WARP_SOLVE_MAX_WARPS * 32) k_solve_sums_warp(EvalArgs a, double* cost,
                                                                               double* weights, double* grad) {
  extern __shared__ __align__(16) unsigned char warp_solve_smem[];
  const int64_t Q = a.sc.Q;
  const int nmax = a.sc.nmax, nm1 = nmax + 1, n1 = nm1;
  const int r = (int)threadIdx.x & 31, wid = (int)threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
  const WarpSolveMem m = warp_solve_mem(warp_solve_smem + (size_t)wid * warp_solve_bytes(n1), n1);
  const ff one_lam = ff_of(1.0 + a.lam);
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int N = u.N, n = N + 1;
    const ff kk = ff_of((double)(u.k1 - u.k0));
    for (int q = u.q0 + wid; q < u.q1; q += nw) {   // warp-uniform from here on
      if (a.active && !a.active[q]) continue;
      // row r >= 1 is pole r - 1: tau (from the column-sum pass), S and h
      ff hv{0.f, 0.f}, gd{0.f, 0.f};
      __syncwarp();
      if (r == 0) {
        hv = ff_of(a.h0[u.s]);
        gd = kk;
      } else if (r < n) {
        m.tau[r] = ff_of(a.sc.x[(int64_t)(r - 1) * Q + q]);
        gd = ff_of(a.sc.G[(int64_t)(r - 1) * Q + q]);
        m.S[r] = gd;
        hv = ff_of(a.sc.G[(int64_t)(N + r - 1) * Q + q]);
      }
      if (r < n) m.dinv[r] = __frsqrt_rn(gd.h);
      __syncwarp();
      // row r of M and of the scaled FP32 matrix (unit diagonal + lam)
      if (r < n) {
        const float dr = m.dinv[r];
        for (int j = 0; j < n; ++j) {
          ff g;
          if (j == r) g = gd;
          else if (r == 0) g = m.S[j];
          else if (j == 0) g = gd;
          else
            g = ff_quot(ff_sum(ff_prod(m.tau[r], m.S[r]), ff_prod(m.tau[j], m.S[j])), ff_sum(m.tau[r], m.tau[j]));
          m.M[r * n1 + j] = (j == r) ? ff_prod(g, one_lam) : g;
          if (j < r) m.L[r * n1 + j] = __fmul_rn(__fmul_rn(g.h, dr), m.dinv[j]);
        }
        m.L[r * n1 + r] = (float)(1.0 + a.lam);
      }
      bool ok = warp_cholesky(m, n1, n, r);
      ff x{0.f, 0.f};
      if (ok) ok = warp_refined_solve(m, n1, n, r, hv, x, grad ? SUMS_REFINE : SUMS_REFINE_COST);
      if (r == 0) record_fail(a, q, u.s, ok);
      if (!ok) {
        if (cost && r == 0) cost[q] = INFINITY;
        if (weights && r < nm1) weights[(int64_t)q * nm1 + r] = 0.0;
        if (grad && r < nmax) grad[(int64_t)q * nmax + r] = 0.0;
        continue;
      }
      // sign flip of negative d_eps (Sec. III-B), then the exact quadratic cost
      const float sg = (r > 0 && r < n && x.h < 0.f) ? -1.f : 1.f;
      if (sg < 0.f) x = ff_neg(x);
      __syncwarp();
      if (r < n) {
        m.v[r] = x;
        m.xh[r] = x;
        m.sgn[r] = sg;
      }
      __syncwarp();
      const ff mx = warp_mrow(m, n1, n, r, m.v);   // (M x_hat)_r
      ff t{0.f, 0.f};
      if (r < n) {
        t = ff_neg(ff_prod(ff{__fmul_rn(2.f, x.h), __fmul_rn(2.f, x.l)}, hv));
        t = ff_sum(t, ff_prod(x, mx));
      }
      for (int o = 16; o > 0; o >>= 1) t = ff_sum(t, ff{__shfl_xor_sync(FULL_MASK, t.h, o),
                                                        __shfl_xor_sync(FULL_MASK, t.l, o)});
      double cv = ff_dbl(ff_sum(ff_of(a.bb[u.s]), t));
      if (!isfinite(cv)) cv = INFINITY;
      if (cv < 0.0) cv = 0.0;
      if (cost && r == 0) cost[q] = cv;
      if (weights && r < nm1) weights[(int64_t)q * nm1 + r] = r < n ? ff_dbl(x) : 0.0;
      if (!grad) continue;
      // adjoint w = M^-1 (s * (M x_hat - h))
      ff rw{0.f, 0.f};
      if (r < n) {
        rw = ff_sum(mx, ff_neg(hv));
        if (sg < 0.f) rw = ff_neg(rw);
      }
      ff w;
      if (!warp_refined_solve(m, n1, n, r, rw, w, SUMS_REFINE)) {
        if (r < nmax) grad[(int64_t)q * nmax + r] = 0.0;
        continue;
      }
      __syncwarp();
      if (r < n) m.w[r] = w;
      __syncwarp();
      // d cost / d theta_i in lane r = i + 1 (the formula of k_solve_sums)
      if (r >= 1 && r <= nmax) {
        const int i = r - 1;
        double gi = 0.0;
        if (i < N) {
          const ff ln10 = ff_of(2.302585092994046);
          const ff Di = ff_of(a.sc.G[(int64_t)(2 * N + i) * Q + q]);
          const ff Ei = ff_of(a.sc.G[(int64_t)(3 * N + i) * Q + q]);
          const ff ti = m.tau[r], Si = m.S[r];
          ff ax = ff_prod(Di, m.xh[0]), aw = ff_prod(Di, m.w[0]), as = ax;
          for (int j = 1; j < n; ++j) {
            if (j == r) continue;
            const ff rr = ff_quot(ff{1.f, 0.f}, ff_sum(ti, m.tau[j]));
            const ff t1 = ff_prod(ff_prod(ti, Di), rr);
            const ff t2 = ff_prod(ff_prod(ff_prod(ln10, ff_prod(ti, m.tau[j])), ff_sum(Si, ff_neg(m.S[j]))),
                                  ff_prod(rr, rr));
            const ff row = ff_sum(t1, t2);
            const ff xj = m.xh[j];
            const ff xs = m.sgn[j] < 0.f ? ff_neg(xj) : xj;
            ax = ff_sum(ax, ff_prod(row, xj));
            aw = ff_sum(aw, ff_prod(row, m.w[j]));
            as = ff_sum(as, ff_prod(row, xs));
          }
          const ff diag = ff_prod(Di, one_lam);
          const ff xhI = x, wI = w;
          const ff xsI = sg < 0.f ? ff_neg(xhI) : xhI;
          const ff x2{__fmul_rn(2.f, xhI.h), __fmul_rn(2.f, xhI.l)};
          ff gsum = ff_neg(ff_prod(x2, Ei));
          gsum = ff_sum(gsum, ff_prod(x2, ax));
          gsum = ff_sum(gsum, ff_prod(diag, ff_prod(xhI, xhI)));
          ff adj = ff_prod(wI, Ei);
          adj = ff_sum(adj, ff_neg(ff_prod(wI, as)));
          adj = ff_sum(adj, ff_neg(ff_prod(xsI, aw)));
          adj = ff_sum(adj, ff_neg(ff_prod(diag, ff_prod(wI, xsI))));
          gsum = ff_sum(gsum, ff{__fmul_rn(2.f, adj.h), __fmul_rn(2.f, adj.l)});
          gi = ff_dbl(gsum);
        }
        grad[(int64_t)q * nmax + i] = gi;
      }
    }
  }
}

// ------------------------------------------------------------------ gradient
// w = M^-1 S g_hat with g_hat = g1 - M (x_hat - x1) = h - M x_hat,
// S = diag(1, sign x1_1, ..., sign x1_N).
template <typename T>
__global__ void __launch_bounds__(256) k_grad_prep(EvalArgs a, const double* g1, double* sg_out) {
  const int64_t Q = a.sc.Q;
  const T* Lg = factor_base<T>(a.sc);
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int q = u.q0 + (int)threadIdx.x;
    if (q >= u.q1 || (a.active && !a.active[q])) continue;
    if (a.sc.fail[q]) continue;
    const int n = u.N + 1;
    T L[NPACK_MAX], t1[NMAX1], t2[NMAX1];
    double e[NMAX1];
    Scale<T> sc;
    sc.load(a.sc, q, n);
    const int npk = n * (n + 1) / 2;
    for (int k = 0; k < npk; ++k) L[k] = Lg[(int64_t)k * Q + q];
    for (int i = 0; i < n; ++i) {
      const double x1 = a.sc.x[(int64_t)i * Q + q];
      e[i] = a.sc.xh[(int64_t)i * Q + q] - x1;
      t1[i] = (T)(sc.d[i] * e[i]);
    }
    lt_mul(L, t1, t2, n);
    l_mul(L, t2, t1, n);           // M e = D t1
    for (int i = 0; i < n; ++i) {
      const double x1 = a.sc.x[(int64_t)i * Q + q];
      double gh = g1[(int64_t)i * Q + q] - sc.d[i] * (double)t1[i];
      if (i > 0 && x1 < 0.0) gh = -gh;
      if (sg_out) sg_out[(int64_t)i * Q + q] = gh;   // S g_hat, kept for the refinement of w
      t2[i] = sc.down(gh, i);
    }
    llt_solve(L, t2, n);
    for (int i = 0; i < n; ++i) a.sc.w[(int64_t)i * Q + q] = sc.up(t2[i], i);
  }
}

__global__ void __launch_bounds__(256) k_grad_finish(EvalArgs a, double* grad) {
  const int64_t Q = a.sc.Q;
  const int nmax = a.sc.nmax;
  for (int ui = blockIdx.x; ui < a.n_units; ui += gridDim.x) {
    const Unit u = a.units[ui];
    const int q = u.q0 + (int)threadIdx.x;
    if (q >= u.q1 || (a.active && !a.active[q])) continue;
    const int N = u.N;
    if (a.sc.fail[q]) {
      for (int i = 0; i < nmax; ++i) grad[(int64_t)q * nmax + i] = 0.0;
      continue;
    }
    for (int i = 0; i < nmax; ++i) {
      double gi = 0.0;
      if (i < N) {
        const double xh = a.sc.xh[(int64_t)(i + 1) * Q + q];
        const double x1 = a.sc.x[(int64_t)(i + 1) * Q + q];
        const double w = a.sc.w[(int64_t)(i + 1) * Q + q];
        const double t_rh = a.sc.gt[(int64_t)i * Q + q];
        const double t_aa = a.sc.gt[(int64_t)(N + i) * Q + q];
        const double t_r = a.sc.gt[(int64_t)(2 * N + i) * Q + q];
        const double t_aw = a.sc.gt[(int64_t)(3 * N + i) * Q + q];
        gi = -2.0 * xh * t_rh + 2.0 * a.lam * xh * xh * t_aa - 2.0 * w * t_r +
             4.0 * a.lam * w * x1 * t_aa + 2.0 * x1 * t_aw;
      }
      grad[(int64_t)q * nmax + i] = gi;
    }
  }
}

// ------------------------------------------------------------------ host launchers
void launch_prep(int64_t n_samples, int64_t S, const int64_t* offsets, const double* omega,
                 const double* er, const double* ei, const double* lo, const double* hi,
                 float4* kf32, float4* kff, double* h0, int* status, int sms, cudaStream_t st) {
  if (n_samples > 0) {
    int grid = (int)std::min<int64_t>((n_samples + 255) / 256, (int64_t)sms * 16);
    k_prep_samples<<<grid, 256, 0, st>>>(n_samples, omega, er, ei, kf32, kff, status);
  }
  if (S > 0) {
    int grid = (int)std::min<int64_t>(S, (int64_t)sms * 8);
    k_prep_spectra<<<grid, 256, 0, st>>>(S, offsets, er, ei, lo, hi, h0, h0 + S, status);
  }
}

static int grid_for(int n_units, int sms, int per_sm) {
  return std::max(1, std::min(n_units, sms * per_sm));
}

// One thread per candidate with per-thread arrays in local memory: a grid of up to
// 32 blocks per SM keeps enough warps resident to hide that memory's latency.
void launch_solve_sums(const EvalArgs& a, double* cost, double* weights, double* grad, int block, int sms,
                       cudaStream_t st) {
  if (!a.n_units) return;
  if (grad) k_solve_sums_t<0, 1><<<grid_for(a.n_units, sms, 32), block, 0, st>>>(a, cost, weights, grad);
  else k_solve_sums_t<0, 0><<<grid_for(a.n_units, sms, 32), block, 0, st>>>(a, cost, weights, nullptr);
}

bool solve_sums_by_warp(int64_t Q, int lanes, int sms) {
  if (lanes == 1 || lanes == 32) return lanes == 32;
  return Q <= (int64_t)sms * WARP_SOLVE_MAX_Q_PER_SM;
}

// A block of up to 8 warps (one candidate each) per unit, within the default 48 KB
// of shared memory (6.3 KB per warp at 20 poles).
void launch_solve_sums_warp(const EvalArgs& a, double* cost, double* weights, double* grad, int cands_per_unit,
                            int sms, cudaStream_t st) {
  if (!a.n_units) return;
  const size_t per = warp_solve_bytes(a.sc.nmax + 1);
  int warps = std::max(1, std::min(WARP_SOLVE_MAX_WARPS, cands_per_unit));
  while (warps > 1 && (size_t)warps * per > 48 * 1024) --warps;
  k_solve_sums_warp<<<grid_for(a.n_units, sms, 16), warps * 32, warps * per, st>>>(a, cost, weights, grad);
}

void launch_solve(const EvalArgs& a, int block, int sms, cudaStream_t st) {
  if (a.n_units) k_solve<double><<<grid_for(a.n_units, sms, 8), block, 0, st>>>(a);
}
void launch_finish(const EvalArgs& a, int final_step, double* cost, double* weights, double* g1,
                   int block, int sms, cudaStream_t st) {
  if (a.n_units) k_finish<double><<<grid_for(a.n_units, sms, 8), block, 0, st>>>(a, final_step, cost, weights, g1);
}
void launch_grad_prep(const EvalArgs& a, const double* g1, double* sg_out, int block, int sms, cudaStream_t st) {
  if (a.n_units) k_grad_prep<double><<<grid_for(a.n_units, sms, 8), block, 0, st>>>(a, g1, sg_out);
}
void launch_grad_finish(const EvalArgs& a, double* grad, int block, int sms, cudaStream_t st) {
  if (a.n_units) k_grad_finish<<<grid_for(a.n_units, sms, 8), block, 0, st>>>(a, grad);
}

}  // namespace debyefit

// ------------------------------------------------------------------ target synthesis (Eqs. 3-7)
namespace debyefit {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx c_add(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx c_scale(cplx a, double s) { return {a.re * s, a.im * s}; }
// Principal power z^p = |z|^p exp(j p arg z).
__device__ __forceinline__ cplx c_pow(cplx z, double p) {
  const double m = pow(hypot(z.re, z.im), p), t = p * atan2(z.im, z.re);
  double sn, cs;
  sincos(t, &sn, &cs);
  return {m * cs, m * sn};
}
// Debye pole eps_inf + d_eps / (1 + j x), x = omega tau (Eq. 3), as a complex number.
__device__ __forceinline__ cplx c_debye(double ei, double de, double x) {
  const double r = 1.0 / (1.0 + x * x);
  return {ei + de * r, -de * x * r};
}

__global__ void k_synth(int64_t S, const int64_t* __restrict__ offsets, const double* __restrict__ omega,
                        const int32_t* __restrict__ model, const double* __restrict__ params,
                        const int64_t* __restrict__ pole_off, const double* __restrict__ ptau,
                        const double* __restrict__ pdeps, const double* __restrict__ nre,
                        const double* __restrict__ nim, double* __restrict__ er,
                        double* __restrict__ ei, int* status) {
  constexpr double PI = 3.141592653589793;
  for (int64_t s = blockIdx.x; s < S; s += gridDim.x) {
    const double* p = params + s * DEBYE_N_PARAMS;
    const int m = model[s];
    for (int64_t k = offsets[s] + threadIdx.x; k < offsets[s + 1]; k += blockDim.x) {
      const double w = omega[k];
      cplx e = {0.0, 0.0};
      double sigma = 0.0;
      switch (m) {
        case DEBYE_MODEL_DEBYE:
          e = c_debye(p[0], p[1], w * p[2]);
          break;
        case DEBYE_MODEL_HN:
        case DEBYE_MODEL_CC:
        case DEBYE_MODEL_CD: {
          // (j w tau0)^alpha on the principal branch, then (1 + .)^beta
          const double al = p[3], be = p[4];
          const double mag = pow(w * p[2], al);
          double sn, cs;
          sincos(al * PI / 2, &sn, &cs);
          const cplx den = c_pow(cplx{1.0 + mag * cs, mag * sn}, be);
          const double dd = den.re * den.re + den.im * den.im;
          e = {p[0] + p[1] * den.re / dd, -p[1] * den.im / dd};
          break;
        }
        case DEBYE_MODEL_JONSCHER: {
          const double f = p[1] * pow(w / p[2], p[3] - 1.0);
          e = {p[0] + f, -f / tan(p[3] * PI / 2)};
          break;
        }
        case DEBYE_MODEL_JONSCHER_EQ5: {
          const double f = p[1] * pow(w / p[2], p[3]);
          double sn, cs;
          sincos(p[3] * PI / 2, &sn, &cs);
          e = {p[0] + f * cs, -f * sn};
          break;
        }
        case DEBYE_MODEL_CRIM: {
          const double a = p[0];
          const int nc = (int)p[1];
          cplx acc = {0.0, 0.0};
          for (int i = 0; i < nc && i < 3; ++i)
            acc = c_add(acc, c_scale(c_pow(c_debye(p[5 + 3 * i], p[6 + 3 * i], w * p[7 + 3 * i]), a), p[2 + i]));
          e = c_pow(acc, 1.0 / a);
          break;
        }
        case DEBYE_MODEL_DEBYE_SUM: {
          e = {p[0], 0.0};
          for (int64_t j = pole_off[s]; j < pole_off[s + 1]; ++j) e = c_add(e, c_debye(0.0, pdeps[j], w * ptau[j]));
          const double f = p[1] * pow(w / p[2], p[3] - 1.0);
          e = c_add(e, cplx{f, -f / tan(p[3] * PI / 2)});
          sigma = p[4];
          break;
        }
        default:
          set_status(status, DEBYE_EBOUNDS);
      }
      double vr = e.re, vi = -e.im;   // eps' and eps'' (Eq. 1)
      if (nre && sigma != 0.0) {
        vr *= 1.0 + sigma * nre[k];
        vi *= 1.0 + sigma * nim[k];
      }
      er[k] = vr;
      ei[k] = vi;
    }
  }
}

void launch_synth(int64_t S, const int64_t* offsets, const double* omega, const int32_t* model,
                  const double* params, const int64_t* pole_off, const double* ptau,
                  const double* pdeps, const double* nre, const double* nim, double* er, double* ei,
                  int* status, int sms, cudaStream_t st) {
  if (S <= 0) return;
  int grid = (int)std::min<int64_t>(S, (int64_t)sms * 8);
  k_synth<<<grid, 256, 0, st>>>(S, offsets, omega, model, params, pole_off, ptau, pdeps, nre, nim,
                                er, ei, status);
}

}  // namespace debyefit
