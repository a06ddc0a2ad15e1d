// Shared device-side definitions of libdebyefit (sm_103a).
//
// Work decomposition: every evaluation works on a flat list of candidates q.
// Candidate q belongs to one spectrum; a Unit is a run of at most `cb`
// consecutive candidates of one spectrum, processed by one thread block with
// one thread per candidate. Per-candidate scratch is stored structure-of-arrays,
// element e of candidate q at base[e * Q + q], so a warp's 32 candidates touch 32
// consecutive doubles.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/debyefit.h"

namespace debyefit {

constexpr int NMAX = DEBYE_MAX_POLES;   // largest pole count
constexpr int NMAX1 = NMAX + 1;         // unknowns: eps_inf + d_eps_1..N
constexpr int NPACK_MAX = NMAX1 * (NMAX1 + 1) / 2;

// Packed lower-triangular index of (I, J), J <= I.
__host__ __device__ constexpr int pk(int I, int J) { return I * (I + 1) / 2 + J; }

enum Phase { PH_GRAM = 0, PH_REFINE = 1, PH_GRAD = 2, PH_SUMS = 3, PH_SUMSG = 4,
             // mixed precision: weights, cost (and gradient) from a bucket's column sums,
             // one thread per candidate, the pole count fixed at compile time
             PH_SOLVE = 5, PH_SOLVEG = 6,
             // FP64 column sums and the Gram from the partial-fraction identity (FP64 path)
             PH_GRAM_SUMS = 7 };
// Largest pole count with a compile-time (register-resident) column-sum solve;
// larger ones use the general kernel.
constexpr int SOLVE_N_MAX = 12;
// The column sums with the derivative sums (eval.cuh, sums_sq_unit) sweep the
// samples once for up to this many poles (14 registers per pole) and twice, about
// N/2 poles each, above it; the cost-only sums (8 registers per pole) always sweep
// once.
constexpr int SQUARED_CHUNK_GRAD = 11;

struct Unit {
  int32_t s;    // spectrum
  int32_t q0;   // first candidate
  int32_t q1;   // one past the last candidate
  int32_t N;    // poles of this spectrum
  int64_t k0;   // first sample of the spectrum
  int64_t k1;   // one past the last sample
};

// Per-call views of the candidate scratch (all device pointers).
struct Scratch {
  int64_t Q;        // candidates in this evaluation (SoA stride)
  int32_t nmax;     // pole capacity of theta / weights rows
  int32_t ng;       // per-candidate Gram record: packed (nmax+1) lower triangle + h
  double* G;        // [ng][Q]   Gram (packed) followed by h = A^T b
  double* L;        // [npk][Q]  Cholesky factor of the scaled damped matrix
  double* dinv;     // [nmax+1][Q] 1 / sqrt(G_ii)
  double* x;        // [nmax+1][Q] current (unflipped) weights
  double* xh;       // [nmax+1][Q] flipped weights
  double* w;        // [nmax+1][Q] adjoint solve M^-1 S g_hat (gradient only)
  double* rt;       // [nmax+2][Q] rr = ||r||^2 then t = A^T r
  double* gt;       // [4*nmax][Q] gradient projections
  int32_t* fail;    // [Q] non-zero: candidate's damped matrix not positive definite
};

// Per-spectrum Chebyshev tables of the column sums (DEBYE_PREC_MIXED_TABLE). Over the
// spectrum's log10(tau) box [lo, lo + nseg TAB_W], each column sum of one Debye pole
// is a function of theta alone: S = sum_k re_k, h = a_i^T b and their theta
// derivatives (tau = 10^theta is tabulated with them). Every term 1 / (1 + w_k^2 tau^2) is analytic in the strip
// |Im ln tau^2| < pi whatever the samples, so on segments of TAB_W decades a
// Chebyshev interpolant of degree TAB_NC - 1 reaches the float-float sums' rounding.
constexpr double TAB_W = 0.2;    // decades of log10(tau) per segment
constexpr double TAB_INV_W = 5.0;   // 1 / TAB_W
constexpr int TAB_NC = 12;       // Chebyshev coefficients per segment and function
// Functions per segment: S, h and tau = 10^theta itself (an entire function, so its
// series converges faster still), which the cost needs, then dS/dtheta and dh/dtheta
// for the gradient.
constexpr int TAB_NF = 5;
constexpr int TAB_NODE_N = 20;   // nodes per pseudo-candidate of the table's node pass
constexpr int TAB_MAX_SEG = 1000;   // segments per spectrum (a box of at most 200 decades)

struct TabView {
  const float2* coef;      // [sum_s nseg_s][TAB_NF][TAB_NC] coefficients (hi, lo), c_0 halved;
                           //   functions S, h, tau, dS/dtheta, dh/dtheta
  const int64_t* seg0;     // [S] first segment of spectrum s
  const int32_t* nseg;     // [S] segments of spectrum s
  const double* lo;        // [S] table origin: the spectrum's lower bound
};

struct EvalArgs {
  const Unit* units;
  int32_t n_units;
  const double* theta;     // [Q][nmax] log10 tau
  const float4* kf32;      // [sum K] {omega_hi, eps'_hi, eps''_hi, 0}
  const float4* kff;       // [sum K] {omega_lo, eps'_lo, eps''_lo, 0}
  const float4* kq32;      // [sum K] {(omega 2^-30)^2, eps', omega eps''} high parts
  const float4* kqff;      // [sum K] their low parts (float-float)
  const double* omega;     // [sum K] FP64 inputs
  const double* eps_re;
  const double* eps_im;
  const double* h0;        // [S] sum_k eps'_k
  const double* bb;        // [S] b^T b = sum_k eps'_k^2 + eps''_k^2
  const uint8_t* active;   // [Q] optional candidate mask (nullptr: all)
  int32_t* n_failed;       // [S] optional: +1 per evaluated candidate whose damped matrix is not
                           //   positive definite (its cost is +inf)
  int32_t ks;              // lanes per candidate in the pass kernels (power of two <= 32)
  double lam;
  double* out_cost;        // PH_SOLVE / PH_SOLVEG outputs: cost [Q], weights [Q][nmax+1] or
  double* out_weights;     //   nullptr, gradient [Q][nmax] (PH_SOLVEG)
  double* out_grad;
  Scratch sc;
  TabView tab;             // DEBYE_PREC_MIXED_TABLE: the spectra's column-sum tables
  int* status;             // device status word
};

// ------------------------------------------------------------------ status word
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Record the outcome of candidate q's factorisation (spectrum s).
__device__ __forceinline__ void record_fail(const EvalArgs& a, int q, int s, bool ok) {
  a.sc.fail[q] = ok ? 0 : 1;
  if (!ok && a.n_failed) atomicAdd(&a.n_failed[s], 1);
}

// ------------------------------------------------------------------ float-float helpers
// Error-free transformations (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2). The
// __f*_rn intrinsics keep the compiler from contracting the rounded operations
// into FMAs, which would break the error terms.
__device__ __forceinline__ float rcp_approx(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// s + e == a + b exactly (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void split_double(double v, float& hi, float& lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}

// acc (hi, lo) += a * b, a and b float-float (one Dot2 step: TwoProduct by FMA,
// TwoSum of the leading part, low-order terms gathered in lo).
__device__ __forceinline__ void ff_add_prod(float& ah, float& al, float xh, float xl, float yh,
                                            float yl) {
  float p = __fmul_rn(xh, yh);
  float pe = __fmaf_rn(xh, yh, -p);
  pe = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, pe));
  float s, e;
  two_sum(ah, p, s, e);
  ah = s;
  al = __fadd_rn(al, __fadd_rn(e, pe));
}

// Float-float product (ph, pl) = (ah, al) * (bh, bl) to about 2^-46 relative.
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  ph = __fmul_rn(ah, bh);
  pl = __fmaf_rn(ah, bh, -ph);
  pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pl));
}

// Float-float value (hi + lo, |lo| <= ulp(hi)/2 after normalisation) for the
// per-candidate small-system algebra of the mixed path.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_of(double v) {
  ff r;
  r.h = __double2float_rn(v);
  r.l = __double2float_rn(v - (double)r.h);
  return r;
}
__device__ __forceinline__ double ff_dbl(ff a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ ff ff_sum(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return ff{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_prod(ff a, ff b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  const float h = __fadd_rn(p, e);
  return ff{h, __fsub_rn(e, __fsub_rn(h, p))};
}
// a / b: quotient q1 = a_h / b_h corrected by the float-float remainder a - q1 b.
// Both quotients multiply by the approximate reciprocal of b_h (rcp.approx, about
// 1 ulp): the float-float remainder carries q1's error, so a / b keeps ~2^-43.
__device__ __forceinline__ ff ff_quot(ff a, ff b) {
  const float rb = rcp_approx(b.h);
  const float q1 = __fmul_rn(a.h, rb);
  const ff r = ff_sum(a, ff_neg(ff_prod(ff{q1, 0.f}, b)));
  const float q2 = __fmul_rn(r.h, rb);
  const float h = __fadd_rn(q1, q2);
  return ff{h, __fsub_rn(q2, __fsub_rn(h, q1))};
}



// ------------------------------------------------------------------ SplitMix64
// Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014: the SplitMix64 output function used as a key mixer.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Key prefix over (seed, tag, spectrum, generation).
__host__ __device__ __forceinline__ uint64_t rng_prefix(uint64_t seed, uint64_t tag, uint64_t s,
                                                        uint64_t g) {
  uint64_t h = splitmix64(seed);
  h = splitmix64(h ^ tag);
  h = splitmix64(h ^ s);
  return splitmix64(h ^ g);
}

// Full 64-bit key for (prefix, particle, dim).
__host__ __device__ __forceinline__ uint64_t rng_key(uint64_t prefix, uint64_t p, uint64_t d) {
  return splitmix64(splitmix64(prefix ^ p) ^ d);
}

// Uniform double in [0, 1) for (prefix, particle, dim): the key's upper 53 bits.
__host__ __device__ __forceinline__ double rng_uniform(uint64_t prefix, uint64_t p, uint64_t d) {
  return (double)(rng_key(prefix, p, d) >> 11) * (1.0 / 9007199254740992.0);
}

// Integer in [0, m), m < 2^32: multiply-shift of the key's upper 32 bits (Lemire 2019,
// without rejection).
__host__ __device__ __forceinline__ uint32_t rng_below(uint64_t key, uint32_t m) {
  return (uint32_t)(((key >> 32) * (uint64_t)m) >> 32);
}

constexpr uint64_t TAG_INIT_POS = 1, TAG_INIT_VEL = 2, TAG_R1 = 3, TAG_R2 = 4;
// differential evolution: donor indices, forced coordinate, crossover, bound re-draw, F
constexpr uint64_t TAG_DE_IDX = 5, TAG_DE_J = 6, TAG_DE_CR = 7, TAG_DE_BOUND = 8, TAG_DE_F = 9;
// dual annealing: uniforms of the visiting deviates, acceptance draws
constexpr uint64_t TAG_DA_VISIT = 10, TAG_DA_ACCEPT = 11;

}  // namespace debyefit
