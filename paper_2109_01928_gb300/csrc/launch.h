// Host-side launchers shared by the translation units of libdebyefit.
#pragma once
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace debyefit {

// One pass kernel per pole count: every warp of a launch runs the same unrolled
// code (no instruction-cache thrashing between pole counts) and each N gets the
// registers it needs. Work units are grouped by N ("buckets").
constexpr int N_BUCKETS = NMAX;
constexpr int MAX_BLOCK = 128; // largest pass block (candidates x lanes)
__host__ __device__ constexpr int bucket_of(int N) { return N - 1; }

// A work layout: candidates per unit (cb) and lanes per candidate (ks); 0 = unset.
struct Layout {
  int cb = 0, ks = 0;
};

// Work layout for spectra with `per_spectrum` candidates each, `total` in the
// batch: `cb` candidates per unit and `ks` lanes per candidate. A population
// that fills the GPU (about 2048 resident threads per SM) is a full population:
// `tuned` (debye_autotune's choice; unset: 64 candidates, one lane each), with
// `forced` (the caller's cands_per_block / lanes_per_candidate options) taking
// precedence field by field; a forced block size alone means one lane per
// candidate, and cb is cut so that cb x ks <= MAX_BLOCK. A forced block size also
// makes any batch with at least a warp of candidates per spectrum a full
// population. A smaller batch (the polish's accepted points, the final re-solve,
// small fits) splits each candidate over ks = 2..32 lanes, sized so that the batch
// fills the GPU and a 64-thread block holds candidates of one spectrum.
inline void choose_layout(int64_t per_spectrum, int64_t total, int sms, Layout forced, Layout tuned, int* cb,
                          int* ks) {
  const int64_t target = (int64_t)std::max(sms, 1) * 2048;
  if (per_spectrum >= 32 && (forced.cb > 0 || 2 * total >= target)) {
    int c = forced.cb > 0 ? forced.cb : (tuned.cb > 0 ? tuned.cb : 64);
    int k = forced.ks > 0 ? forced.ks : (forced.cb > 0 ? 1 : (tuned.ks > 0 ? tuned.ks : 1));
    *ks = k;
    *cb = std::max(1, std::min(c, MAX_BLOCK / k));
    return;
  }
  int p2 = 1;
  while (p2 < per_spectrum && p2 < 64) p2 <<= 1;
  int k = 1;
  while (k < 32 && total * (2 * k) <= target) k <<= 1;
  k = std::min(32, std::max(k, 64 / p2));
  *ks = k;
  *cb = std::max(1, 64 / k);
}

// Per-N passes (eval.cuh); pole counts 1-4, 5-8, 9-12, 13-16 and 17-20 compile in
// separate translation units (pass_b0.cu .. pass_b4.cu) so that they build in parallel.
void launch_pass_b0(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b1(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b2(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b3(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b4(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st);
inline void launch_pass(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch ((N - 1) / 4) {
    case 0: launch_pass_b0(N, phase, a, grid, block, st); break;
    case 1: launch_pass_b1(N, phase, a, grid, block, st); break;
    case 2: launch_pass_b2(N, phase, a, grid, block, st); break;
    case 3: launch_pass_b3(N, phase, a, grid, block, st); break;
    default: launch_pass_b4(N, phase, a, grid, block, st); break;
  }
}

// kf32, kff: [2 n_samples] records (the second half for the squared-form column sums);
// h0: [2 S] doubles, sum_k eps'_k per spectrum, then b^T b per spectrum.
void launch_prep(int64_t n_samples, int64_t S, const int64_t* offsets, const double* omega,
                 const double* er, const double* ei, const double* lo, const double* hi,
                 float4* kf32, float4* kff, double* h0, int* status, int sms, cudaStream_t st);
// Mixed evaluation after the column-sum pass: weights, flip, cost and (grad != nullptr,
// after the pass with derivative sums) the gradient in theta.
void launch_solve_sums(const EvalArgs& a, double* cost, double* weights, double* grad, int block, int sms,
                       cudaStream_t st);
// The same with one warp per candidate (lane r: row r of the small systems), for
// evaluations too small to fill the GPU one thread per candidate. solve_sums_by_warp
// picks it: lanes 1 or 32 force a kernel, 0 takes the warp kernel when the
// evaluation has at most 256 candidates per SM.
bool solve_sums_by_warp(int64_t Q, int lanes, int sms);
void launch_solve_sums_warp(const EvalArgs& a, double* cost, double* weights, double* grad, int cands_per_unit,
                            int sms, cudaStream_t st);
inline int warp_round(int n) { return (n + 31) / 32 * 32; }
void launch_solve(const EvalArgs& a, int block, int sms, cudaStream_t st);
void launch_finish(const EvalArgs& a, int final_step, double* cost, double* weights, double* g1,
                   int block, int sms, cudaStream_t st);
void launch_grad_prep(const EvalArgs& a, const double* g1, double* sg_out, int block, int sms, cudaStream_t st);
void launch_grad_finish(const EvalArgs& a, double* grad, int block, int sms, cudaStream_t st);

}  // namespace debyefit

namespace debyefit {
// Column-sum tables (tables.cu, DEBYE_PREC_MIXED_TABLE). Nodes: theta of every node of
// every spectrum's table into theta_n[qn0[S]][TAB_NODE_N]; coefficients from the node
// pass's sums G[4 TAB_NODE_N][Qn] and taus X[TAB_NODE_N][Qn]; eval: the units' column sums (and with grad their
// theta derivatives) from a.tab into a.sc.x / a.sc.G, as the column-sum pass writes them.
void launch_tab_nodes(int64_t S, const int32_t* qn0, const int32_t* nseg, const double* lo, double* theta_n,
                      int sms, cudaStream_t st);
void launch_tab_coef(int64_t S, const int32_t* qn0, const int32_t* nseg, const int64_t* seg0, const double* G,
                     const double* X, int64_t Qn, float2* coef, int sms, cudaStream_t st);
void launch_tab_eval(const EvalArgs& a, bool grad, int sms, cudaStream_t st);
// One block running the column-sum pass's bounded staging wait with nothing to wait
// for (waitcheck.cu): it records DEBYE_ETIMEOUT after the wait's clock budget;
// waited_ok (device, or nullptr) receives 0.
void launch_stage_wait_check(int* status, int* waited_ok, cudaStream_t st);
void launch_synth(int64_t S, const int64_t* offsets, const double* omega, const int32_t* model,
                  const double* params, const int64_t* pole_off, const double* ptau,
                  const double* pdeps, const double* nre, const double* nim, double* er, double* ei,
                  int* status, int sms, cudaStream_t st);
}  // namespace debyefit
