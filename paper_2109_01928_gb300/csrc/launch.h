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
constexpr int MAX_BLOCK = 128; // largest pass block (candidates x lanes; mixed Gram shared memory at N = 20)
__host__ __device__ constexpr int bucket_of(int N) { return N - 1; }

// Work layout for spectra with `per_spectrum` candidates each: `cb` candidates per
// unit and `ks` lanes per candidate, 64 threads per pass block. Full populations
// get one lane per candidate; a handful of candidates (line-search points, one
// re-solve per spectrum) get several lanes each so that warps stay full.
// cb_opt > 0 fixes the candidates per unit (lanes stay 1 unless the spectrum has
// fewer candidates than a warp).
inline void choose_layout(int64_t per_spectrum, int cb_opt, int* cb, int* ks) {
  int p2 = 1;
  while (p2 < per_spectrum && p2 < 64) p2 <<= 1;
  if (cb_opt > 0 && per_spectrum >= 32) {
    *cb = cb_opt;
    *ks = 1;
    return;
  }
  *ks = std::min(32, std::max(1, 64 / p2));
  *cb = std::max(1, 64 / *ks);
}

// Per-N passes (eval.cuh); pole counts 1-4, 5-8, 9-12, 13-16 and 17-20 compile in
// separate translation units (pass_b0.cu .. pass_b4.cu) so that they build in parallel.
void launch_pass_b0(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b1(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b2(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b3(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b4(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
inline void launch_pass(int N, int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch ((N - 1) / 4) {
    case 0: launch_pass_b0(N, phase, mixed, a, grid, block, st); break;
    case 1: launch_pass_b1(N, phase, mixed, a, grid, block, st); break;
    case 2: launch_pass_b2(N, phase, mixed, a, grid, block, st); break;
    case 3: launch_pass_b3(N, phase, mixed, a, grid, block, st); break;
    default: launch_pass_b4(N, phase, mixed, a, grid, block, st); break;
  }
}

void launch_prep(int64_t n_samples, int64_t S, const int64_t* offsets, const double* omega,
                 const double* er, const double* ei, const double* lo, const double* hi,
                 float4* kf32, float4* kff, double* h0, int* status, int sms, cudaStream_t st);
inline int warp_round(int n) { return (n + 31) / 32 * 32; }
void launch_solve(const EvalArgs& a, int block, int sms, cudaStream_t st);
void launch_finish(const EvalArgs& a, int final_step, double* cost, double* weights, double* g1,
                   int block, int sms, cudaStream_t st);
void launch_grad_prep(const EvalArgs& a, const double* g1, double* sg_out, int block, int sms, cudaStream_t st);
void launch_adjoint_refine(const EvalArgs& a, const double* sg, int block, int sms, cudaStream_t st);
void launch_grad_finish(const EvalArgs& a, double* grad, int block, int sms, cudaStream_t st);

}  // namespace debyefit

namespace debyefit {
void launch_synth(int64_t S, const int64_t* offsets, const double* omega, const int32_t* model,
                  const double* params, const int64_t* pole_off, const double* ptau,
                  const double* pdeps, const double* nre, const double* nim, double* er, double* ei,
                  int* status, int sms, cudaStream_t st);
}  // namespace debyefit
