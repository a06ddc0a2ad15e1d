// Host-side launchers shared by the translation units of libdebyefit.
#pragma once
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace debyefit {

constexpr int N_BUCKETS = 5;  // pole buckets compiled into separate kernels
constexpr int MAX_BLOCK = 128; // largest pass block (candidates x lanes; mixed Gram shared memory at N = 20)
__host__ __device__ constexpr int bucket_lo(int b) { return 4 * b + 1; }
__host__ __device__ constexpr int bucket_hi(int b) { return 4 * b + 4; }
__host__ __device__ constexpr int bucket_of(int N) { return (N - 1) / 4; }

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

// Per-N passes (eval.cuh), one translation unit per bucket.
void launch_pass_b0(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b1(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b2(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b3(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b4(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);

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
