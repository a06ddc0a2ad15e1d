// Host-side launchers shared by the translation units of libdebyefit.
#pragma once
#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace debyefit {

constexpr int N_BUCKETS = 5;  // pole buckets compiled into separate kernels
constexpr int MAX_BLOCK = 128; // largest candidates-per-block (mixed Gram shared memory at N = 20)
__host__ __device__ constexpr int bucket_lo(int b) { return 4 * b + 1; }
__host__ __device__ constexpr int bucket_hi(int b) { return 4 * b + 4; }
__host__ __device__ constexpr int bucket_of(int N) { return (N - 1) / 4; }

// Per-N passes (eval.cuh), one translation unit per bucket.
void launch_pass_b0(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b1(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b2(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b3(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);
void launch_pass_b4(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st);

void launch_prep(int64_t n_samples, int64_t S, const int64_t* offsets, const double* omega,
                 const double* er, const double* ei, const double* lo, const double* hi,
                 float4* kf32, float4* kff, double* h0, int* status, int sms, cudaStream_t st);
void launch_solve(const EvalArgs& a, int block, int sms, cudaStream_t st);
void launch_finish(const EvalArgs& a, int final_step, double* cost, double* weights, double* g1,
                   int block, int sms, cudaStream_t st);
void launch_grad_prep(const EvalArgs& a, const double* g1, int block, int sms, cudaStream_t st);
void launch_grad_finish(const EvalArgs& a, double* grad, int block, int sms, cudaStream_t st);

}  // namespace debyefit

namespace debyefit {
void launch_synth(int64_t S, const int64_t* offsets, const double* omega, const int32_t* model,
                  const double* params, const int64_t* pole_off, const double* ptau,
                  const double* pdeps, const double* nre, const double* nim, double* er, double* ei,
                  int* status, int sms, cudaStream_t st);
}  // namespace debyefit
