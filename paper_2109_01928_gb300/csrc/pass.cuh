// Launch of the pass kernels of one pole count N (included by pass_b*.cu).
#pragma once
#include "eval.cuh"
#include "launch.h"
#include "solve_sums.cuh"

namespace debyefit {

// The column-sum passes (PH_SUMS, PH_SUMSG) and the per-N column-sum solves
// (PH_SOLVE, PH_SOLVEG, N <= SOLVE_N_MAX) are the mixed-precision path; the
// Gram, residual and gradient passes the FP64 path.
template <int N>
void launch_pass_n(int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  // the cost-only column-sum pass up to 12 poles fits in 168 registers without
  // spills: cap it for 3 resident 128-thread blocks; larger N, the gradient
  // variant and the FP64 passes keep the full register file (one sweep over the
  // samples keeps a lone active lane's latency low in masked evaluations)
  constexpr int MB_SUMS = N <= 12 ? 3 : 1;
  constexpr int MAXT = N <= 12 ? 128 : 256;
  switch (phase) {
    case PH_SUMS: k_pass_sums<N, false, MAXT, MB_SUMS><<<grid, block, 0, st>>>(a); break;
    case PH_SUMSG: k_pass_sums<N, true, MAXT, 1><<<grid, block, 0, st>>>(a); break;
    case PH_GRAM: k_pass<PH_GRAM, N, N, MAXT, 1><<<grid, block, 0, st>>>(a); break;
    case PH_GRAM_SUMS: k_pass<PH_GRAM_SUMS, N, N, MAXT, 1><<<grid, block, 0, st>>>(a); break;
    case PH_REFINE: k_pass<PH_REFINE, N, N, MAXT, 1><<<grid, block, 0, st>>>(a); break;
    case PH_SOLVE:
    case PH_SOLVEG:
      if constexpr (N <= SOLVE_N_MAX) {   // one thread per candidate (block = candidates per unit)
        const size_t smem = solve_smem_per_thread(N) * block;   // <= 46.6 KB (N = 12, 128 threads)
        if (phase == PH_SOLVE) k_solve_sums_t<N, 0><<<grid, block, smem, st>>>(a, a.out_cost, a.out_weights, nullptr);
        else k_solve_sums_t<N, 1><<<grid, block, smem, st>>>(a, a.out_cost, a.out_weights, a.out_grad);
      }
      break;
    default: k_pass<PH_GRAD, N, N, MAXT, 1><<<grid, block, 0, st>>>(a); break;
  }
}

}  // namespace debyefit
