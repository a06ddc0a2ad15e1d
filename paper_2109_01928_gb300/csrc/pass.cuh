// Launch of the pass kernels of one pole count N (included by pass_b*.cu).
#pragma once
#include "eval.cuh"
#include "launch.h"

namespace debyefit {

template <int N>
void launch_pass_n(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  // mixed-precision passes up to 12 poles fit in 168 registers without spills:
  // cap them for 3 resident 128-thread blocks; larger N keeps the full register
  // file, and its Gram pass may run two warps per candidate group (256 threads)
  constexpr int MB_MIXED = N <= 12 ? 3 : 1;
  constexpr int MAXT = N <= 12 ? 128 : 256;
  if (mixed) {
    if (phase == PH_GRAM) {
      const int per_thread = a.gs == 2 ? split_part_floats(N) : gram_smem_stride(N);
      const size_t smem = sizeof(float) * per_thread * block;
      static bool attr_set = false;
      if (!attr_set) {
        const int most = std::max(gram_smem_stride(N) * MAX_BLOCK, split_part_floats(N) * 2 * MAX_BLOCK);
        cudaFuncSetAttribute(k_pass<PH_GRAM, N, N, true, MAXT, MB_MIXED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * most));
        attr_set = true;
      }
      k_pass<PH_GRAM, N, N, true, MAXT, MB_MIXED><<<grid, block, smem, st>>>(a);
    }
    else if (phase == PH_REFINE) k_pass<PH_REFINE, N, N, true, MAXT, MB_MIXED><<<grid, block, 0, st>>>(a);
    else if (phase == PH_SUMS) k_pass<PH_SUMS, N, N, true, MAXT, MB_MIXED><<<grid, block, 0, st>>>(a);
    else if (phase == PH_SUMSG) k_pass<PH_SUMSG, N, N, true, MAXT, 1><<<grid, block, 0, st>>>(a);
    else k_pass<PH_GRAD, N, N, true, MAXT, 1><<<grid, block, 0, st>>>(a);
  } else {
    if (phase == PH_GRAM) k_pass<PH_GRAM, N, N, false, MAXT, 1><<<grid, block, 0, st>>>(a);
    else if (phase == PH_REFINE) k_pass<PH_REFINE, N, N, false, MAXT, 1><<<grid, block, 0, st>>>(a);
    else k_pass<PH_GRAD, N, N, false, MAXT, 1><<<grid, block, 0, st>>>(a);
  }
}

}  // namespace debyefit
