// Per-N pass kernels for poles N = 17..20 (one translation unit per bucket so
// the buckets compile in parallel).
#include "eval.cuh"
#include "launch.h"

namespace debyefit {

void launch_pass_b4(int phase, bool mixed, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  constexpr int LO = 17, HI = 20;
  // mixed-precision passes up to 12 poles fit in 168 registers without spills:
  // cap them for 3 resident 128-thread blocks; larger N keeps the full register
  // file, and its Gram pass may run two warps per candidate group (256 threads)
  constexpr int MB_MIXED = HI <= 12 ? 3 : 1;
  constexpr int MAXT = HI <= 12 ? 128 : 256;
  if (mixed) {
    if (phase == PH_GRAM) {
      const int per_thread = a.gs == 2 ? split_part_floats(HI) : gram_smem_stride(HI);
      const size_t smem = sizeof(float) * per_thread * block;
      static bool attr_set = false;
      if (!attr_set) {
        const int most = std::max(gram_smem_stride(HI) * MAX_BLOCK, split_part_floats(HI) * 2 * MAX_BLOCK);
        cudaFuncSetAttribute(k_pass<PH_GRAM, LO, HI, true, MAXT, MB_MIXED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * most));
        attr_set = true;
      }
      k_pass<PH_GRAM, LO, HI, true, MAXT, MB_MIXED><<<grid, block, smem, st>>>(a);
    }
    else if (phase == PH_REFINE) k_pass<PH_REFINE, LO, HI, true, MAXT, MB_MIXED><<<grid, block, 0, st>>>(a);
    else k_pass<PH_GRAD, LO, HI, true, MAXT, 1><<<grid, block, 0, st>>>(a);
  } else {
    if (phase == PH_GRAM) k_pass<PH_GRAM, LO, HI, false, MAXT, 1><<<grid, block, 0, st>>>(a);
    else if (phase == PH_REFINE) k_pass<PH_REFINE, LO, HI, false, MAXT, 1><<<grid, block, 0, st>>>(a);
    else k_pass<PH_GRAD, LO, HI, false, MAXT, 1><<<grid, block, 0, st>>>(a);
  }
}

}  // namespace debyefit
