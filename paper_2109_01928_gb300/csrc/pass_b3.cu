// Pass kernels for pole counts N = 13..16, one kernel per N (one translation
// unit per group of four so that the groups compile in parallel).
#include "pass.cuh"

namespace debyefit {

void launch_pass_b3(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch (N) {
    case 13: launch_pass_n<13>(phase, a, grid, block, st); break;
    case 14: launch_pass_n<14>(phase, a, grid, block, st); break;
    case 15: launch_pass_n<15>(phase, a, grid, block, st); break;
    default: launch_pass_n<16>(phase, a, grid, block, st); break;
  }
}

}  // namespace debyefit
