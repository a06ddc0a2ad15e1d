// Pass kernels for pole counts N = 1..4, one kernel per N (one translation
// unit per group of four so that the groups compile in parallel).
#include "pass.cuh"

namespace debyefit {

void launch_pass_b0(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch (N) {
    case 1: launch_pass_n<1>(phase, a, grid, block, st); break;
    case 2: launch_pass_n<2>(phase, a, grid, block, st); break;
    case 3: launch_pass_n<3>(phase, a, grid, block, st); break;
    default: launch_pass_n<4>(phase, a, grid, block, st); break;
  }
}

}  // namespace debyefit
