// Pass kernels for pole counts N = 5..8, one kernel per N (one translation
// unit per group of four so that the groups compile in parallel).
#include "pass.cuh"

namespace debyefit {

void launch_pass_b1(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch (N) {
    case 5: launch_pass_n<5>(phase, a, grid, block, st); break;
    case 6: launch_pass_n<6>(phase, a, grid, block, st); break;
    case 7: launch_pass_n<7>(phase, a, grid, block, st); break;
    default: launch_pass_n<8>(phase, a, grid, block, st); break;
  }
}

}  // namespace debyefit
