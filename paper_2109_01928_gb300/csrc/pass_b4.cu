// Pass kernels for pole counts N = 17..20, one kernel per N (one translation
// unit per group of four so that the groups compile in parallel).
#include "pass.cuh"

namespace debyefit {

void launch_pass_b4(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch (N) {
    case 17: launch_pass_n<17>(phase, a, grid, block, st); break;
    case 18: launch_pass_n<18>(phase, a, grid, block, st); break;
    case 19: launch_pass_n<19>(phase, a, grid, block, st); break;
    default: launch_pass_n<20>(phase, a, grid, block, st); break;
  }
}

}  // namespace debyefit
