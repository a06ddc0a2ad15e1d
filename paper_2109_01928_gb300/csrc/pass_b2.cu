// Pass kernels for pole counts N = 9..12, one kernel per N (one translation
// unit per group of four so that the groups compile in parallel).
#include "pass.cuh"

namespace debyefit {

void launch_pass_b2(int N, int phase, const EvalArgs& a, int grid, int block, cudaStream_t st) {
  switch (N) {
    case 9: launch_pass_n<9>(phase, a, grid, block, st); break;
    case 10: launch_pass_n<10>(phase, a, grid, block, st); break;
    case 11: launch_pass_n<11>(phase, a, grid, block, st); break;
    default: launch_pass_n<12>(phase, a, grid, block, st); break;
  }
}

}  // namespace debyefit
