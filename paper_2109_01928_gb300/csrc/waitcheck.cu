// Check of the bounded waits (debye_check_bounded_wait): the staging wait of the
// column-sum pass, run on a buffer whose mbarrier no copy will ever complete. The wait
// gives up after its clock budget (STAGE_WAIT_CYCLES, about 1 s), the block agrees on
// it, records DEBYE_ETIMEOUT in the status word and leaves the kernel: the context
// stays usable and the host reads the status at the next debye_sync.
#include "eval.cuh"
#include "launch.h"

namespace debyefit {

__global__ void k_stage_wait_check(EvalArgs a, int* waited_ok) {
  __shared__ __align__(128) float4 stage_buf[4 * STAGE_SAMPLES];
  __shared__ __align__(8) uint64_t stage_bar[2];
  Stage st;
  stage_init(st, stage_buf, stage_bar);
  // no stage_issue: nothing arrives at buffer 0's mbarrier, and no copy is in flight
  const bool ok = stage_wait(a, st, 0);
  if (threadIdx.x == 0 && waited_ok) *waited_ok = ok ? 1 : 0;
}

void launch_stage_wait_check(int* status, int* waited_ok, cudaStream_t st) {
  EvalArgs a{};
  a.status = status;
  k_stage_wait_check<<<1, 64, 0, st>>>(a, waited_ok);
}

}  // namespace debyefit
