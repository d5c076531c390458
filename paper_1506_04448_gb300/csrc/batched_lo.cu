// Batched Alg. 1 kernels for sketch lengths 2^10 .. 2^12 (block sizes b/16 and b/32).
#include "batched.cuh"

namespace tsk {

int batch_launch_lo(int log2b, int nt, int kind, const BatchProblem* probs, int B, int L, int T,
                    int t, int r, int nprob, int* status, cudaStream_t st) {
#define TSK_CASE(LB, NTV) \
  if (log2b == LB && nt == NTV) return batch_launch_t<LB, NTV>(kind, probs, B, L, T, t, r, nprob, status, st);
  TSK_CASE(10, 64) TSK_CASE(10, 32)
  TSK_CASE(11, 128) TSK_CASE(11, 64)
  TSK_CASE(12, 256) TSK_CASE(12, 128)
#undef TSK_CASE
  return TSK_EUNSUPPORTED;
}

}  // namespace tsk
