// Batched Alg. 1 kernels for sketch lengths 2^13 and 2^14 (block sizes b/16 and, at 2^13, b/32).
#include "batched.cuh"

namespace tsk {

int batch_launch_hi(int log2b, int nt, int kind, const BatchProblem* probs, int B, int L, int T,
                    int t, int r, int nprob, int* status, cudaStream_t st) {
#define TSK_CASE(LB, NTV) \
  if (log2b == LB && nt == NTV) return batch_launch_t<LB, NTV>(kind, probs, B, L, T, t, r, nprob, status, st);
  TSK_CASE(13, 512) TSK_CASE(13, 256)
  TSK_CASE(14, 1024)
#undef TSK_CASE
  return TSK_EUNSUPPORTED;
}

}  // namespace tsk
