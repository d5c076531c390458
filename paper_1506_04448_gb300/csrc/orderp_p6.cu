// Order-6 instances of the order-p contraction and deflation kernels (orderp.cuh).
#include "orderp.cuh"

namespace tsk {

int launch_contract_p6(int log2b, const PArgs& a, int L, cudaStream_t st) {
  return launch_contract_p_order<6>(log2b, a, L, st);
}

int launch_deflate_p6(int log2b, float2* FS, float2* S, const int32_t* h, const uint8_t* g,
                      int n, int L, const float* Uf, const float* lm, int r, double* lo, float* Vo,
                      int32_t* to, int B, cudaStream_t st) {
  return launch_deflate_p_order<6>(log2b, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
}

}  // namespace tsk
