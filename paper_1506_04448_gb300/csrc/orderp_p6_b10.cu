// Order-6 instance of the order-p contraction and deflation kernels for sketch length 2^10
// (orderp.cuh; one translation unit per sketch length keeps each compile short).
#include "orderp.cuh"

namespace tsk {

template int launch_contract_p_t<10, 6>(const PArgs&, int, cudaStream_t);
template int launch_deflate_p_t<10, 6>(float2*, float2*, const int32_t*, const uint8_t*, int, int,
                                        const float*, const float*, int, double*, float*, int32_t*,
                                        int, cudaStream_t);

}  // namespace tsk
