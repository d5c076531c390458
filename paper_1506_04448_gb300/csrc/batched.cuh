// Many independent decompositions (Alg. 1) of uneven size in one enqueued sequence.
//
// Problems are grouped by sketch length b.  Within a group every power step of every active
// problem is one launch of B x L x P blocks (one block per (sketch, vector, problem)); problems
// are sorted by decreasing rank k so that the problems still active in round r are a prefix.
// Groups run on separate streams forked from and joined into the caller's stream, so a plan's
// run is a pure launch sequence that can be captured into one CUDA graph.  The block size of
// each group's contraction kernel (elements per thread, i.e. the FFT tile) is picked by timing
// the candidates on the group's own data when the plan is created.
#pragma once

#include "contract.cuh"

namespace tsk {

struct BatchProblem {            // device-side descriptor of one problem
  float2* FS;                    // [B][b] DFT of the sketches (workspace copy)
  float2* S;                     // [B][b] time-domain sketches (workspace copy, deflated)
  const int32_t* h;              // [B][n]
  const uint8_t* g;              // [B][n]
  const float* U0;               // [k][L][n]
  float* Vall;                   // [L][B][n]
  float* lam_all;                // [L][B]
  float* Ubuf;                   // [2][L][n]
  float* lam_med;                // [k][L] (caller's trace or workspace)
  double* lam_med64;             // [k][L] the same medians in FP64 (selection, deflation)
  unsigned* counters;            // [L]
  double* lambda;                // [k]
  float* V;                      // [k][n]
  int32_t* tau;                  // [k] or NULL
  float* U_iters;                // [k][T][L][n] or NULL
  int n, k;
};

// Power step t (MODE_IUU) or selection (MODE_UUU) of round r; grid (B, L, active problems).
template <int LOGB, int MODE, int NT>
__global__ void __launch_bounds__(NT, contract_min_blocks(LOGB, NT))
    batch_contract_kernel(const BatchProblem* probs, int B,
                                                               int L, int T, int t, int r,
                                                               int* status) {
  constexpr int b = 1 << LOGB;
  extern __shared__ float2 smem[];
  float2* A = smem;
  float2* Eb = smem + padded_len(b);
  float* red = reinterpret_cast<float*>(Eb + padded_len(b / 2));
  __shared__ float2 tw[kTwEntries];
  __shared__ int s_last;
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, tau = blockIdx.y;
  const BatchProblem& P = probs[blockIdx.z];
  const int n = P.n;
  const float* u;
  if constexpr (MODE == MODE_IUU)
    u = t == 0 ? P.U0 + ((size_t)r * L + tau) * n : P.Ubuf + ((size_t)(t & 1) * L + tau) * n;
  else
    u = P.Ubuf + ((size_t)(T & 1) * L + tau) * n;   // u_T of round r
  const float lam = contract_one<LOGB, MODE, NT>(
      A, Eb, red, tw, P.FS + (size_t)m * b, P.S + (size_t)m * b, P.h + (size_t)m * n,
      P.g + (size_t)m * n, u, n, MODE == MODE_IUU && t == 0, status,
      MODE == MODE_IUU ? P.Vall + ((size_t)tau * B + m) * n : nullptr);
  if (threadIdx.x == 0) P.lam_all[(size_t)tau * B + m] = lam;
  if (!arrive_is_last(&P.counters[tau], (unsigned)B, &s_last)) return;
  if constexpr (MODE == MODE_IUU) {
    float* un = P.Ubuf + ((size_t)((t + 1) & 1) * L + tau) * n;
    median_vector<NT>(P.Vall + (size_t)tau * B * n, B, n, un, un, red, status,
                      reinterpret_cast<float*>(A), 2 * (padded_len(b) + padded_len(b / 2)));
    if (P.U_iters) {
      float* tr = P.U_iters + (((size_t)r * T + t) * L + tau) * n;
      for (int i = threadIdx.x; i < n; i += NT) tr[i] = un[i];
    }
  } else {
    if (threadIdx.x == 0) {
      const double med = median_of64(P.lam_all + (size_t)tau * B, B);
      P.lam_med[(size_t)r * L + tau] = (float)med;
      P.lam_med64[(size_t)r * L + tau] = med;
    }
  }
  if (threadIdx.x == 0) P.counters[tau] = 0u;
}

// Selection and deflation of round r; grid (B, active problems).
template <int LOGB, int NT>
__global__ void __launch_bounds__(NT, 1) batch_deflate_kernel(const BatchProblem* probs, int B,
                                                              int L, int T, int r) {
  constexpr int b = 1 << LOGB;
  extern __shared__ float2 smem[];
  __shared__ float2 tw[kTwEntries];
  __shared__ int s_best;
  fill_twiddles(tw, NT);
  const int m = blockIdx.x;
  const BatchProblem& P = probs[blockIdx.y];
  const int n = P.n;
  const double* lam_r = P.lam_med64 + (size_t)r * L;
  if (threadIdx.x == 0) s_best = first_argmax(lam_r, L);
  __syncthreads();
  const int best = s_best;
  const double lam = __ldcg(lam_r + best);
  const float* u = P.Ubuf + ((size_t)(T & 1) * L + best) * n;
  if (m == 0) {
    if (threadIdx.x == 0) {
      P.lambda[r] = lam;
      if (P.tau) P.tau[r] = best;
    }
    for (int i = threadIdx.x; i < n; i += NT) P.V[(size_t)r * n + i] = __ldcg(u + i);
  }
  deflate_one<LOGB, NT>(smem, tw, P.FS + (size_t)m * b, P.S + (size_t)m * b, P.h + (size_t)m * n,
                        P.g + (size_t)m * n, u, n, lam);
}

// Host side, one definition per translation unit that instantiates a range of sketch lengths:
// launch the kernel compiled for (log2b, nt); TSK_EUNSUPPORTED if that pair is not compiled there.
int batch_launch_lo(int log2b, int nt, int kind, const BatchProblem* probs, int B, int L, int T,
                    int t, int r, int nprob, int* status, cudaStream_t st);
int batch_launch_hi(int log2b, int nt, int kind, const BatchProblem* probs, int B, int L, int T,
                    int t, int r, int nprob, int* status, cudaStream_t st);
enum { BATCH_STEP = 0, BATCH_SELECT = 1, BATCH_DEFLATE = 2 };

template <int LOGB, int NT>
int batch_launch_t(int kind, const BatchProblem* probs, int B, int L, int T, int t, int r,
                   int nprob, int* status, cudaStream_t st) {
  if (kind == BATCH_DEFLATE) {
    constexpr size_t smem = (size_t)padded_len(1 << LOGB) * sizeof(float2);
    TSK_CUDA(tsk_smem_attr<batch_deflate_kernel<LOGB, NT>>(smem));
    batch_deflate_kernel<LOGB, NT><<<dim3(B, nprob), NT, smem, st>>>(probs, B, L, T, r);
    TSK_CHECK_LAUNCH();
    return TSK_OK;
  }
  constexpr size_t smem = contract_smem_bytes<LOGB>();
  if (kind == BATCH_STEP) {
    TSK_CUDA(tsk_smem_attr<batch_contract_kernel<LOGB, MODE_IUU, NT>>(smem));
    batch_contract_kernel<LOGB, MODE_IUU, NT><<<dim3(B, L, nprob), NT, smem, st>>>(probs, B, L, T, t, r, status);
  } else {
    TSK_CUDA(tsk_smem_attr<batch_contract_kernel<LOGB, MODE_UUU, NT>>(smem));
    batch_contract_kernel<LOGB, MODE_UUU, NT><<<dim3(B, L, nprob), NT, smem, st>>>(probs, B, L, T, t, r, status);
  }
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

}  // namespace tsk
