// Tensor-core accumulation of the whitened third moment's document term (moments_tc.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace tsk {

struct Moments3TcArgs {
  const float* P;       // [D][kp] whitened documents p_d = W^T n_d
  const float* mdoc;    // [D] document lengths m_d
  long long D;
  int k, kp;            // topics, row stride of P (multiple of 8)
  int N;                // MMA columns: k rounded up to 16, at most 128
  long long npairs;     // k (k + 1) / 2 pairs a <= b, pair p = b (b + 1) / 2 + a
  long long rows_pad;   // npairs rounded up to 128
  double* part;         // [splits][rows_pad][N]: sum_d w_d p_da p_db p_dc per split
  int* status;          // TSK_ETIMEOUT if an MMA completion never arrived
};

constexpr int kMoments3TcMaxN = 128;

size_t moments3_tc_smem(int N, int kp);
int moments3_tc_splits(int npairs, int num_sms, long long D);
int launch_moments3_tc(const Moments3TcArgs& a, int splits, cudaStream_t st);

}  // namespace tsk
