// Fused sketched contractions against B colliding sketches (Prop. 1, App. B) and the
// persistent kernel that runs Alg. 1 end to end.
//
// One thread block handles one (vector tau, sketch m) pair entirely on chip (contract_one):
//   1. count sketches of u in shared memory: s_u[h_i] += sigma_i u_i (length b, complex) and
//      s_2[2 h_i mod b] += sigma_i^2 u_i^2.  s_2 is real (sigma^2 = +-1) and supported on even
//      positions only, so it is kept as the length-b/2 vector e[h_i mod b/2];
//      F(s_2)[f] = DFT_{b/2}(e)[f mod b/2];
//   2. forward DFTs: U = F s_u (length b), V' = DFT_{b/2}(e);
//   3. spectral products with FS = F s~_T (read from L2):
//        Y12[f] = FS[f] (conj(U_f)^2 + conj(V'_{f mod b/2}))      -> g_2 + g_1 after F^-1
//        Y0'[f] = FS[f] conj(U_f) + FS[f+b/2] conj(U_{f+b/2})     (f < b/2)
//      Y0' is the spectrum folded to length b/2: its length-b/2 inverse DFT is g_0 at the even
//      positions, the only ones the read-off needs (2 h_i mod b is even);
//   4. inverse DFTs and the hashed read-off of App. B, Eq. 14 (coefficients 1/3,1/6,1/6,1/3):
//        v_i = Re[ 1/6 conj(s_i)(g_2+g_1)[h_i] + 1/3 conj(s_i)^2 u_i g_0[2h_i] + 1/3 conj(s_i)^3 u_i^2 S[3h_i] ]
//   5. lambda^(m) = sum_i u_i v_i (equal to T^(m)(u,u,u), App. B).
// MODE_UUU evaluates T^(m)(u,u,u) directly (App. B, Eq. 13) after step 2:
//   (1/b) sum_f Re(FS[f] conj(U_f^3/6 + V'_f U_f/2)) + 1/3 Re(sum_i S[3h_i] conj(s_i)^3 u_i^3).
// The last block to finish for a vector (arrival counter) takes the median over the B sketches
// (Alg. 1) and, in a power step, normalises it into the next iterate.  Values written by other
// blocks (per-sketch results, iterates) are read with ld.global.cg, never through L1.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "reduce.cuh"

namespace tsk {

enum { MODE_IUU = 0, MODE_UUU = 1 };
constexpr int kMaxB = 64;

struct ContractArgs {
  const float2* FS;      // [B][b] DFT of the sketches
  const float2* S;       // [B][b] time-domain sketches
  const int32_t* h;      // [B][n]
  const uint8_t* g;      // [B][n]
  const float* U;        // [L][n] input vectors
  int n, B, L;
  int normalize_input;   // scale each u by 1/||u|| first
  float* Vall;           // [L][B][n] per-sketch T^(I,u,u)      (MODE_IUU)
  float* lam_all;        // [L][B]    per-sketch T^(u,u,u)
  float* Vmed;           // [L][n]    median over sketches, or NULL
  float* Unext;          // [L][n]    normalised median (power step), or NULL
  float* lam_med;        // [L]       median of lam_all, or NULL
  double* lam_med64;     // [L]       the same median in FP64 (eigenvalue bookkeeping), or NULL
  int fs_class_major;    // split sketches (P > 1): FS stored per class, FS_c[f'] = FS[P f' + c]
  unsigned* counters;    // [L]       arrival counters, zero between launches
  int* status;
};

template <int LOGB>
constexpr size_t contract_smem_bytes() {
  return (size_t)(padded_len(1 << LOGB) + padded_len(1 << (LOGB - 1))) * sizeof(float2) +
         64 * sizeof(float);
}

// ------------------------------------------------------------------ device building blocks

// One (vector, sketch) contraction.  MODE_IUU writes v^(m) to vout[0..n); both modes return
// lambda^(m) = T^(m)(u,u,u) in every thread.  Must be called by all NT threads of the block.
//
// Sketch lengths beyond one block (LOGP > 0, P = 2^LOGP): the block handles the residue class
// `part` of the frequencies, f = P f' + part, with transforms of length M = b / P.  Splitting
// the DFT by f mod P, X[P f' + c] = DFT_M(a_c)[f'] with a_c[p mod M] += x_p w_b^(c p), so each
// count-sketch nonzero is scattered with one twiddle; on the way back the read-off output
// g[t] = (1/b) sum_c w_b^(-c t) G_c[t mod M] is a sum over the P blocks, so each block writes its
// share of v^(m) (the S[3 h_i] term goes with part 0) and the last block adds the P shares.
template <int LOGB, int MODE, int NT = threads_for_logb(LOGB), int LOGP = 0>
__device__ __forceinline__ float contract_one(float2* A, float2* Eb, float* red, const float2* tw,
                                              const float2* FSm, const float2* Sm,
                                              const int32_t* hm, const uint8_t* gm,
                                              const float* u, int n, bool normalize, int* status,
                                              float* vout, int part = 0, int fs_cls = 0) {
  constexpr int b = 1 << LOGB;
  constexpr int hb = b / 2;
  constexpr int LOGM = LOGB - LOGP;
  constexpr int M = 1 << LOGM;
  constexpr int hM = M / 2;
  constexpr int P = 1 << LOGP;
  // spectrum of frequency f of this class: FS[P f + part], or FS_part[f] when class-major
  const int fs_step = fs_cls ? 1 : P;
  const float2* FSc = FSm + (fs_cls ? (size_t)part * M : (size_t)part);
  constexpr float inv_b = 1.f / (float)b;
  const int tid = threadIdx.x;

  float uscale = 1.f;
  if (normalize) {
    float ss = 0.f;
    for (int i = tid; i < n; i += NT) {
      const float x = __ldcg(u + i);
      ss += x * x;
    }
    ss = block_sum<NT>(ss, red);
    if (!(ss > 0.f) || !isfinite(ss)) {
      if (tid == 0) tsk_set_status(status, TSK_ENONFINITE);
      uscale = 0.f;
    } else {
      uscale = 1.f / sqrtf(ss);
    }
  }

  // 1. zero both buffers, then scatter the count sketches of u.
  for (int i = tid; i < padded_len(M); i += NT) A[i] = make_float2(0.f, 0.f);
  for (int i = tid; i < padded_len(hM); i += NT) Eb[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const float x = __ldcg(u + i) * uscale;
    const int hi = hm[i] & (b - 1);
    const int gi = gm[i] & 3;
    if constexpr (LOGP == 0) {
      float* slot = reinterpret_cast<float*>(&A[pad_idx(hi)]);
      atomicAdd(slot + (gi & 1), (gi & 2) ? -x : x);
      atomicAdd(&Eb[pad_idx(hi & (hb - 1))].x, (gi & 1) ? -x * x : x * x);
    } else {
      // twiddles w_b^(part h) for s_u and w_(b/2)^(part (h mod b/2)) = (w_b^(part h))^2 for s_2
      const float2 w1 = unit_root_direct((part * hi) & (b - 1), LOGB, -1);
      const float2 v = cmul(cmul_ipow(make_float2(x, 0.f), gi), w1);
      float* slot = reinterpret_cast<float*>(&A[pad_idx(hi & (M - 1))]);
      atomicAdd(slot, v.x);
      atomicAdd(slot + 1, v.y);
      const float e = (gi & 1) ? -x * x : x * x;
      const float2 w2 = cmul(w1, w1);
      float* es = reinterpret_cast<float*>(&Eb[pad_idx(hi & (hM - 1))]);
      atomicAdd(es, e * w2.x);
      atomicAdd(es + 1, e * w2.y);
    }
  }
  __syncthreads();

  // 2. forward DFTs (the two transforms' passes interleaved).  The loops below touch only each
  // thread's own slots t + NT s (f = tid + NT s), so no barrier is needed after the transforms
  // or between the spectral products and the inverse transforms (slot ownership, fft.cuh).
  block_fft_pair<LOGM, LOGM - 1, NT, -1, false>(A, Eb, tw);

  float lam = 0.f;
  if constexpr (MODE == MODE_IUU) {
    // 3. spectral products (each f < M/2 owns positions f and f + M/2 of A and f of Eb).
    for (int f = tid; f < hM; f += NT) {
      const float2 cu0 = cconj(A[pad_idx(f)]);
      const float2 cu1 = cconj(A[pad_idx(f + hM)]);
      const float2 cv = cconj(Eb[pad_idx(f)]);
      const float2 F0 = __ldcg(FSc + fs_step * f);
      const float2 F1 = __ldcg(FSc + fs_step * (f + hM));
      A[pad_idx(f)] = cmul(F0, cadd(cmul(cu0, cu0), cv));
      A[pad_idx(f + hM)] = cmul(F1, cadd(cmul(cu1, cu1), cv));
      Eb[pad_idx(f)] = cadd(cmul(F0, cu0), cmul(F1, cu1));
    }
    // 4. inverse DFTs and hashed read-off.
    block_fft_pair<LOGM, LOGM - 1, NT, +1>(A, Eb, tw);
    for (int i = tid; i < n; i += NT) {
      const float x = __ldcg(u + i) * uscale;
      const int hi = hm[i] & (b - 1);
      const int gi = gm[i] & 3;
      float2 g12 = A[pad_idx(hi & (M - 1))];
      float2 g0 = Eb[pad_idx(hi & (hM - 1))];
      if constexpr (LOGP > 0) {
        const float2 w1 = unit_root_direct((part * hi) & (b - 1), LOGB, +1);
        g12 = cmul(g12, w1);
        g0 = cmul(g0, cmul(w1, w1));
      }
      float v = (re_ipow(g12, -gi) * (1.f / 6.f) + re_ipow(g0, -2 * gi) * x * (1.f / 3.f)) * inv_b;
      if (LOGP == 0 || part == 0) {
        const float2 s3 = __ldcg(Sm + ((3 * hi) & (b - 1)));
        v += re_ipow(s3, -3 * gi) * x * x * (1.f / 3.f);
      }
      vout[i] = v;
      lam += x * v;
    }
  } else {
    for (int f = tid; f < M; f += NT) {
      const float2 U = A[pad_idx(f)];
      const float2 V = Eb[pad_idx(f & (hM - 1))];
      const float2 U2 = cmul(U, U);
      const float2 Y = cadd(cscale(cmul(U2, U), 1.f / 6.f), cscale(cmul(V, U), 0.5f));
      const float2 F = __ldcg(FSc + fs_step * f);
      lam += F.x * Y.x + F.y * Y.y;     // Re(F conj(Y))
    }
    lam *= inv_b;
    if (LOGP == 0 || part == 0)
    for (int i = tid; i < n; i += NT) {
      const float x = __ldcg(u + i) * uscale;
      const int hi = hm[i] & (b - 1);
      const int gi = gm[i] & 3;
      lam += re_ipow(__ldcg(Sm + ((3 * hi) & (b - 1))), -3 * gi) * x * x * x * (1.f / 3.f);
    }
  }
  return block_sum<NT>(lam, red);
}

// Count this block's arrival on `counter`; true (in every thread) for the block that completes
// a group of `group` arrivals.  Writes of this block are made visible device-wide first.
__device__ __forceinline__ bool arrive_is_last(unsigned* counter, unsigned group, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    *s_flag = (prev == group - 1);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Median over the B sketches of every entry of one vector (Vt: [B][n]) into dst; if unext is
// given, dst / ||dst|| is written there (dst may equal unext).  Called by the last block, with
// `scratch` a shared-memory area of scratch_floats >= B floats that the block no longer needs
// (its FFT buffers): each taking part thread sorts its B values in a column of it (entry c at
// scratch[c * P + t], P threads taking part), not in a per-thread local-memory array, whose
// traffic would go to L2 when shared memory leaves little L1.  Ends synchronised.
//
// With parts > 1 (sketch lengths split over several blocks), Vt is [B][parts][n] and each
// sketch's value is the sum of its parts.
template <int NT>
__device__ __forceinline__ void median_vector(const float* Vt, int B, int n, float* dst,
                                              float* unext, float* red, int* status,
                                              float* scratch, int scratch_floats, int parts = 1) {
  const int P = min(NT, scratch_floats / B);
  const int t = threadIdx.x;
  float ss = 0.f;
  if (t < P) {
    float* x = scratch + t;
    for (int i = t; i < n; i += P) {
      for (int c = 0; c < B; ++c) {
        float v = __ldcg(Vt + (size_t)c * parts * n + i);
        for (int q = 1; q < parts; ++q) v += __ldcg(Vt + ((size_t)c * parts + q) * n + i);
        x[c * P] = v;
      }
      const float med = small_median_strided(x, B, P);
      dst[i] = med;
      ss += med * med;
    }
  }
  if (unext) {
    ss = block_sum<NT>(ss, red);
    float inv = 0.f;
    if (!(ss > 0.f) || !isfinite(ss)) {
      if (t == 0) tsk_set_status(status, TSK_ENONFINITE);
    } else {
      inv = 1.f / sqrtf(ss);
    }
    if (t < P)
      for (int i = t; i < n; i += P) unext[i] = dst[i] * inv;
  }
  __syncthreads();
}

__device__ __forceinline__ float median_of(const float* x, int B, int parts = 1) {
  float vals[kMaxB];
  for (int c = 0; c < B; ++c) {
    float v = __ldcg(x + (size_t)c * parts);
    for (int q = 1; q < parts; ++q) v += __ldcg(x + (size_t)c * parts + q);
    vals[c] = v;
  }
  return small_median(vals, B);
}

// The same median in FP64: the P shares of each sketch's value are summed and the middle values
// averaged in double, so the eigenvalue estimate is not rounded to float again.
__device__ __forceinline__ double median_of64(const float* x, int B, int parts = 1) {
  double vals[kMaxB];
  for (int c = 0; c < B; ++c) {
    double v = (double)__ldcg(x + (size_t)c * parts);
    for (int q = 1; q < parts; ++q) v += (double)__ldcg(x + (size_t)c * parts + q);
    vals[c] = v;
  }
  return small_median(vals, B);
}

// lambda^ D as lambda_hi D + lambda_lo D with lambda = lambda_hi + lambda_lo (two floats, about
// 48 significant bits): the FP64 eigenvalue enters the FP32 sketch update unrounded; the only
// rounding is that of the product.
__device__ __forceinline__ float2 scale_by_double(float2 D, double lam) {
  const float hi = (float)lam;
  const float lo = (float)(lam - (double)hi);
  return make_float2(fmaf(D.x, hi, D.x * lo), fmaf(D.y, hi, D.y * lo));
}

// Deflation of one sketch by lambda^ u(x)u(x)u (Alg. 1, deflation step; Sec. 3.3):
//   U = F s~_u,  D = lambda^ U^3,  FS[m] -= D,  S[m] -= F^-1 D.
template <int LOGB, int NT = threads_for_logb(LOGB)>
__device__ __forceinline__ void deflate_one(float2* A, const float2* tw, float2* FSm, float2* Sm,
                                            const int32_t* hm,
                                            const uint8_t* gm, const float* u, int n, double lam) {
  constexpr int b = 1 << LOGB;
  const int tid = threadIdx.x;
  for (int i = tid; i < padded_len(b); i += NT) A[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const int gi = gm[i] & 3;
    const float x = __ldcg(u + i);
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hm[i] & (b - 1))]);
    atomicAdd(slot + (gi & 1), (gi & 2) ? -x : x);
  }
  __syncthreads();
  block_fft<LOGB, NT, -1>(A, tw);
  for (int f = tid; f < b; f += NT) {
    const float2 U = A[pad_idx(f)];
    const float2 D = scale_by_double(cmul(cmul(U, U), U), lam);
    FSm[f] = csub(__ldcg(FSm + f), D);
    A[pad_idx(f)] = D;
  }
  __syncthreads();
  block_fft<LOGB, NT, +1>(A, tw);
  constexpr float inv_b = 1.f / (float)b;
  for (int t = tid; t < b; t += NT) Sm[t] = csub(__ldcg(Sm + t), cscale(A[pad_idx(t)], inv_b));
  __syncthreads();
}

// Deflation of one frequency class of one sketch when the sketch length is split over P = 2^LOGP
// blocks (see contract_one): U_c = DFT_M of the class's scattered count sketch, D_c = lambda^ U_c^3,
// FS[P f' + part] -= D_c[f'], and the unnormalised inverse G_c = IDFT_M(D_c) is written to Gm; the
// time-domain update S[t] -= (1/b) sum_c w_b^(-c t) G_c[t mod M] needs every class and is applied
// by deflate_combine_kernel afterwards.
template <int LOGB, int LOGP, int NT>
__device__ __forceinline__ void deflate_part(float2* A, const float2* tw, float2* FSm, float2* Gm,
                                             const int32_t* hm, const uint8_t* gm, const float* u,
                                             int n, double lam, int part, int fs_cls) {
  constexpr int b = 1 << LOGB;
  constexpr int LOGM = LOGB - LOGP;
  constexpr int M = 1 << LOGM;
  constexpr int P = 1 << LOGP;
  const int tid = threadIdx.x;
  for (int i = tid; i < padded_len(M); i += NT) A[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const int hi = hm[i] & (b - 1);
    const float2 v = cmul(cmul_ipow(make_float2(__ldcg(u + i), 0.f), gm[i] & 3),
                          unit_root_wide(tw, (part * hi) & (b - 1), b, -1));
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hi & (M - 1))]);
    atomicAdd(slot, v.x);
    atomicAdd(slot + 1, v.y);
  }
  __syncthreads();
  block_fft<LOGM, NT, -1>(A, tw);
  for (int f = tid; f < M; f += NT) {
    const float2 U = A[pad_idx(f)];
    const float2 D = scale_by_double(cmul(cmul(U, U), U), lam);
    const size_t fi = fs_cls ? (size_t)part * M + f : (size_t)P * f + part;
    FSm[fi] = csub(__ldcg(FSm + fi), D);
    A[pad_idx(f)] = D;
  }
  __syncthreads();
  block_fft<LOGM, NT, +1>(A, tw);
  for (int t = tid; t < M; t += NT) Gm[t] = A[pad_idx(t)];
  __syncthreads();
}

// S[m][t] -= (1/b) sum_c w_b^(-c t) G[m][c][t mod M] for the P frequency classes c (the inverse
// DFT of the deflation term, assembled from the classes' length-M inverses).  Grid (chunks, B).
template <int LOGB, int LOGP>
__global__ void __launch_bounds__(256) deflate_combine_kernel(float2* S, const float2* G) {
  constexpr int b = 1 << LOGB;
  constexpr int M = 1 << (LOGB - LOGP);
  constexpr int P = 1 << LOGP;
  constexpr float inv_b = 1.f / (float)b;
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, 256);
  const int m = blockIdx.y;
  const float2* Gm = G + (size_t)m * P * M;
  float2* Sm = S + (size_t)m * b;
  for (int t = blockIdx.x * 256 + threadIdx.x; t < b; t += gridDim.x * 256) {
    float2 acc = __ldcg(Gm + (t & (M - 1)));
    for (int c = 1; c < P; ++c)
      acc = cadd(acc, cmul(__ldcg(Gm + (size_t)c * M + (t & (M - 1))),
                           unit_root_wide(tw, (c * t) & (b - 1), b, +1)));
    Sm[t] = csub(__ldcg(Sm + t), cscale(acc, inv_b));
  }
}

// FS = DFT_b of the sketches S when b is split over P blocks: block (m, c) forms
// a_c[j] = sum_q S[m][j + q M] w_b^(c (j + q M)), j < M, and FS[m][P f' + c] = DFT_M(a_c)[f']
// (or FS[m][c M + f'] when class_major: each class contiguous, read with whole sectors).
template <int LOGB, int LOGP>
__global__ void __launch_bounds__(threads_for_logb(LOGB - LOGP), 1) fft_split_kernel(const float2* S,
                                                                                    float2* FS,
                                                                                    int class_major) {
  constexpr int LOGM = LOGB - LOGP;
  constexpr int NT = threads_for_logb(LOGM);
  constexpr int b = 1 << LOGB;
  constexpr int M = 1 << LOGM;
  constexpr int P = 1 << LOGP;
  extern __shared__ float2 smem[];
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x >> LOGP, c = blockIdx.x & (P - 1);
  const float2* Sm = S + (size_t)m * b;
  for (int j = threadIdx.x; j < M; j += NT) {
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < P; ++q) {
      const int t = j + q * M;
      acc = cadd(acc, cmul(__ldcg(Sm + t), unit_root_wide(tw, (c * t) & (b - 1), b, -1)));
    }
    smem[pad_idx(j)] = acc;
  }
  __syncthreads();
  block_fft<LOGM, NT, -1>(smem, tw);
  float2* FSm = FS + (size_t)m * b;
  for (int f = threadIdx.x; f < M; f += NT)
    FSm[class_major ? (size_t)c * M + f : (size_t)P * f + c] = smem[pad_idx(f)];
}

// First index of the maximum of x[0..L) (the selection tau* of Alg. 1).
template <typename V>
__device__ __forceinline__ int first_argmax(const V* x, int L) {
  int best = 0;
  V bv = __ldcg(x);
  for (int t = 1; t < L; ++t) {
    const V v = __ldcg(x + t);
    if (v > bv) {
      bv = v;
      best = t;
    }
  }
  return best;
}

// ------------------------------------------------------------------ single-step kernels

// Grid (B P, L): block x handles sketch x / P and frequency class x mod P (P = 2^LOGP; Vall and
// lam_all then hold [L][B][P] shares); the last of the B P blocks of a vector takes the medians.
template <int LOGB, int MODE, int LOGP = 0>
__global__ void __launch_bounds__(threads_for_logb(LOGB - LOGP),
                                  contract_min_blocks(LOGB - LOGP, threads_for_logb(LOGB - LOGP)))
    contract_kernel(ContractArgs a) {
  constexpr int LOGM = LOGB - LOGP;
  constexpr int NT = threads_for_logb(LOGM);
  constexpr int b = 1 << LOGB;
  constexpr int M = 1 << LOGM;
  constexpr int P = 1 << LOGP;
  extern __shared__ float2 smem[];
  float2* A = smem;
  float2* Eb = smem + padded_len(M);
  float* red = reinterpret_cast<float*>(Eb + padded_len(M / 2));
  __shared__ int s_last;
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x >> LOGP, part = blockIdx.x & (P - 1);
  const int tau = blockIdx.y, n = a.n, B = a.B;
  const size_t share = ((size_t)tau * B + m) * P + part;
  const float lam = contract_one<LOGB, MODE, NT, LOGP>(
      A, Eb, red, tw, a.FS + (size_t)m * b, a.S + (size_t)m * b, a.h + (size_t)m * n,
      a.g + (size_t)m * n, a.U + (size_t)tau * n, n, a.normalize_input != 0, a.status,
      MODE == MODE_IUU ? a.Vall + share * n : nullptr, part, a.fs_class_major);
  if (threadIdx.x == 0) a.lam_all[share] = lam;
  if (!arrive_is_last(&a.counters[tau], (unsigned)(B * P), &s_last)) return;
  if (threadIdx.x == 0) {
    if (a.lam_med || a.lam_med64) {
      const double med = median_of64(a.lam_all + (size_t)tau * B * P, B, P);
      if (a.lam_med) a.lam_med[tau] = (float)med;
      if (a.lam_med64) a.lam_med64[tau] = med;
    }
    a.counters[tau] = 0u;
  }
  if constexpr (MODE == MODE_IUU) {
    if (a.Vmed == nullptr && a.Unext == nullptr) return;
    float* dst = a.Vmed ? a.Vmed + (size_t)tau * n : a.Unext + (size_t)tau * n;
    median_vector<NT>(a.Vall + (size_t)tau * B * P * n, B, n, dst,
                      a.Unext ? a.Unext + (size_t)tau * n : nullptr, red, a.status,
                      reinterpret_cast<float*>(A), 2 * (padded_len(M) + padded_len(M / 2)), P);
  }
}

// ------------------------------------------------------------------ persistent Alg. 1

// Selection tau* = first argmax of the round's eigenvalue medians, outputs, and deflation of
// sketch m = blockIdx.x (Alg. 1, selection and deflation steps).
struct DeflateArgs {
  float2* FS;
  float2* S;
  const int32_t* h;
  const uint8_t* g;
  int n, L;
  const float* Ufinal;      // [L][n] final iterates of the round
  const double* lam_med;    // [L] eigenvalue medians of the round (FP64)
  int round;
  double* lambda_out;       // [k]
  float* Vout;              // [k][n]
  int32_t* tau_out;         // [k] or NULL
  float2* G;                // [B][P][b/P] workspace when the sketch length is split (P > 1)
  int fs_class_major;       // FS stored per frequency class (see ContractArgs)
};

template <int LOGB, int LOGP = 0>
__global__ void __launch_bounds__(threads_for_logb(LOGB - LOGP), 1) deflate_kernel(DeflateArgs a) {
  constexpr int LOGM = LOGB - LOGP;
  constexpr int NT = threads_for_logb(LOGM);
  constexpr int b = 1 << LOGB;
  constexpr int P = 1 << LOGP;
  extern __shared__ float2 smem[];
  __shared__ int s_best;
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x >> LOGP, part = blockIdx.x & (P - 1), n = a.n;
  if (threadIdx.x == 0) s_best = first_argmax(a.lam_med, a.L);
  __syncthreads();
  const int best = s_best;
  const double lam = a.lam_med[best];
  const float* u = a.Ufinal + (size_t)best * n;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      a.lambda_out[a.round] = lam;
      if (a.tau_out) a.tau_out[a.round] = best;
    }
    for (int i = threadIdx.x; i < n; i += NT) a.Vout[(size_t)a.round * n + i] = u[i];
  }
  if constexpr (LOGP == 0) {
    deflate_one<LOGB>(smem, tw, a.FS + (size_t)m * b, a.S + (size_t)m * b, a.h + (size_t)m * n,
                      a.g + (size_t)m * n, u, n, lam);
  } else {
    deflate_part<LOGB, LOGP, NT>(smem, tw, a.FS + (size_t)m * b,
                                 a.G + ((size_t)m * P + part) * (b / P), a.h + (size_t)m * n,
                                 a.g + (size_t)m * n, u, n, lam, part, a.fs_class_major);
  }
}

// Host launchers (defined in contract.cu).
// logp: the sketch's frequencies are split over 2^logp blocks per (vector, sketch); the blocks'
// transforms (length b / 2^logp) must be 2^13 or 2^14 when logp > 0.
int launch_contract(int log2b, int logp, int mode, const ContractArgs& args, cudaStream_t st);
int launch_deflate(int log2b, int logp, const DeflateArgs& args, int B, cudaStream_t st);
int launch_fft_split(int log2b, int logp, const float2* S, float2* FS, int B, cudaStream_t st,
                     int class_major = 0);

}  // namespace tsk
