// Order-p symmetric (colliding) tensor sketches, p = 3..6: the extension of Sec. 3.3 to tensors
// of order p, their sketched contractions and Alg. 1 for order p.
//
// Sketch (Eq. 7 with p indices): s~_T(t) = sum over ordered p-tuples with
// (h(i_1) + ... + h(i_p)) mod b = t of T_{i_1..i_p} sigma(i_1)...sigma(i_p), sigma uniform on the
// m-th roots of unity (m = 4 for p = 3, 8 for p = 4..6, so E[sigma^k] = 0 for 0 < |k| <= p).
//
// Contractions.  The colliding sketch counts each multiset of indices once per ordering, so the
// estimate of T(u,...,u) pairs S with the sketch of the complete homogeneous polynomial h_p in
// the variables sigma(i) u_i x^{h(i)}.  Written in power sums, h_p = sum over the partitions
// lambda of p of p_lambda / z_lambda (z_lambda = prod_k k^{m_k} m_k!), and the power sum p_k is
// the count sketch s_k[(k h(i)) mod b] += sigma(i)^k u_i^k:
//   T^(u,...,u)   = (1/b) sum_f Re(FS_f conj(Y_f)) + (1/p) sum_i Re(S[p h_i] conj(sigma_i)^p) u_i^p,
//                   Y = sum_{lambda != (p)} (1/z_lambda) prod_{parts j} F(s_{lambda_j});
//   T^(I,u,...,u)_i = (1/p) Re[ sum_{k<p} k conj(sigma_i)^k u_i^(k-1) G_k[k h_i] / b
//                               + conj(sigma_i)^p u_i^(p-1) S[p h_i] ],
//                   G_k = F^-1-unnormalised(FS conj(F R_k)), F R_k = sum over lambda containing k of
//                   (m_k(lambda) / z_lambda) prod over lambda's other parts of F(s_part).
// At p = 3 these are App. B's Eq. 13 and Eq. 14 (coefficients 1/6, 1/6, 1/3, 1/3).  The
// partitions are enumerated at compile time (compile_terms).
//
// s_k for even k lives on even positions only, so it is transformed at length b/2 and its
// spectral product folded to b/2 before the inverse (xlen, power_sum_ffts).
//
// Deflation: the sketch of u^{(x)p} is the p-fold convolution of s_1, so FS -= lambda (F s_1)^p
// and S -= F^-1 of the same.
//
// This header holds the contraction and deflation kernels and their launch templates;
// orderp_p3.cu .. orderp_p6.cu instantiate one order each (compiled in parallel), orderp.cu holds
// the builds and the C entry points.
#pragma once

#include "contract.cuh"
#include "partitions.h"

namespace tsk {

// exp(2 pi i j / m) for m in {4, 8} (the sign roots), j taken mod m.
__device__ __forceinline__ float2 root_of_unity(int j, int m) {
  const int e = (m == 4 ? 2 * j : j) & 7;   // as an 8th root
  switch (e) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(TSK_R2, TSK_R2);
    case 2: return make_float2(0.f, 1.f);
    case 3: return make_float2(-TSK_R2, TSK_R2);
    case 4: return make_float2(-1.f, 0.f);
    case 5: return make_float2(-TSK_R2, -TSK_R2);
    case 6: return make_float2(0.f, -1.f);
    default: return make_float2(TSK_R2, -TSK_R2);
  }
}

// ------------------------------------------------------------------ contraction
struct PArgs {
  const float2* FS;      // [B][b]
  const float2* S;       // [B][b]
  const int32_t* h;      // [B][n]
  const uint8_t* g;      // [B][n]
  const float* U;        // [L][n]
  int n, B, normalize_input;
  float* Vall;           // [L][B][n]
  float* lam_all;        // [L][B]
  int* status;
  unsigned* counters;    // [L] arrival counters (zero between launches), or NULL: no medians
  float* Vmed;           // [L][n] median over the sketches, or NULL
  float* Unext;          // [L][n] normalised median, or NULL
  float* lam_med;        // [L] median of lam_all, or NULL
};

// Shared-memory layout of the power-sum sketches: s_k for odd k has length b; for even k it lives
// on even positions only (k h mod b is even), so it is kept at half length, e[(k/2) h mod b/2],
// with F s_k[f] = DFT_{b/2}(e)[f mod b/2]; its inverse is read only at even positions too, so the
// spectrum is folded to b/2 before it (as for the length-b/2 sketch of the order-3 kernels).
template <int LOGB>
constexpr int xlen(int k) {
  return (k & 1) ? padded_len(1 << LOGB) : padded_len(1 << (LOGB - 1));
}
template <int LOGB>
constexpr int xoff(int k) {      // offset of s_k (k >= 1); xoff(p) is the total
  int o = 0;
  for (int j = 1; j < k; ++j) o += xlen<LOGB>(j);
  return o;
}
template <int LOGB>
constexpr size_t contract_p_smem(int p) {
  return (size_t)xoff<LOGB>(p) * sizeof(float2) + 64 * sizeof(float);
}
// Two resident blocks per SM where their shared memory fits (p <= 5 at b = 2^12), else one.
template <int LOGB, int P>
constexpr int contract_p_min_blocks() {
  return 2 * (contract_p_smem<LOGB>(P) + 3 * 1024) <= 227 * 1024 ? 2 : 1;
}

// The P-1 transforms of one direction: each odd k (length b) interleaved with the even k + 1
// (length b/2) by block_fft_pair; a last odd k alone.
template <int LOGB, int NT, int P, int DIR>
__device__ __forceinline__ void power_sum_ffts(float2* X, const float2* tw) {
#pragma unroll
  for (int k = 1; k + 1 < P; k += 2)
    block_fft_pair<LOGB, LOGB - 1, NT, DIR>(X + xoff<LOGB>(k), X + xoff<LOGB>(k + 1), tw);
  if constexpr ((P - 1) % 2 == 1) block_fft<LOGB, NT, DIR>(X + xoff<LOGB>(P - 1), tw);
}

// Grid (B, L): block (m, tau) computes T^(m)(I,u_tau,...,u_tau) into Vall[tau][m] and
// T^(m)(u_tau,...,u_tau) into lam_all[tau][m] (formulas at the top of this file).
template <int LOGB, int P>
__global__ void __launch_bounds__(threads_for_logb(LOGB), (contract_p_min_blocks<LOGB, P>()))
    contract_p_kernel(PArgs a) {
  constexpr int b = 1 << LOGB;
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int m_roots = P < 4 ? 4 : 8;
  constexpr float inv_b = 1.f / (float)b;
  constexpr int hb = b / 2;
  extern __shared__ float2 smem[];
  float* red = reinterpret_cast<float*>(smem + xoff<LOGB>(P));
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, tau = blockIdx.y, n = a.n, tid = threadIdx.x;
  const float* u = a.U + (size_t)tau * n;
  const int32_t* hm = a.h + (size_t)m * n;
  const uint8_t* gm = a.g + (size_t)m * n;
  const float2* FSm = a.FS + (size_t)m * b;
  const float2* Sm = a.S + (size_t)m * b;

  float uscale = 1.f;
  if (a.normalize_input) {
    float ss = 0.f;
    for (int i = tid; i < n; i += NT) {
      const float x = __ldcg(u + i);
      ss += x * x;
    }
    ss = block_sum<NT>(ss, red);
    if (!(ss > 0.f) || !isfinite(ss)) {
      if (tid == 0) tsk_set_status(a.status, TSK_ENONFINITE);
      uscale = 0.f;
    } else {
      uscale = 1.f / sqrtf(ss);
    }
  }
  // power-sum sketches s_k, k = 1..P-1 (even k at half length)
  for (int i = tid; i < xoff<LOGB>(P); i += NT) smem[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const float x = __ldcg(u + i) * uscale;
    const int hi = hm[i] & (b - 1), gi = gm[i] & (m_roots - 1);
    float xk = 1.f;
#pragma unroll
    for (int k = 1; k < P; ++k) {
      xk *= x;
      const float2 v = cscale(root_of_unity(k * gi, m_roots), xk);
      const int pos = (k & 1) ? (k * hi) & (b - 1) : ((k / 2) * hi) & (hb - 1);
      float* slot = reinterpret_cast<float*>(&smem[xoff<LOGB>(k) + pad_idx(pos)]);
      atomicAdd(slot, v.x);
      atomicAdd(slot + 1, v.y);
    }
  }
  __syncthreads();
  power_sum_ffts<LOGB, NT, P, -1>(smem, tw);

  // per frequency pair (f, f + b/2): Y for the eigenvalue, then X_k <- FS conj(F R_k), the even
  // k folded to length b/2
  float lam = 0.f;
  for (int f0 = tid; f0 < hb; f0 += NT) {
    float2 U[P];
    U[0] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 2; k < P; k += 2) U[k] = smem[xoff<LOGB>(k) + pad_idx(f0)];
    float2 Wfold[P];
#pragma unroll
    for (int k = 0; k < P; ++k) Wfold[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int f = f0 + half * hb;
#pragma unroll
      for (int k = 1; k < P; k += 2) U[k] = smem[xoff<LOGB>(k) + pad_idx(f)];
      float2 Y = make_float2(0.f, 0.f);
      float2 R[P];
#pragma unroll
      for (int k = 0; k < P; ++k) R[k] = make_float2(0.f, 0.f);
      constexpr CTerms<P> tt = TermTable<P>::value;
#pragma unroll
      for (int q = 0; q < tt.count; ++q) {
        float2 prod = U[tt.parts[q][0]];
#pragma unroll
        for (int j = 1; j < tt.nparts[q]; ++j) prod = cmul(prod, U[tt.parts[q][j]]);
        prod = cscale(prod, tt.coef[q]);
        if (tt.target[q] == 0) Y = cadd(Y, prod);
        else R[tt.target[q]] = cadd(R[tt.target[q]], prod);
      }
      const float2 F = __ldcg(FSm + f);
      lam += F.x * Y.x + F.y * Y.y;               // Re(F conj(Y))
#pragma unroll
      for (int k = 1; k < P; ++k) {
        const float2 W = cmulconj(F, R[k]);
        if (k & 1) smem[xoff<LOGB>(k) + pad_idx(f)] = W;
        else Wfold[k] = cadd(Wfold[k], W);
      }
    }
#pragma unroll
    for (int k = 2; k < P; k += 2) smem[xoff<LOGB>(k) + pad_idx(f0)] = Wfold[k];
  }
  lam *= inv_b;
  __syncthreads();
  power_sum_ffts<LOGB, NT, P, +1>(smem, tw);

  // hashed read-off
  float* vout = a.Vall + ((size_t)tau * a.B + m) * n;
  for (int i = tid; i < n; i += NT) {
    const float x = __ldcg(u + i) * uscale;
    const int hi = hm[i] & (b - 1), gi = gm[i] & (m_roots - 1);
    float v = 0.f, xk = 1.f;                      // xk = x^(k-1)
#pragma unroll
    for (int k = 1; k < P; ++k) {
      const int pos = (k & 1) ? (k * hi) & (b - 1) : ((k / 2) * hi) & (hb - 1);
      const float2 G = smem[xoff<LOGB>(k) + pad_idx(pos)];
      const float2 c = root_of_unity(-k * gi, m_roots);            // conj(sigma)^k
      v += (float)k * (c.x * G.x - c.y * G.y) * xk * inv_b;
      xk *= x;
    }
    const float2 sp = __ldcg(Sm + ((P * hi) & (b - 1)));
    const float2 cp = root_of_unity(-P * gi, m_roots);
    const float re = cp.x * sp.x - cp.y * sp.y;   // Re(S[p h] conj(sigma)^p)
    v += re * xk;                                  // xk = x^(p-1)
    v *= 1.f / (float)P;
    vout[i] = v;
    lam += re * xk * x * (1.f / (float)P);
  }
  lam = block_sum<NT>(lam, red);
  if (tid == 0) a.lam_all[(size_t)tau * a.B + m] = lam;
  // the last of the vector's B blocks takes the medians (Alg. 1), in the now free buffers
  if (a.counters == nullptr) return;
  __shared__ int s_last;
  if (!arrive_is_last(&a.counters[tau], (unsigned)a.B, &s_last)) return;
  if (tid == 0) {
    if (a.lam_med) a.lam_med[tau] = median_of(a.lam_all + (size_t)tau * a.B, a.B);
    a.counters[tau] = 0u;
  }
  if (a.Vmed == nullptr && a.Unext == nullptr) return;
  float* dst = a.Vmed ? a.Vmed + (size_t)tau * n : a.Unext + (size_t)tau * n;
  median_vector<NT>(a.Vall + (size_t)tau * a.B * n, a.B, n, dst,
                    a.Unext ? a.Unext + (size_t)tau * n : nullptr, red, a.status,
                    reinterpret_cast<float*>(smem), 2 * xoff<LOGB>(P));
}

// Selection and deflation for order P: tau* = first argmax of lam_med, outputs, and per sketch m
// FS -= lam (F s_1(u))^P, S -= F^-1(same) / b.
template <int LOGB, int P>
__global__ void __launch_bounds__(threads_for_logb(LOGB), 1) deflate_p_kernel(
    float2* FS, float2* S, const int32_t* h, const uint8_t* g, int n, int L, const float* Ufinal,
    const float* lam_med, int round, double* lambda_out, float* Vout, int32_t* tau_out) {
  constexpr int b = 1 << LOGB;
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int m_roots = P < 4 ? 4 : 8;
  extern __shared__ float2 A[];
  __shared__ float2 tw[kTwEntries];
  __shared__ int s_best;
  fill_twiddles(tw, NT);
  const int m = blockIdx.x;
  if (threadIdx.x == 0) s_best = first_argmax(lam_med, L);
  __syncthreads();
  const int best = s_best;
  const float lam = lam_med[best];
  const float* u = Ufinal + (size_t)best * n;
  if (m == 0) {
    if (threadIdx.x == 0) {
      lambda_out[round] = (double)lam;
      if (tau_out) tau_out[round] = best;
    }
    for (int i = threadIdx.x; i < n; i += NT) Vout[(size_t)round * n + i] = u[i];
  }
  for (int i = threadIdx.x; i < padded_len(b); i += NT) A[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int32_t* hm = h + (size_t)m * n;
  const uint8_t* gm = g + (size_t)m * n;
  for (int i = threadIdx.x; i < n; i += NT) {
    const float2 v = cscale(root_of_unity(gm[i] & (m_roots - 1), m_roots), __ldcg(u + i));
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hm[i] & (b - 1))]);
    atomicAdd(slot, v.x);
    atomicAdd(slot + 1, v.y);
  }
  __syncthreads();
  block_fft<LOGB, NT, -1>(A, tw);
  float2* FSm = FS + (size_t)m * b;
  for (int f = threadIdx.x; f < b; f += NT) {
    const float2 X = A[pad_idx(f)];
    float2 D = X;
#pragma unroll
    for (int k = 1; k < P; ++k) D = cmul(D, X);
    D = cscale(D, lam);
    FSm[f] = csub(__ldcg(FSm + f), D);
    A[pad_idx(f)] = D;
  }
  __syncthreads();
  block_fft<LOGB, NT, +1>(A, tw);
  float2* Sm = S + (size_t)m * b;
  constexpr float inv_b = 1.f / (float)b;
  for (int t = threadIdx.x; t < b; t += NT) Sm[t] = csub(__ldcg(Sm + t), cscale(A[pad_idx(t)], inv_b));
}

template <int LOGB, int P>
int launch_contract_p_t(const PArgs& a, int L, cudaStream_t st) {
  constexpr size_t smem = contract_p_smem<LOGB>(P);
  static_assert(contract_p_smem<LOGB>(P) <= 227 * 1024, "transform buffers exceed shared memory");
  TSK_CUDA(tsk_smem_attr<contract_p_kernel<LOGB, P>>(smem));
  contract_p_kernel<LOGB, P><<<dim3(a.B, L), threads_for_logb(LOGB), smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <int LOGB, int P>
int launch_deflate_p_t(float2* FS, float2* S, const int32_t* h, const uint8_t* g, int n,
                              int L, const float* Ufinal, const float* lam_med, int round,
                              double* lambda_out, float* Vout, int32_t* tau_out, int B,
                              cudaStream_t st) {
  constexpr size_t smem = (size_t)padded_len(1 << LOGB) * sizeof(float2);
  TSK_CUDA(tsk_smem_attr<deflate_p_kernel<LOGB, P>>(smem));
  deflate_p_kernel<LOGB, P><<<B, threads_for_logb(LOGB), smem, st>>>(
      FS, S, h, g, n, L, Ufinal, lam_med, round, lambda_out, Vout, tau_out);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

// All sketch lengths of one order (the translation unit of that order instantiates them).
template <int P>
int launch_contract_p_order(int log2b, const PArgs& a, int L, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_contract_p_t<8, P>(a, L, st);
    case 9: return launch_contract_p_t<9, P>(a, L, st);
    case 10: return launch_contract_p_t<10, P>(a, L, st);
    case 11: return launch_contract_p_t<11, P>(a, L, st);
    case 12: return launch_contract_p_t<12, P>(a, L, st);
    default: return TSK_EUNSUPPORTED;
  }
}

template <int P>
int launch_deflate_p_order(int log2b, float2* FS, float2* S, const int32_t* h, const uint8_t* g,
                           int n, int L, const float* Uf, const float* lm, int r, double* lo,
                           float* Vo, int32_t* to, int B, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_deflate_p_t<8, P>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 9: return launch_deflate_p_t<9, P>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 10: return launch_deflate_p_t<10, P>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 11: return launch_deflate_p_t<11, P>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 12: return launch_deflate_p_t<12, P>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

// Order 6 is instantiated one sketch length per translation unit (orderp_p6_b<LOGB>.cu); its
// dispatcher (orderp_p6.cu) only refers to those instances.
#define TSK_ORDERP_EXTERN(LOGB)                                                                 \
  extern template int launch_contract_p_t<LOGB, 6>(const PArgs&, int, cudaStream_t);           \
  extern template int launch_deflate_p_t<LOGB, 6>(float2*, float2*, const int32_t*,             \
                                                  const uint8_t*, int, int, const float*,       \
                                                  const float*, int, double*, float*, int32_t*, \
                                                  int, cudaStream_t);
TSK_ORDERP_EXTERN(8)
TSK_ORDERP_EXTERN(9)
TSK_ORDERP_EXTERN(10)
TSK_ORDERP_EXTERN(11)
TSK_ORDERP_EXTERN(12)
#undef TSK_ORDERP_EXTERN

// Defined in orderp_p<P>.cu.
#define TSK_ORDERP_DECL(P)                                                                      \
  int launch_contract_p##P(int log2b, const PArgs& a, int L, cudaStream_t st);                   \
  int launch_deflate_p##P(int log2b, float2* FS, float2* S, const int32_t* h, const uint8_t* g,  \
                          int n, int L, const float* Uf, const float* lm, int r, double* lo,     \
                          float* Vo, int32_t* to, int B, cudaStream_t st);
TSK_ORDERP_DECL(3)
TSK_ORDERP_DECL(4)
TSK_ORDERP_DECL(5)
TSK_ORDERP_DECL(6)
#undef TSK_ORDERP_DECL

}  // namespace tsk
