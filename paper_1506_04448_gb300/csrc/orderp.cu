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
#include <stdio.h>

#include "contract.cuh"
#include "partitions.h"

namespace tsk {

// dynamic shared memory of sketch_p_kernel: the b <= 2^14 histogram and two n <= 8192 tables
constexpr size_t kSketchPSmemMax = ((size_t)1 << 14) * sizeof(float2) + 2 * (size_t)8192 * sizeof(int);

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

// ------------------------------------------------------------------ build
// Grid (blocks, B); block 256 threads.  Each warp takes rows r = (i_1..i_{p-1}) of the dense
// order-p tensor (row-major, n^p FP32) and its lanes the last index, accumulating
// T sigma(i_1)...sigma(i_p) at (sum h) mod b into a shared-memory histogram of sketch m, which is
// added to S[m] (zeroed by the caller) at the end.
__global__ void __launch_bounds__(256) sketch_p_kernel(const float* T, int n, int p, long long rows,
                                                       const int32_t* h, const uint8_t* g, int log2b,
                                                       int mroots, float2* S) {
  extern __shared__ float2 hist[];
  const int b = 1 << log2b, m = blockIdx.y;
  int* hs = reinterpret_cast<int*>(hist + b);
  int* gs = hs + n;
  const int32_t* hm = h + (size_t)m * n;
  const uint8_t* gm = g + (size_t)m * n;
  for (int t = threadIdx.x; t < b; t += blockDim.x) hist[t] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    hs[i] = hm[i] & (b - 1);
    gs[i] = gm[i] & (mroots - 1);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
       r += warps) {
    long long q = r;
    int hr = 0, gr = 0;
    for (int j = 0; j < p - 1; ++j) {
      const int i = (int)(q % n);
      q /= n;
      hr += hs[i];
      gr += gs[i];
    }
    const float* row = T + r * n;
    for (int i = lane; i < n; i += 32) {
      const float x = __ldg(row + i);
      const float2 v = cscale(root_of_unity(gr + gs[i], mroots), x);
      float* slot = reinterpret_cast<float*>(&hist[(hr + hs[i]) & (b - 1)]);
      atomicAdd(slot, v.x);
      atomicAdd(slot + 1, v.y);
    }
  }
  __syncthreads();
  float2* Sm = S + (size_t)m * b;
  for (int t = threadIdx.x; t < b; t += blockDim.x) {
    const float2 v = hist[t];
    if (v.x != 0.f || v.y != 0.f) {
      atomicAdd(&Sm[t].x, v.x);
      atomicAdd(&Sm[t].y, v.y);
    }
  }
}

// Wedge-only build for a symmetric tensor: only sorted tuples i_1 <= ... <= i_p, each weighted by
// its number of orderings kappa = p! / prod(run lengths)! (Sec. 3.3: symmetric entries collide, so
// reading one per multiset suffices; kappa in {1, 3, 6} at p = 3).  A warp takes a sorted prefix
// (i_1..i_{p-2}) (flat index over n^{p-2}, unsorted ones skipped), loops i_{p-1} >= i_{p-2}, and its
// lanes take i_p >= i_{p-1}, a contiguous segment of the row.
__global__ void __launch_bounds__(256) sketch_p_wedge_kernel(const float* T, int n, int p,
                                                             long long prefixes, const int32_t* h,
                                                             const uint8_t* g, int log2b, int mroots,
                                                             float2* S) {
  extern __shared__ float2 hist[];
  const int b = 1 << log2b, m = blockIdx.y;
  int* hs = reinterpret_cast<int*>(hist + b);
  int* gs = hs + n;
  const int32_t* hm = h + (size_t)m * n;
  const uint8_t* gm = g + (size_t)m * n;
  for (int t = threadIdx.x; t < b; t += blockDim.x) hist[t] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    hs[i] = hm[i] & (b - 1);
    gs[i] = gm[i] & (mroots - 1);
  }
  __syncthreads();
  float fact[kMaxOrder + 1];
  fact[0] = 1.f;
  for (int j = 1; j <= kMaxOrder; ++j) fact[j] = fact[j - 1] * (float)j;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long q0 = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); q0 < prefixes;
       q0 += warps) {
    // digits of q0 in base n, most significant first = i_1 .. i_{p-2}; skip unsorted prefixes
    int idx[kMaxOrder];
    long long q = q0;
    for (int j = p - 3; j >= 0; --j) {
      idx[j] = (int)(q % n);
      q /= n;
    }
    bool sorted = true;
    for (int j = 1; j < p - 2; ++j) sorted &= idx[j - 1] <= idx[j];
    if (!sorted) continue;
    int hp = 0, gp = 0;
    float denom = 1.f;       // product of factorials of the prefix's runs except the last
    int run = 1;
    for (int j = 0; j < p - 2; ++j) {
      hp += hs[idx[j]];
      gp += gs[idx[j]];
      if (j > 0) {
        if (idx[j] == idx[j - 1]) {
          ++run;
        } else {
          denom *= fact[run];
          run = 1;
        }
      }
    }
    const int v = idx[p - 3];
    long long base = 0;
    for (int j = 0; j < p - 2; ++j) base = base * n + idx[j];
    for (int x = v; x < n; ++x) {
      const float* row = T + (base * n + x) * n;
      const int hx = hp + hs[x], gx = gp + gs[x];
      for (int y = x + lane; y < n; y += 32) {
        float dd;
        if (x == v) dd = (y == x) ? denom * fact[run + 2] : denom * fact[run + 1];
        else dd = (y == x) ? denom * fact[run] * 2.f : denom * fact[run];
        const float kappa = fact[p] / dd;
        const float2 val = cscale(root_of_unity(gx + gs[y], mroots), kappa * __ldg(row + y));
        float* slot = reinterpret_cast<float*>(&hist[(hx + hs[y]) & (b - 1)]);
        atomicAdd(slot, val.x);
        atomicAdd(slot + 1, val.y);
      }
    }
  }
  __syncthreads();
  float2* Sm = S + (size_t)m * b;
  for (int t = threadIdx.x; t < b; t += blockDim.x) {
    const float2 val = hist[t];
    if (val.x != 0.f || val.y != 0.f) {
      atomicAdd(&Sm[t].x, val.x);
      atomicAdd(&Sm[t].y, val.y);
    }
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
static int launch_contract_p_t(const PArgs& a, int L, cudaStream_t st) {
  constexpr size_t smem = contract_p_smem<LOGB>(P);
  static_assert(contract_p_smem<LOGB>(P) <= 227 * 1024, "transform buffers exceed shared memory");
  TSK_CUDA(tsk_smem_attr<contract_p_kernel<LOGB, P>>(smem));
  contract_p_kernel<LOGB, P><<<dim3(a.B, L), threads_for_logb(LOGB), smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <int LOGB>
static int launch_contract_p_b(int p, const PArgs& a, int L, cudaStream_t st) {
  switch (p) {
    case 3: return launch_contract_p_t<LOGB, 3>(a, L, st);
    case 4: return launch_contract_p_t<LOGB, 4>(a, L, st);
    case 5: return launch_contract_p_t<LOGB, 5>(a, L, st);
    case 6: return launch_contract_p_t<LOGB, 6>(a, L, st);
    default: return TSK_EUNSUPPORTED;
  }
}

static int launch_contract_p(int log2b, int p, const PArgs& a, int L, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_contract_p_b<8>(p, a, L, st);
    case 9: return launch_contract_p_b<9>(p, a, L, st);
    case 10: return launch_contract_p_b<10>(p, a, L, st);
    case 11: return launch_contract_p_b<11>(p, a, L, st);
    case 12: return launch_contract_p_b<12>(p, a, L, st);
    default: return TSK_EUNSUPPORTED;
  }
}

template <int LOGB, int P>
static int launch_deflate_p_t(float2* FS, float2* S, const int32_t* h, const uint8_t* g, int n,
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

template <int LOGB>
static int launch_deflate_p_b(int p, float2* FS, float2* S, const int32_t* h, const uint8_t* g,
                              int n, int L, const float* Uf, const float* lm, int r, double* lo,
                              float* Vo, int32_t* to, int B, cudaStream_t st) {
  switch (p) {
    case 3: return launch_deflate_p_t<LOGB, 3>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 4: return launch_deflate_p_t<LOGB, 4>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 5: return launch_deflate_p_t<LOGB, 5>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 6: return launch_deflate_p_t<LOGB, 6>(FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

static int launch_deflate_p(int log2b, int p, float2* FS, float2* S, const int32_t* h,
                            const uint8_t* g, int n, int L, const float* Uf, const float* lm, int r,
                            double* lo, float* Vo, int32_t* to, int B, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_deflate_p_b<8>(p, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 9: return launch_deflate_p_b<9>(p, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 10: return launch_deflate_p_b<10>(p, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 11: return launch_deflate_p_b<11>(p, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 12: return launch_deflate_p_b<12>(p, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

int launch_fft_batched(int log2b, const float2* in, float2* out, int B, int inverse, cudaStream_t st);

}  // namespace tsk

using namespace tsk;

static int check_order_p(int p, int B, int log2b, int64_t n) {
  if (p < 3 || p > kMaxOrder || log2b < 8 || log2b > 12 || B > kMaxB || n > 8192)
    return TSK_EUNSUPPORTED;
  return TSK_OK;
}

extern "C" int sketch_tensor_p(tsk_ctx* ctx, const float* T, int p, int64_t n, const int32_t* h,
                               const uint8_t* g, int B, int log2b, int symmetric, float* S) {
  if (!ctx || !T || !h || !g || !S) return TSK_EINVAL;
  if (B < 1 || n < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (p < 3 || p > kMaxOrder || log2b > 14 || B > kMaxB || n > 8192) return TSK_EUNSUPPORTED;
  long long rows = 1;
  for (int j = 0; j < p - 1; ++j) {
    rows *= n;
    if (rows > (1ll << 40)) return TSK_EUNSUPPORTED;
  }
  const size_t b = (size_t)1 << log2b;
  TSK_CUDA(cudaMemsetAsync(S, 0, (size_t)B * b * sizeof(float2), ctx->stream));
  const size_t smem = b * sizeof(float2) + 2 * (size_t)n * sizeof(int);
  if (smem > kSketchPSmemMax) return TSK_EUNSUPPORTED;
  // the limit is set once per device, so to the largest size any call may need
  const long long cap = 4LL * ctx->num_sms / B + 1;   // ~4 blocks per SM over all sketches
  if (symmetric) {
    const long long prefixes = rows / n;              // n^(p-2) flat prefixes
    long long blocks = (prefixes + 7) / 8;            // 8 warps of 256 threads, a prefix each
    if (blocks > cap) blocks = cap;
    TSK_CUDA(tsk_smem_attr<sketch_p_wedge_kernel>(kSketchPSmemMax));
    sketch_p_wedge_kernel<<<dim3((unsigned)blocks, B), 256, smem, ctx->stream>>>(
        T, (int)n, p, prefixes, h, g, log2b, p < 4 ? 4 : 8, reinterpret_cast<float2*>(S));
  } else {
    long long blocks = (rows + 7) / 8;                // 8 warps of 256 threads, a row each
    if (blocks > cap) blocks = cap;
    TSK_CUDA(tsk_smem_attr<sketch_p_kernel>(kSketchPSmemMax));
    sketch_p_kernel<<<dim3((unsigned)blocks, B), 256, smem, ctx->stream>>>(
        T, (int)n, p, rows, h, g, log2b, p < 4 ? 4 : 8, reinterpret_cast<float2*>(S));
  }
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

extern "C" int contract_p(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                          const uint8_t* g, int B, int log2b, int p, const float* U, int L,
                          int64_t n, float* Vmed, float* Vall, float* lam_med, float* lam_all) {
  if (!ctx || !FS || !S || !h || !g || !U) return TSK_EINVAL;
  if (B < 1 || L < 1 || n < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (!Vmed && !Vall && !lam_med && !lam_all) return TSK_EINVAL;
  int rc = check_order_p(p, B, log2b, n);
  if (rc != TSK_OK) return rc;
  if (L > 65535) return TSK_EUNSUPPORTED;
  const bool medians = Vmed || lam_med;
  const size_t need = (Vall ? 0 : ws_round((size_t)L * B * n * sizeof(float))) +
                      (lam_all ? 0 : ws_round((size_t)L * B * sizeof(float))) +
                      (medians ? ws_round((size_t)L * sizeof(unsigned)) : 0);
  if ((rc = tsk_ws_reserve(ctx, need)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  PArgs a{};
  a.FS = reinterpret_cast<const float2*>(FS);
  a.S = reinterpret_cast<const float2*>(S);
  a.h = h;
  a.g = g;
  a.U = U;
  a.n = (int)n;
  a.B = B;
  a.normalize_input = 0;
  a.Vall = Vall ? Vall : wc.take<float>((size_t)L * B * n);
  a.lam_all = lam_all ? lam_all : wc.take<float>((size_t)L * B);
  a.status = ctx->status;
  if (medians) {
    a.counters = wc.take<unsigned>(L);
    TSK_CUDA(cudaMemsetAsync(a.counters, 0, L * sizeof(unsigned), ctx->stream));
    a.Vmed = Vmed;
    a.lam_med = lam_med;
  }
  return launch_contract_p(log2b, p, a, L, ctx->stream);
}

extern "C" int64_t robust_power_method_p_launches(tsk_ctx* ctx, int p, int k, int T) {
  if (!ctx || p < 3 || p > kMaxOrder || k < 0 || T < 1) return -1;
  return 1 + (int64_t)k * ((int64_t)T + 2);
}

extern "C" int robust_power_method_p(tsk_ctx* ctx, const float* S, const int32_t* h,
                                     const uint8_t* g, int B, int log2b, int p, int64_t n, int k,
                                     int L, int T, const float* U0, double* lambda, float* Vout,
                                     int32_t* tau_star, float* S_deflated, float* lam_all_out,
                                     float* U_iters) {
  if (!ctx || !S || !h || !g) return TSK_EINVAL;
  if (k < 0 || T < 0 || B < 1 || L < 1 || n < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  int rc = check_order_p(p, B, log2b, n);
  if (rc != TSK_OK) return rc;
  if (L > 4096 || T < 1) return TSK_EUNSUPPORTED;
  const size_t b = (size_t)1 << log2b;
  if (k == 0) {
    if (S_deflated && S_deflated != S)
      TSK_CUDA(cudaMemcpyAsync(S_deflated, S, (size_t)B * b * sizeof(float2),
                               cudaMemcpyDeviceToDevice, ctx->stream));
    return TSK_OK;
  }
  if (!U0 || !lambda || !Vout) return TSK_EINVAL;
  const size_t need = 2 * ws_round((size_t)B * b * sizeof(float2)) +
                      ws_round((size_t)L * B * n * 4) + ws_round((size_t)L * B * 4) +
                      ws_round(2 * (size_t)L * n * 4) + ws_round((size_t)k * L * 4) +
                      ws_round((size_t)L * sizeof(unsigned));
  if ((rc = tsk_ws_reserve(ctx, need)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  float2* Sw = wc.take<float2>((size_t)B * b);
  float2* FSw = wc.take<float2>((size_t)B * b);
  float* Vall = wc.take<float>((size_t)L * B * n);
  float* lam_all = wc.take<float>((size_t)L * B);
  float* Ubuf = wc.take<float>(2 * (size_t)L * n);
  float* lam_med = lam_all_out ? lam_all_out : wc.take<float>((size_t)k * L);
  unsigned* counters = wc.take<unsigned>(L);
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(counters, 0, L * sizeof(unsigned), st));
  TSK_CUDA(cudaMemcpyAsync(Sw, S, (size_t)B * b * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_fft_batched(log2b, Sw, FSw, B, 0, st)) != TSK_OK) return rc;
  PArgs a{};
  a.FS = FSw;
  a.S = Sw;
  a.h = h;
  a.g = g;
  a.n = (int)n;
  a.B = B;
  a.Vall = Vall;
  a.lam_all = lam_all;
  a.status = ctx->status;
  a.counters = counters;
  for (int r = 0; r < k; ++r) {
    const float* cur = U0 + (size_t)r * L * n;
    for (int t = 0; t < T; ++t) {
      float* next = U_iters ? U_iters + ((size_t)r * T + t) * L * n : Ubuf + (size_t)((t + 1) & 1) * L * n;
      a.U = cur;
      a.normalize_input = (t == 0);
      a.Vmed = nullptr;
      a.Unext = next;
      a.lam_med = nullptr;
      if ((rc = launch_contract_p(log2b, p, a, L, st)) != TSK_OK) return rc;
      cur = next;
    }
    a.U = cur;
    a.normalize_input = 0;
    a.Unext = nullptr;
    a.lam_med = lam_med + (size_t)r * L;
    if ((rc = launch_contract_p(log2b, p, a, L, st)) != TSK_OK) return rc;
    if ((rc = launch_deflate_p(log2b, p, FSw, Sw, h, g, (int)n, L, cur, lam_med + (size_t)r * L, r,
                               lambda, Vout, tau_star, B, st)) != TSK_OK)
      return rc;
  }
  if (S_deflated)
    TSK_CUDA(cudaMemcpyAsync(S_deflated, Sw, (size_t)B * b * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  return TSK_OK;
}
