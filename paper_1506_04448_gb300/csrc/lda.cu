// Spectral LDA (App. D, Alg. 3) on the GPU.
//
//   * document statistics and M1^ (Eq. moment1) from a CSR corpus;
//   * the M2^ operator X -> M2^ X (Eq. moment2) without forming the V x V matrix;
//   * whitening (Alg. 3, line 3): randomized subspace iteration on M2^, Cholesky-QR
//     orthonormalisation and a parallel cyclic Jacobi eigensolver, all small dense algebra in
//     FP64; W = Q U_k diag(sigma)^(-1/2);
//   * the whitened third moment M3^(W,W,W) (Eq. moment3 with the per-document Eq. td):
//       sum_d a_d p_d^(x)3  with p_d = W^T n_d and a_d = 1 / (m_d (m_d-1)(m_d-2)),
//       minus the per-word corrections sum_i (w_i w_i r_i + w_i r_i w_i + r_i w_i w_i - 2 c_i w_i^(x)3)
//       with r_i = sum_d a_d n_di p_d and c_i = sum_d a_d n_di (the paper's per-word sums),
//     evaluated on the wedge a <= b <= c of the k x k x k tensor and expanded symmetrically;
//   * recovery (Alg. 3, line 6): alpha^ and mu^ = (alpha0+2)/2 lambda (W^+)^T v.
//
// The paper sketches every document's p_d^(x)3 by one FFT and accumulates in the frequency
// domain (2 * 10^7 transforms of length 2^14 for 10^6 documents and B = 20).  Because the
// sketch (Eq. 7) is linear in the tensor, the same sketch follows from the dense k^3 moment; on
// this GPU the dense wedge accumulation (D k^3 / 6 multiply-adds) costs far less than the
// transforms, so the moment is accumulated densely and sketched once (sketch_tensor).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "moments_tc.cuh"
#include "reduce.cuh"

namespace tsk {
namespace lda {

struct Corpus {
  const int64_t* indptr;
  const int32_t* idx;
  const int32_t* cnt;
  int64_t D;
  int64_t V;
};

constexpr int kWarpsPerBlock = 8;       // warp-per-document kernels: 256 threads
constexpr int kMaxWhitenCols = 128;     // k + oversampling
constexpr int kMaxTopics = 256;
constexpr int kTileItems = 32;          // documents (or words) staged per shared-memory tile
constexpr int kUnitThreads = 256;

TSK_HD int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ double weight2(double m) { return m >= 2.0 ? 1.0 / (m * (m - 1.0)) : 0.0; }
__device__ __forceinline__ double weight3(double m) {
  return m >= 3.0 ? 1.0 / (m * (m - 1.0) * (m - 2.0)) : 0.0;
}

__device__ __forceinline__ float4 f4_fma(float s, float4 x, float4 acc) {
  acc.x = fmaf(s, x.x, acc.x);
  acc.y = fmaf(s, x.y, acc.y);
  acc.z = fmaf(s, x.z, acc.z);
  acc.w = fmaf(s, x.w, acc.w);
  return acc;
}
__device__ __forceinline__ float4 f4_scale(float s, float4 x) {
  return make_float4(s * x.x, s * x.y, s * x.z, s * x.w);
}

// One (word id, count) pair of document entry j, with ids outside [0, V) and counts below 1
// recorded as TSK_EINVAL and read as an empty entry.
__device__ __forceinline__ void load_entry(const Corpus& c, int64_t j, int64_t end, int* status,
                                           int& i, float& n) {
  i = 0;
  n = 0.f;
  if (j < end) {
    const int ii = __ldg(c.idx + j);
    const int nn = __ldg(c.cnt + j);
    if (ii < 0 || ii >= c.V || nn < 1) {
      tsk_set_status(status, TSK_EINVAL);
    } else {
      i = ii;
      n = (float)nn;
    }
  }
}

// ------------------------------------------------------------------ document statistics
// Per document m_d; the numbers of documents with m_d >= 1, 2, 3 (counts[0..2]); optionally
// M1acc_i += n_di / m_d (double) and e_i += n_di / (m_d (m_d - 1)) (float).
__global__ void __launch_bounds__(256) doc_stats_kernel(Corpus c, float* mdoc,
                                                         unsigned long long* counts,
                                                         double* M1acc, float* e, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  unsigned long long c1 = 0, c2 = 0, c3 = 0;
  for (int64_t d = warp; d < c.D; d += nwarps) {
    const int64_t beg = c.indptr[d], end = c.indptr[d + 1];
    float msum = 0.f;
    for (int64_t j = beg + lane; j < end; j += 32) {
      int i;
      float n;
      load_entry(c, j, end, status, i, n);
      msum += n;
    }
    const float m = warp_sum(msum);   // exact: integer counts below 2^24
    if (lane == 0) {
      mdoc[d] = m;
      c1 += m >= 1.f;
      c2 += m >= 2.f;
      c3 += m >= 3.f;
    }
    if (M1acc && m >= 1.f) {
      const double inv_m = 1.0 / (double)m;
      const float a2 = (float)weight2(m);
      for (int64_t j = beg + lane; j < end; j += 32) {
        int i;
        float n;
        load_entry(c, j, end, nullptr, i, n);
        if (n > 0.f) {
          atomicAdd(M1acc + i, (double)n * inv_m);
          if (a2 != 0.f) atomicAdd(e + i, a2 * n);
        }
      }
    }
  }
  __shared__ unsigned long long red[3];
  if (threadIdx.x < 3) red[threadIdx.x] = 0;
  __syncthreads();
  if (lane == 0 && (c1 | c2 | c3)) {
    atomicAdd(&red[0], c1);
    atomicAdd(&red[1], c2);
    atomicAdd(&red[2], c3);
  }
  __syncthreads();
  if (threadIdx.x < 3 && red[threadIdx.x]) atomicAdd(counts + threadIdx.x, red[threadIdx.x]);
}

// M1 = M1acc / max(D1, 1) as float.
__global__ void m1_finish_kernel(const double* M1acc, const unsigned long long* counts, int64_t V,
                                 float* M1) {
  const double inv = 1.0 / (double)(counts[0] > 0 ? counts[0] : 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (int64_t)gridDim.x * blockDim.x)
    M1[i] = (float)(M1acc[i] * inv);
}

// ------------------------------------------------------------------ M2^ operator (Eq. moment2)
// Document part of M2^ X: Yacc_i += n_di / (m (m-1)) * (sum_j n_dj X_j) for every document with
// m >= 2.  X, Yacc: [V][cp] (cp a multiple of 4, NQ * 128 >= cp).
template <int NQ>
__global__ void __launch_bounds__(256) m2_docs_kernel(Corpus c, const float* mdoc, const float* X,
                                                       int cp, float* Yacc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const int cq = cp >> 2;
  for (int64_t d = warp; d < c.D; d += nwarps) {
    const float m = mdoc[d];
    if (m < 2.f) continue;
    const float a2 = (float)weight2(m);
    const int64_t beg = c.indptr[d], end = c.indptr[d + 1];
    float4 t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t base = beg; base < end; base += 32) {
      int i;
      float n;
      load_entry(c, base + lane, end, nullptr, i, n);
      const int cnt = (int)min64(32, end - base);
      for (int s = 0; s < cnt; ++s) {
        const int ii = __shfl_sync(0xffffffffu, i, s);
        const float nn = __shfl_sync(0xffffffffu, n, s);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int qd = lane + 32 * q;
          if (qd < cq) t[q] = f4_fma(nn, __ldg(reinterpret_cast<const float4*>(X + (int64_t)ii * cp) + qd), t[q]);
        }
      }
    }
    for (int64_t base = beg; base < end; base += 32) {
      int i;
      float n;
      load_entry(c, base + lane, end, nullptr, i, n);
      const int cnt = (int)min64(32, end - base);
      for (int s = 0; s < cnt; ++s) {
        const int ii = __shfl_sync(0xffffffffu, i, s);
        const float w = a2 * __shfl_sync(0xffffffffu, n, s);
        if (w == 0.f) continue;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int qd = lane + 32 * q;
          if (qd < cq) atomicAdd(reinterpret_cast<float4*>(Yacc + (int64_t)ii * cp) + qd, f4_scale(w, t[q]));
        }
      }
    }
  }
}

// s[col] += sum_i M1_i X[i][col]  (double, one atomic per block and column).
__global__ void m1_dot_kernel(const float* M1, const float* X, int64_t V, int cp, double* s) {
  for (int col = threadIdx.x; col < cp; col += blockDim.x) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x; i < V; i += gridDim.x) acc += (double)M1[i] * (double)X[i * cp + col];
    atomicAdd(s + col, acc);
  }
}

// Y = (Yacc - e_i X_i) / D2 - alpha0/(alpha0+1) M1_i s   (the diagonal term of E^[x1 (x) x2] and
// the rank-1 term of Eq. moment2).  Y may alias Yacc.
__global__ void m2_finish_kernel(const float* Yacc, const float* X, const float* e, const float* M1,
                                 const double* s, const unsigned long long* counts, double coef,
                                 int64_t V, int cp, float* Y) {
  const double invD2 = 1.0 / (double)(counts[1] > 0 ? counts[1] : 1);
  const int64_t total = V * cp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cp;
    const int col = (int)(t - i * cp);
    const double v = ((double)Yacc[t] - (double)e[i] * (double)X[t]) * invD2 - coef * (double)M1[i] * s[col];
    Y[t] = (float)v;
  }
}

// ------------------------------------------------------------------ small dense FP64 algebra
// Compensated FP32 dot products (the Dot2 scheme of Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005): each product x y is split exactly into p + e
// with an FMA, p is added to the running sum s by Knuth's TwoSum, and the two rounding errors
// are summed in c.  s + c carries the sum as accurately as FP64 accumulation of the exact
// products to within a factor of the condition of the sum, at about ten FP32 operations per
// term against one FP64 FMA at this part's 1/64 FP64 rate.  Every operation is an explicit
// round-to-nearest intrinsic, so that no multiply-add is contracted into an FMA.
__device__ __forceinline__ void dot2_acc(float x, float y, float& s, float& c) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
}

// Partial Gram matrices part[blk][a][b] = sum over the block's rows of X[r][a] Y[r][b], a, b < c,
// accumulated with dot2_acc and written in FP64.  Each thread owns a 4 x 4 tile; blockIdx.y
// selects a group of 256 tiles.
constexpr int kGramRows = 32;
__global__ void __launch_bounds__(256) gram_partial_kernel(const float* X, int ldx, const float* Y,
                                                            int ldy, int64_t rows, int c,
                                                            int64_t rows_per_block, double* part) {
  __shared__ float xs[kGramRows][kMaxWhitenCols + 4];
  __shared__ float ys[kGramRows][kMaxWhitenCols + 4];
  const int c4 = (c + 3) >> 2;
  const int tile = blockIdx.y * 256 + threadIdx.x;
  const bool active = tile < c4 * c4;
  const int ta = active ? tile / c4 : 0, tb = active ? tile % c4 : 0;
  float accs[4][4] = {}, accc[4][4] = {};
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min64(rows, r0 + rows_per_block);
  for (int64_t base = r0; base < r1; base += kGramRows) {
    const int nr = (int)min64(kGramRows, r1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < kGramRows * c4 * 4; e += blockDim.x) {
      const int r = e / (c4 * 4), col = e % (c4 * 4);
      const bool ok = r < nr && col < c;
      xs[r][col] = ok ? X[(base + r) * ldx + col] : 0.f;
      ys[r][col] = ok ? Y[(base + r) * ldy + col] : 0.f;
    }
    __syncthreads();
    if (active) {
      for (int r = 0; r < nr; ++r) {
        const float4 xa = *reinterpret_cast<const float4*>(&xs[r][4 * ta]);
        const float4 yb = *reinterpret_cast<const float4*>(&ys[r][4 * tb]);
        const float xv[4] = {xa.x, xa.y, xa.z, xa.w};
        const float yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) dot2_acc(xv[i], yv[j], accs[i][j], accc[i][j]);
      }
    }
  }
  if (!active) return;
  double* out = part + (size_t)blockIdx.x * c * c;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = 4 * ta + i, b = 4 * tb + j;
      if (a < c && b < c) out[a * c + b] = (double)accs[i][j] + (double)accc[i][j];
    }
}

__global__ void gram_reduce_kernel(const double* part, int nblk, int c, double* G) {
  const int cc = c * c;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cc; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * cc + e];
    G[e] = s;
  }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) red[32] = r;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

// Cholesky G + shift I = L L^T (one block, FP64, L in shared memory) and Minv = L^-T, so that
// X Minv has orthonormal columns when G = X^T X.  shift_scale > 0 adds
// shift_scale * trace(G) to the diagonal (shifted Cholesky-QR: the first pass on an
// ill-conditioned block).  A non-positive pivot records TSK_ENONFINITE and leaves Minv = I.
__global__ void __launch_bounds__(1024) chol_inv_kernel(const double* G, int c, double shift_scale,
                                                         double* Minv, int* status) {
  extern __shared__ double sh[];
  const int ld = c + 1;
  double* A = sh;
  __shared__ double red[33];
  __shared__ int bad;
  double tr = 0.0;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    A[i * ld + j] = G[e];
    if (i == j) tr += G[e];
  }
  if (threadIdx.x == 0) bad = 0;
  tr = block_sum_d(tr, red);
  const double shift = shift_scale * tr;
  for (int i = threadIdx.x; i < c; i += blockDim.x) A[i * ld + i] += shift;
  __syncthreads();
  for (int j = 0; j < c; ++j) {
    if (threadIdx.x == 0) {
      const double dj = A[j * ld + j];
      if (!(dj > 0.0) || !isfinite(dj)) {
        bad = 1;
        A[j * ld + j] = 1.0;
      } else {
        A[j * ld + j] = sqrt(dj);
      }
    }
    __syncthreads();
    const double ljj = A[j * ld + j];
    for (int i = j + 1 + threadIdx.x; i < c; i += blockDim.x) A[i * ld + j] /= ljj;
    __syncthreads();
    const int rem = c - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, l = j + 1 + e % rem;
      if (l <= i) A[i * ld + l] -= A[i * ld + j] * A[l * ld + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) tsk_set_status(status, TSK_ENONFINITE);
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) Minv[e] = (e / c == e % c) ? 1.0 : 0.0;
    return;
  }
  // column j of L^-1 by forward substitution; stored as row j of Minv = L^-T
  for (int j = threadIdx.x; j < c; j += blockDim.x) {
    double* x = Minv + (size_t)j * c;
    for (int i = 0; i < j; ++i) x[i] = 0.0;
    x[j] = 1.0 / A[j * ld + j];
    for (int i = j + 1; i < c; ++i) {
      double s = 0.0;
      for (int l = j; l < i; ++l) s = fma(A[i * ld + l], x[l], s);
      x[i] = -s / A[i * ld + i];
    }
  }
}

// out = Y M with Y [rows][c] (ld ldy, float) and M [c][cout] (FP64); one warp per row.  M is
// held in shared memory as M_hi + M_lo (float, M_lo = M - M_hi rounded), and each output sums
// y M_hi with dot2_acc and y M_lo plainly into the compensation term, which keeps the
// cancellation of an ill-conditioned first orthogonalisation pass (large M, orthonormal result)
// to FP32 rounding of the result.  transposed_out = 1 stores out[j][row] (ld ldo) instead of
// out[row][j].  In place (out == Y) is safe: each warp reads its whole row before writing it.
__global__ void __launch_bounds__(256) rmul_kernel(const float* Y, int ldy, int64_t rows, int c,
                                                    const double* M, int cout, float* out, int ldo,
                                                    int transposed_out) {
  extern __shared__ float Mhl[];
  float* Mhi = Mhl;
  float* Mlo = Mhl + c * cout;
  for (int e = threadIdx.x; e < c * cout; e += blockDim.x) {
    const double m = M[e];
    const float hi = __double2float_rn(m);
    Mhi[e] = hi;
    Mlo[e] = __double2float_rn(m - (double)hi);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t r = warp; r < rows; r += nwarps) {
    float yr[kMaxWhitenCols / 32];
#pragma unroll
    for (int t = 0; t < kMaxWhitenCols / 32; ++t) {
      const int a = lane + 32 * t;
      yr[t] = a < c ? Y[r * ldy + a] : 0.f;
    }
    float accs[kMaxWhitenCols / 32] = {}, accc[kMaxWhitenCols / 32] = {};
#pragma unroll
    for (int t = 0; t < kMaxWhitenCols / 32; ++t) {
      for (int l = 0; l < 32; ++l) {
        const int a = 32 * t + l;
        if (a >= c) break;
        const float ya = __shfl_sync(0xffffffffu, yr[t], l);
#pragma unroll
        for (int u = 0; u < kMaxWhitenCols / 32; ++u) {
          const int j = lane + 32 * u;
          if (j < cout) {
            dot2_acc(ya, Mhi[a * cout + j], accs[u], accc[u]);
            accc[u] = __fmaf_rn(ya, Mlo[a * cout + j], accc[u]);
          }
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kMaxWhitenCols / 32; ++u) {
      const int j = lane + 32 * u;
      if (j < cout) {
        const float v = __fadd_rn(accs[u], accc[u]);
        if (transposed_out) out[(int64_t)j * ldo + r] = v;
        else out[r * ldo + j] = v;
      }
    }
  }
}

// Symmetric eigendecomposition of (Bm + Bm^T)/2 (c x c, FP64) by the cyclic Jacobi method with
// the round-robin ordering: every round applies c/2 disjoint plane rotations at once (disjoint
// pairs commute), a sweep is c-1 rounds (every pair once).  A round updates A <- J^T A J as 2 x 2
// blocks: block (t1, t2) of pairs t1 <= t2 becomes R1^T X R2 (rows by pair t1's rotation, columns
// by pair t2's), and its mirror is written as the transpose, so each element of the symmetric A
// is computed once; the eigenvectors accumulate E <- E J.  A rotation whose off-diagonal element
// is below 2^-54 of both diagonal elements (smaller than their rounding) is not applied: the
// element is set to zero (Rutishauser's threshold rule), and blocks of two such pairs are
// skipped.  Stops when the off-diagonal Frobenius norm is below 1e-15 of the whole norm, or after
// max_sweeps.  One block; A in shared memory; eigenvectors in global memory (columns of evec).
__global__ void __launch_bounds__(1024) jacobi_eig_kernel(const double* Bm, int c, int max_sweeps,
                                                           double* evec, double* evals) {
  extern __shared__ double sh[];
  const int ld = c + 1;
  double* A = sh;
  __shared__ double rc[kMaxWhitenCols / 2], rs[kMaxWhitenCols / 2];
  __shared__ int rp[kMaxWhitenCols / 2], rq[kMaxWhitenCols / 2];
  __shared__ double red[33];
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    const int i = e / c, j = e % c;
    A[i * ld + j] = 0.5 * (Bm[i * c + j] + Bm[j * c + i]);
    evec[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int n2 = c + (c & 1);          // even number of players (one dummy when c is odd)
  const int npair = n2 / 2;
  const int nblk = npair * (npair + 1) / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
      const int i = e / c, j = e % c;
      const double v = A[i * ld + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    off = block_sum_d(off, red);
    tot = block_sum_d(tot, red);
    if (!(off > 1e-30 * tot)) break;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        const int pa = t, pb = n2 - 1 - t;
        const int x = pa == 0 ? 0 : 1 + (pa - 1 + r) % (n2 - 1);
        const int y = 1 + (pb - 1 + r) % (n2 - 1);
        const int p = min(x, y), q = max(x, y);
        double cs = 1.0, sn = 0.0;
        if (q < c) {
          const double apq = A[p * ld + q];
          const double app = A[p * ld + p], aqq = A[q * ld + q];
          const double tiny = 0x1p-54 * fmin(fabs(app), fabs(aqq));
          if (fabs(apq) <= tiny) {
            A[p * ld + q] = 0.0;           // below the diagonal's rounding: dropped
            A[q * ld + p] = 0.0;
          } else {
            const double tau = (aqq - app) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
            cs = 1.0 / sqrt(1.0 + tt * tt);
            sn = tt * cs;
          }
        }
        rc[t] = cs;
        rs[t] = sn;
        rp[t] = p;
        rq[t] = q < c ? q : -1;
      }
      __syncthreads();
      // A <- J^T A J by 2 x 2 blocks (t1 <= t2); a missing index (the dummy) is a 1-wide block
      for (int e = threadIdx.x; e < nblk; e += blockDim.x) {
        int t1 = 0, rem = e;
        while (rem >= npair - t1) { rem -= npair - t1; ++t1; }
        const int t2 = t1 + rem;
        const double s1 = rs[t1], s2 = rs[t2];
        if (s1 == 0.0 && s2 == 0.0) continue;
        const double c1 = rc[t1], c2 = rc[t2];
        const int p1 = rp[t1], q1 = rq[t1], p2 = rp[t2], q2 = rq[t2];
        const double x00 = A[p1 * ld + p2];
        const double x01 = q2 >= 0 ? A[p1 * ld + q2] : 0.0;
        const double x10 = q1 >= 0 ? A[q1 * ld + p2] : 0.0;
        const double x11 = (q1 >= 0 && q2 >= 0) ? A[q1 * ld + q2] : 0.0;
        // rows by (c1, s1): row p1' = c1 row p1 - s1 row q1, row q1' = s1 row p1 + c1 row q1
        const double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
        const double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
        // columns by (c2, s2)
        const double z00 = c2 * y00 - s2 * y01, z01 = s2 * y00 + c2 * y01;
        const double z10 = c2 * y10 - s2 * y11, z11 = s2 * y10 + c2 * y11;
        if (t1 == t2) {
          // the pair's own block: the rotation annihilates its off-diagonal element
          A[p1 * ld + p1] = z00;
          if (q1 >= 0) {
            A[q1 * ld + q1] = z11;
            A[p1 * ld + q1] = 0.0;
            A[q1 * ld + p1] = 0.0;
          }
          continue;
        }
        A[p1 * ld + p2] = z00;
        if (q2 >= 0) A[p1 * ld + q2] = z01;
        if (q1 >= 0) A[q1 * ld + p2] = z10;
        if (q1 >= 0 && q2 >= 0) A[q1 * ld + q2] = z11;
        {
          A[p2 * ld + p1] = z00;
          if (q2 >= 0) A[q2 * ld + p1] = z01;
          if (q1 >= 0) A[p2 * ld + q1] = z10;
          if (q1 >= 0 && q2 >= 0) A[q2 * ld + q1] = z11;
        }
      }
      // E <- E J (columns p, q of every row)
      for (int e = threadIdx.x; e < npair * c; e += blockDim.x) {
        const int t = e / c, i = e % c;
        const int q = rq[t];
        if (q < 0 || rs[t] == 0.0) continue;
        const int p = rp[t];
        const double ea = evec[i * c + p], eb = evec[i * c + q];
        evec[i * c + p] = rc[t] * ea - rs[t] * eb;
        evec[i * c + q] = rs[t] * ea + rc[t] * eb;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < c; i += blockDim.x) evals[i] = A[i * ld + i];
}

// Top-k eigenpairs by value (ties by index): sigma[j] = evals[o_j], Mk[a][j] = evec[a][o_j] /
// sqrt(sigma_j).  A non-positive sigma among the k records TSK_EINVAL (M2^ has fewer than k
// positive eigenvalues in the sampled subspace) and writes zeros.
__global__ void select_topk_kernel(const double* evec, const double* evals, int c, int k,
                                   double* sigma, double* Mk, int* status) {
  __shared__ int order[kMaxWhitenCols];
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    const double li = evals[i];
    int rank = 0;
    for (int j = 0; j < c; ++j) {
      const double lj = evals[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * k; e += blockDim.x) {
    const int a = e / k, j = e % k;
    const double s = evals[order[j]];
    Mk[e] = s > 0.0 ? evec[a * c + order[j]] / sqrt(s) : 0.0;
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double s = evals[order[j]];
    sigma[j] = s;
    if (!(s > 0.0)) tsk_set_status(status, TSK_EINVAL);
  }
}

// ------------------------------------------------------------------ whitened moments
// Projection pass, one warp per document: p_d = sum_i n_di w_i (stored, [D][kp]);
// qpart[block] += p_d / m_d; R_i += a3 n_di p_d (float4 atomics), ce_i += (a3 n_di, a2 n_di).
template <int NQ>
__global__ void __launch_bounds__(256) project_kernel(Corpus c, const float* mdoc, const float* Wp,
                                                       int kp, float* P, float* R, float* ce,
                                                       float* qpart) {
  __shared__ __align__(16) float qsh[kWarpsPerBlock][kMaxTopics];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp = (int64_t)blockIdx.x * kWarpsPerBlock + wib;
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  const int kq = kp >> 2;
  float4 qacc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) qacc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t d = warp; d < c.D; d += nwarps) {
    const float m = mdoc[d];
    const int64_t beg = c.indptr[d], end = c.indptr[d + 1];
    float4 p[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t base = beg; base < end; base += 32) {
      int i;
      float n;
      load_entry(c, base + lane, end, nullptr, i, n);
      const int cnt = (int)min64(32, end - base);
#pragma unroll 4
      for (int s = 0; s < cnt; ++s) {
        const int ii = __shfl_sync(0xffffffffu, i, s);
        const float nn = __shfl_sync(0xffffffffu, n, s);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int qd = lane + 32 * q;
          if (qd < kq) p[q] = f4_fma(nn, __ldg(reinterpret_cast<const float4*>(Wp + (int64_t)ii * kp) + qd), p[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int qd = lane + 32 * q;
      if (qd < kq) reinterpret_cast<float4*>(P + d * kp)[qd] = p[q];
    }
    if (m >= 1.f) {
      const float a1 = 1.f / m;
#pragma unroll
      for (int q = 0; q < NQ; ++q) qacc[q] = f4_fma(a1, p[q], qacc[q]);
    }
    const float a3 = (float)weight3(m), a2 = (float)weight2(m);
    if (a2 == 0.f) continue;
    for (int64_t base = beg; base < end; base += 32) {
      int i;
      float n;
      load_entry(c, base + lane, end, nullptr, i, n);
      if (n > 0.f) atomicAdd(reinterpret_cast<float2*>(ce) + i, make_float2(a3 * n, a2 * n));
      if (a3 == 0.f) continue;
      const int cnt = (int)min64(32, end - base);
      for (int s = 0; s < cnt; ++s) {
        const int ii = __shfl_sync(0xffffffffu, i, s);
        const float w = a3 * __shfl_sync(0xffffffffu, n, s);
        if (w == 0.f) continue;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int qd = lane + 32 * q;
          if (qd < kq) atomicAdd(reinterpret_cast<float4*>(R + (int64_t)ii * kp) + qd, f4_scale(w, p[q]));
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int qd = lane + 32 * q;
    if (qd < kq) reinterpret_cast<float4*>(qsh[wib])[qd] = qacc[q];
  }
  __syncwarp();
  __syncthreads();
  for (int a = threadIdx.x; a < kp; a += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < kWarpsPerBlock; ++w) s += qsh[w][a];
    qpart[(size_t)blockIdx.x * kp + a] = s;
  }
}

// Work units of the wedge accumulation.  ORDER 3: unit (a, bb, cb) owns the 8 x 8 block of
// entries (a, 8bb + j, 8cb + l) with bb <= cb and a <= min(8bb + 7, k - 1); ORDER 2: unit (a, bb)
// owns (a, 8bb + j) with the same bound on a.  Units are listed by (bb, cb, a) so that the 32
// units of a warp share their b and c blocks (broadcast shared-memory reads); packed as
// a | bb << 10 | cb << 20.  unit_of maps (bb, cb, a) back to the unit's index.
__global__ void build_units_kernel(int k, int kp, int* units3, int* unit3_of, int* units2,
                                   int* unit2_of) {
  const int nb = kp / 8;
  const int bb = blockIdx.x, cb = threadIdx.x;
  if (cb >= nb) return;
  const int cnt_bb = min(8 * bb + 8, k);
  if (cb >= bb) {
    int off = 0;
    for (int b2 = 0; b2 < bb; ++b2) off += (nb - b2) * min(8 * b2 + 8, k);
    off += (cb - bb) * cnt_bb;
    for (int a = 0; a < cnt_bb; ++a) {
      units3[off + a] = a | (bb << 10) | (cb << 20);
      unit3_of[(bb * nb + cb) * kp + a] = off + a;
    }
  }
  if (cb == 0) {
    int off = 0;
    for (int b2 = 0; b2 < bb; ++b2) off += min(8 * b2 + 8, k);
    for (int a = 0; a < cnt_bb; ++a) {
      units2[off + a] = a | (bb << 10);
      unit2_of[bb * kp + a] = off + a;
    }
  }
}

inline int count_units3(int k, int kp) {
  const int nb = kp / 8;
  int n = 0;
  for (int bb = 0; bb < nb; ++bb) n += (nb - bb) * std::min(8 * bb + 8, k);
  return n;
}
inline int count_units2(int k, int kp) {
  int n = 0;
  for (int bb = 0; bb < kp / 8; ++bb) n += std::min(8 * bb + 8, k);
  return n;
}

enum { FROM_DOCS = 0, FROM_WORDS = 1 };

struct MomentArgs {
  const int* units;
  int units_pad;            // multiple of kUnitThreads; rows of unit slots in `part`
  const float* rows0;       // FROM_DOCS: P [items][kp]; FROM_WORDS: Wp [items][kp]
  const float* rows1;       // FROM_WORDS, ORDER 3: R [items][kp]
  const float* wsrc;        // FROM_DOCS: m_d; FROM_WORDS: ce [items][2]
  int64_t items;
  int64_t per_split;        // items per blockIdx.y (multiple of kTileItems)
  int kp;
  float* part;              // [gridDim.y][E][units_pad], E = 64 (ORDER 3) or 8 (ORDER 2)
};

// Wedge accumulation over items (documents or words) for the units of this block:
//   ORDER 3, FROM_DOCS : acc[j][l] += a3_d p_a p_b p_c
//   ORDER 3, FROM_WORDS: acc[j][l] += w_a w_b (r_c - 2 c_i w_c) + (w_a r_b + r_a w_b) w_c
//   ORDER 2, FROM_DOCS : acc[j] += a2_d p_a p_b;  ORDER 2, FROM_WORDS: acc[j] += e_i w_a w_b
// with b = 8bb + j, c = 8cb + l.  Each split of items writes its own partial sums (summed later
// in FP64), so every FP32 running sum covers at most per_split items.
template <int ORDER, int MODE>
__global__ void __launch_bounds__(kUnitThreads, 2) moments_kernel(MomentArgs m) {
  extern __shared__ __align__(16) float smem[];
  constexpr bool TWO_ROWS = (ORDER == 3 && MODE == FROM_WORDS);
  const int kp = m.kp;
  float* s0 = smem;                                   // [kTileItems][kp]
  float* s1 = s0 + kTileItems * kp;                   // [kTileItems][kp] (TWO_ROWS)
  float* sw = s1 + (TWO_ROWS ? kTileItems * kp : 0);  // [kTileItems]
  const int slot = blockIdx.x * kUnitThreads + threadIdx.x;
  const int u = m.units[slot];
  const int a = u & 1023, b0 = 8 * ((u >> 10) & 1023), c0 = 8 * (u >> 20);
  constexpr int NL = ORDER == 3 ? 8 : 1;
  float acc[8][NL];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int l = 0; l < NL; ++l) acc[j][l] = 0.f;
  const int64_t i0 = (int64_t)blockIdx.y * m.per_split;
  const int64_t i1 = min64(m.items, i0 + m.per_split);
  const int kq = kp >> 2;
  for (int64_t base = i0; base < i1; base += kTileItems) {
    const int nr = (int)min64(kTileItems, i1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * kq; e += kUnitThreads) {
      const int r = e / kq, qd = e % kq;
      reinterpret_cast<float4*>(s0 + r * kp)[qd] =
          __ldg(reinterpret_cast<const float4*>(m.rows0 + (base + r) * kp) + qd);
      if (TWO_ROWS)
        reinterpret_cast<float4*>(s1 + r * kp)[qd] =
            __ldg(reinterpret_cast<const float4*>(m.rows1 + (base + r) * kp) + qd);
    }
    for (int r = threadIdx.x; r < nr; r += kUnitThreads) {
      float w;
      if (MODE == FROM_DOCS) {
        const double md = m.wsrc[base + r];
        w = (float)(ORDER == 3 ? weight3(md) : weight2(md));
      } else {
        w = m.wsrc[2 * (base + r) + (ORDER == 3 ? 0 : 1)];
      }
      sw[r] = w;
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const float* row = s0 + r * kp;
      const float4 pb0 = *reinterpret_cast<const float4*>(row + b0);
      const float4 pb1 = *reinterpret_cast<const float4*>(row + b0 + 4);
      const float pb[8] = {pb0.x, pb0.y, pb0.z, pb0.w, pb1.x, pb1.y, pb1.z, pb1.w};
      if (ORDER == 2) {
        const float xa = sw[r] * row[a];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = fmaf(xa, pb[j], acc[j][0]);
      } else {
        const float4 pc0 = *reinterpret_cast<const float4*>(row + c0);
        const float4 pc1 = *reinterpret_cast<const float4*>(row + c0 + 4);
        const float pc[8] = {pc0.x, pc0.y, pc0.z, pc0.w, pc1.x, pc1.y, pc1.z, pc1.w};
        if (MODE == FROM_DOCS) {
          const float xa = sw[r] * row[a];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float x = xa * pb[j];
#pragma unroll
            for (int l = 0; l < NL; ++l) acc[j][l] = fmaf(x, pc[l], acc[j][l]);
          }
        } else {
          const float* rrow = s1 + r * kp;
          const float4 rb0 = *reinterpret_cast<const float4*>(rrow + b0);
          const float4 rb1 = *reinterpret_cast<const float4*>(rrow + b0 + 4);
          const float4 rc0 = *reinterpret_cast<const float4*>(rrow + c0);
          const float4 rc1 = *reinterpret_cast<const float4*>(rrow + c0 + 4);
          const float rb[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
          const float rcv[8] = {rc0.x, rc0.y, rc0.z, rc0.w, rc1.x, rc1.y, rc1.z, rc1.w};
          const float wa = row[a], ra = rrow[a], cw2 = 2.f * sw[r];
          float z[8];
#pragma unroll
          for (int l = 0; l < 8; ++l) z[l] = fmaf(-cw2, pc[l], rcv[l]);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float x = wa * pb[j];
            const float y = fmaf(wa, rb[j], ra * pb[j]);
#pragma unroll
            for (int l = 0; l < NL; ++l) acc[j][l] = fmaf(x, z[l], fmaf(y, pc[l], acc[j][l]));
          }
        }
      }
    }
  }
  constexpr int E = 8 * NL;
  float* out = m.part + (size_t)blockIdx.y * E * m.units_pad + slot;
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int l = 0; l < NL; ++l) out[(size_t)(j * NL + l) * m.units_pad] = acc[j][l];
}

// q = sum of the projection blocks' partial sums / D1;
// E2 (k x k, FP64, symmetric) = (sum_s docs - sum_s words) / D2 on the pairs a <= b.
__global__ void finalize2_kernel(const float* qpart, int nqpart, const float* part2d, int S2d,
                                 const float* part2w, int S2w, int units2_pad, const int* unit2_of,
                                 const unsigned long long* counts, int k, int kp, double* q,
                                 double* E2) {
  const double invD1 = 1.0 / (double)(counts[0] > 0 ? counts[0] : 1);
  const double invD2 = 1.0 / (double)(counts[1] > 0 ? counts[1] : 1);
  const int b = blockIdx.x;
  for (int a = threadIdx.x; a <= b; a += blockDim.x) {
    const int u = unit2_of[(b / 8) * kp + a];
    const int e = b % 8;
    double s = 0.0;
    for (int t = 0; t < S2d; ++t) s += part2d[((size_t)t * 8 + e) * units2_pad + u];
    for (int t = 0; t < S2w; ++t) s -= part2w[((size_t)t * 8 + e) * units2_pad + u];
    s *= invD2;
    E2[a * k + b] = s;
    E2[b * k + a] = s;
  }
  if (b == 0) {
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
      double s = 0.0;
      for (int t = 0; t < nqpart; ++t) s += qpart[(size_t)t * kp + a];
      q[a] = s * invD1;
    }
  }
}

// M3(a,b,c) = E3 - alpha0/(alpha0+2) (E2_ab q_c + E2_ac q_b + E2_bc q_a)
//             + 2 alpha0^2/((alpha0+1)(alpha0+2)) q_a q_b q_c  on the wedge a <= b <= c,
// written to all six permutations of the dense k^3 output.  Block (b, c), thread a.
__global__ void finalize3_kernel(const float* part3d, int S3d, const float* part3w, int S3w,
                                 int units3_pad, const int* unit3_of,
                                 const unsigned long long* counts, const double* q,
                                 const double* E2, int k, int kp, double alpha0, float* M3,
                                 const double* tcpart, int Stc, long long tc_rows, int tc_N) {
  const int b = blockIdx.x, c = blockIdx.y;
  if (c < b) return;
  const double invD3 = 1.0 / (double)(counts[2] > 0 ? counts[2] : 1);
  const double c1 = alpha0 / (alpha0 + 2.0);
  const double c2 = 2.0 * alpha0 * alpha0 / ((alpha0 + 1.0) * (alpha0 + 2.0));
  const int nb = kp / 8;
  const int e = (b % 8) * 8 + (c % 8);
  for (int a = threadIdx.x; a <= b; a += blockDim.x) {
    const int u = unit3_of[((b / 8) * nb + (c / 8)) * kp + a];
    double s = 0.0;
    if (tcpart) {   // document term from the tensor-core splits: row of pair (a, b), column c
      const size_t row = (size_t)b * (b + 1) / 2 + a;
      for (int t = 0; t < Stc; ++t) s += tcpart[((size_t)t * tc_rows + row) * tc_N + c];
    } else {
      for (int t = 0; t < S3d; ++t) s += part3d[((size_t)t * 64 + e) * units3_pad + u];
    }
    for (int t = 0; t < S3w; ++t) s -= part3w[((size_t)t * 64 + e) * units3_pad + u];
    const double E3 = s * invD3;
    const double v = E3 - c1 * (E2[a * k + b] * q[c] + E2[a * k + c] * q[b] + E2[b * k + c] * q[a]) +
                     c2 * q[a] * q[b] * q[c];
    const float f = (float)v;
    const int64_t kk = k;
    M3[(a * kk + b) * kk + c] = f;
    M3[(a * kk + c) * kk + b] = f;
    M3[(b * kk + a) * kk + c] = f;
    M3[(b * kk + c) * kk + a] = f;
    M3[(c * kk + a) * kk + b] = f;
    M3[(c * kk + b) * kk + a] = f;
  }
}

// Alg. 3, line 6 (small, one block): alpha^_i = 4 alpha0 (alpha0+1) / ((alpha0+2)^2 lambda_i^2);
// Mrec[:, i] = (alpha0+2)/2 lambda_i G^-1 v_i with G^-1 = Minv Minv^T (Minv = L^-T of G = W^T W),
// so that mu_i = W Mrec[:, i] = (alpha0+2)/2 lambda_i (W^+)^T v_i.
__global__ void recover_small_kernel(const double* Minv, const double* lam, const float* Vv, int k,
                                     double alpha0, double* alpha_hat, double* Mrec, double* tmp) {
  // tmp[a][i] = sum_b Minv[b][a] v_i[b]  (Minv^T v_i)
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, i = e % k;
    double s = 0.0;
    for (int b = 0; b < k; ++b) s = fma(Minv[b * k + a], (double)Vv[i * k + b], s);
    tmp[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, i = e % k;
    double s = 0.0;
    for (int b = 0; b < k; ++b) s = fma(Minv[a * k + b], tmp[b * k + i], s);
    Mrec[e] = 0.5 * (alpha0 + 2.0) * lam[i] * s;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    alpha_hat[i] = 4.0 * alpha0 * (alpha0 + 1.0) / ((alpha0 + 2.0) * (alpha0 + 2.0) * lam[i] * lam[i]);
}

// ------------------------------------------------------------------ host orchestration
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

int grid_for(const tsk_ctx* ctx, int64_t warps_needed) {
  const int64_t full = (int64_t)ctx->num_sms * 8;
  const int64_t need = (warps_needed + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return (int)std::max<int64_t>(1, std::min(full, need));
}

int check_corpus(const Corpus& c) {
  if (!c.indptr || (c.D > 0 && (!c.idx || !c.cnt))) return TSK_EINVAL;
  if (c.D < 0 || c.V < 1 || c.V > (int64_t(1) << 31) - 1) return TSK_EINVAL;
  return TSK_OK;
}

int run_stats(tsk_ctx* ctx, const Corpus& c, float* mdoc, unsigned long long* counts,
              double* M1acc, float* e) {
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), st));
  if (M1acc) {
    TSK_CUDA(cudaMemsetAsync(M1acc, 0, c.V * sizeof(double), st));
    TSK_CUDA(cudaMemsetAsync(e, 0, c.V * sizeof(float), st));
  }
  if (c.D > 0) {
    doc_stats_kernel<<<grid_for(ctx, c.D), 256, 0, st>>>(c, mdoc, counts, M1acc, e, ctx->status);
    TSK_CHECK_LAUNCH();
  }
  return TSK_OK;
}

// Y = M2^ X for X, Y: [V][cp] (device, padded columns zero).  Yacc may alias Y.
int run_m2_apply(tsk_ctx* ctx, const Corpus& c, const float* mdoc, const unsigned long long* counts,
                 const float* M1, const float* e, double alpha0, const float* X, int cp,
                 float* Y, double* sdot) {
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(Y, 0, (size_t)c.V * cp * sizeof(float), st));
  TSK_CUDA(cudaMemsetAsync(sdot, 0, cp * sizeof(double), st));
  if (c.D > 0) {
    const int grid = grid_for(ctx, c.D);
    if (cp <= 128) m2_docs_kernel<1><<<grid, 256, 0, st>>>(c, mdoc, X, cp, Y);
    else m2_docs_kernel<2><<<grid, 256, 0, st>>>(c, mdoc, X, cp, Y);
    TSK_CHECK_LAUNCH();
  }
  m1_dot_kernel<<<ctx->num_sms, 128, 0, st>>>(M1, X, c.V, cp, sdot);
  TSK_CHECK_LAUNCH();
  m2_finish_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(Y, X, e, M1, sdot, counts,
                                                     alpha0 / (alpha0 + 1.0), c.V, cp, Y);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

struct GramWs {
  double* part;
  int nblk;
};

inline int gram_blocks(const tsk_ctx* ctx, int64_t rows) {
  return (int)std::max<int64_t>(1, min64(ctx->num_sms, (rows + 255) / 256));
}

int run_gram(tsk_ctx* ctx, const float* X, int ldx, const float* Y, int ldy, int64_t rows, int c,
             GramWs gw, double* G) {
  cudaStream_t st = ctx->stream;
  const int c4 = (c + 3) / 4;
  const int groups = (c4 * c4 + 255) / 256;
  const int64_t per = (rows + gw.nblk - 1) / gw.nblk;
  gram_partial_kernel<<<dim3(gw.nblk, groups), 256, 0, st>>>(X, ldx, Y, ldy, rows, c, per, gw.part);
  TSK_CHECK_LAUNCH();
  gram_reduce_kernel<<<(c * c + 255) / 256, 256, 0, st>>>(gw.part, gw.nblk, c, G);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

size_t chol_smem(int c) { return (size_t)c * (c + 1) * sizeof(double); }

int run_chol_inv(tsk_ctx* ctx, const double* G, int c, double shift_scale, double* Minv) {
  const size_t smem = chol_smem(c);
  TSK_CUDA(tsk_smem_attr<chol_inv_kernel>(chol_smem(kMaxWhitenCols)));
  chol_inv_kernel<<<1, 1024, smem, ctx->stream>>>(G, c, shift_scale, Minv, ctx->status);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

int run_rmul(tsk_ctx* ctx, const float* Y, int ldy, int64_t rows, int c, const double* M, int cout,
             float* out, int ldo, int transposed) {
  const size_t smem = (size_t)c * cout * 2 * sizeof(float);
  TSK_CUDA(tsk_smem_attr<rmul_kernel>((size_t)kMaxWhitenCols * kMaxWhitenCols * 2 * sizeof(float)));
  rmul_kernel<<<grid_for(ctx, rows), 256, smem, ctx->stream>>>(Y, ldy, rows, c, M, cout, out, ldo,
                                                               transposed);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

// Orthonormalise the columns of Y [V][cp] (first c columns) in place: shifted Cholesky-QR, then
// two plain Cholesky-QR passes (the shift keeps the first factorisation positive definite for
// any condition number; the plain passes restore orthogonality to rounding level).
int run_orth(tsk_ctx* ctx, float* Y, int64_t V, int c, int cp, GramWs gw, double* G, double* Minv) {
  const double u = 1.1102230246251565e-16;
  const double shift = 11.0 * ((double)V * c + (double)c * (c + 1)) * u;
  int rc;
  for (int pass = 0; pass < 3; ++pass) {
    if ((rc = run_gram(ctx, Y, cp, Y, cp, V, c, gw, G)) != TSK_OK) return rc;
    if ((rc = run_chol_inv(ctx, G, c, pass == 0 ? shift : 0.0, Minv)) != TSK_OK) return rc;
    if ((rc = run_rmul(ctx, Y, cp, V, c, Minv, c, Y, cp, 0)) != TSK_OK) return rc;
  }
  return TSK_OK;
}

}  // namespace lda
}  // namespace tsk

using namespace tsk::lda;
using tsk::Moments3TcArgs;
using tsk::kMoments3TcMaxN;
using tsk::moments3_tc_splits;
using tsk::launch_moments3_tc;

extern "C" int lda_m2_apply(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx,
                            const int32_t* cnt, int64_t D, int64_t V, double alpha0,
                            const float* X, int c, float* Y) {
  if (!ctx || !X || !Y) return TSK_EINVAL;
  Corpus cp_{indptr, idx, cnt, D, V};
  int rc = check_corpus(cp_);
  if (rc != TSK_OK) return rc;
  if (c < 1 || !(alpha0 > 0.0)) return TSK_EINVAL;
  if (c > 256) return TSK_EUNSUPPORTED;
  const int cp = round_up(c, 4);
  WsCarve probe{nullptr, 0};
  probe.take<float>(D);
  probe.take<unsigned long long>(3);
  probe.take<double>(V);
  probe.take<float>(V);
  probe.take<float>(V);
  probe.take<float>((size_t)V * cp);
  probe.take<float>((size_t)V * cp);
  probe.take<double>(cp);
  if ((rc = tsk_ws_reserve(ctx, probe.off + 256)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  float* mdoc = wc.take<float>(D);
  auto* counts = wc.take<unsigned long long>(3);
  double* M1acc = wc.take<double>(V);
  float* M1 = wc.take<float>(V);
  float* e = wc.take<float>(V);
  float* Xp = wc.take<float>((size_t)V * cp);
  float* Yp = wc.take<float>((size_t)V * cp);
  double* sdot = wc.take<double>(cp);
  cudaStream_t st = ctx->stream;
  if ((rc = run_stats(ctx, cp_, mdoc, counts, M1acc, e)) != TSK_OK) return rc;
  m1_finish_kernel<<<ctx->num_sms * 2, 256, 0, st>>>(M1acc, counts, V, M1);
  TSK_CHECK_LAUNCH();
  TSK_CUDA(cudaMemsetAsync(Xp, 0, (size_t)V * cp * sizeof(float), st));
  TSK_CUDA(cudaMemcpy2DAsync(Xp, cp * sizeof(float), X, c * sizeof(float), c * sizeof(float), V,
                             cudaMemcpyDeviceToDevice, st));
  if ((rc = run_m2_apply(ctx, cp_, mdoc, counts, M1, e, alpha0, Xp, cp, Yp, sdot)) != TSK_OK) return rc;
  TSK_CUDA(cudaMemcpy2DAsync(Y, c * sizeof(float), Yp, cp * sizeof(float), c * sizeof(float), V,
                             cudaMemcpyDeviceToDevice, st));
  return TSK_OK;
}

extern "C" int lda_whiten(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx,
                          const int32_t* cnt, int64_t D, int64_t V, int k, double alpha0,
                          const float* Omega, int c, int power_iters, float* W, double* sigma,
                          float* M1_out) {
  if (!ctx || !Omega || !W || !sigma) return TSK_EINVAL;
  Corpus cp_{indptr, idx, cnt, D, V};
  int rc = check_corpus(cp_);
  if (rc != TSK_OK) return rc;
  if (k < 1 || c < k || c > V || power_iters < 0 || power_iters > 64 || !(alpha0 > 0.0))
    return TSK_EINVAL;
  if (c > kMaxWhitenCols) return TSK_EUNSUPPORTED;
  const int cp = round_up(c, 4);
  const int nblk = gram_blocks(ctx, V);
  auto carve = [&](WsCarve& wc, float*& mdoc, unsigned long long*& counts, double*& M1acc,
                   float*& M1, float*& e, float*& Q, float*& Y, double*& sdot, double*& part,
                   double*& G, double*& Minv, double*& evec, double*& evals, double*& Mk) {
    mdoc = wc.take<float>(D);
    counts = wc.take<unsigned long long>(3);
    M1acc = wc.take<double>(V);
    M1 = wc.take<float>(V);
    e = wc.take<float>(V);
    Q = wc.take<float>((size_t)V * cp);
    Y = wc.take<float>((size_t)V * cp);
    sdot = wc.take<double>(cp);
    part = wc.take<double>((size_t)nblk * c * c);
    G = wc.take<double>((size_t)c * c);
    Minv = wc.take<double>((size_t)c * c);
    evec = wc.take<double>((size_t)c * c);
    evals = wc.take<double>(c);
    Mk = wc.take<double>((size_t)c * k);
  };
  float *mdoc, *M1, *e, *Q, *Y;
  unsigned long long* counts;
  double *M1acc, *sdot, *part, *G, *Minv, *evec, *evals, *Mk;
  WsCarve probe{nullptr, 0};
  carve(probe, mdoc, counts, M1acc, M1, e, Q, Y, sdot, part, G, Minv, evec, evals, Mk);
  if ((rc = tsk_ws_reserve(ctx, probe.off + 256)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  carve(wc, mdoc, counts, M1acc, M1, e, Q, Y, sdot, part, G, Minv, evec, evals, Mk);
  cudaStream_t st = ctx->stream;
  GramWs gw{part, nblk};

  if ((rc = run_stats(ctx, cp_, mdoc, counts, M1acc, e)) != TSK_OK) return rc;
  m1_finish_kernel<<<ctx->num_sms * 2, 256, 0, st>>>(M1acc, counts, V, M1);
  TSK_CHECK_LAUNCH();
  if (M1_out) TSK_CUDA(cudaMemcpyAsync(M1_out, M1, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
  // Q <- Omega (padded), Y = M2 Q, then power_iters rounds of Q = orth(Y), Y = M2 Q
  TSK_CUDA(cudaMemsetAsync(Q, 0, (size_t)V * cp * sizeof(float), st));
  TSK_CUDA(cudaMemcpy2DAsync(Q, cp * sizeof(float), Omega, c * sizeof(float), c * sizeof(float), V,
                             cudaMemcpyDeviceToDevice, st));
  for (int it = 0; it <= power_iters; ++it) {
    if ((rc = run_m2_apply(ctx, cp_, mdoc, counts, M1, e, alpha0, Q, cp, Y, sdot)) != TSK_OK) return rc;
    if ((rc = run_orth(ctx, Y, V, c, cp, gw, G, Minv)) != TSK_OK) return rc;
    std::swap(Q, Y);
  }
  // Rayleigh-Ritz: B = Q^T M2 Q, eigenpairs, W = Q U_k diag(sigma)^-1/2
  if ((rc = run_m2_apply(ctx, cp_, mdoc, counts, M1, e, alpha0, Q, cp, Y, sdot)) != TSK_OK) return rc;
  if ((rc = run_gram(ctx, Q, cp, Y, cp, V, c, gw, G)) != TSK_OK) return rc;
  TSK_CUDA(tsk_smem_attr<jacobi_eig_kernel>(chol_smem(kMaxWhitenCols)));
  jacobi_eig_kernel<<<1, 1024, chol_smem(c), st>>>(G, c, 40, evec, evals);
  TSK_CHECK_LAUNCH();
  select_topk_kernel<<<1, 128, 0, st>>>(evec, evals, c, k, sigma, Mk, ctx->status);
  TSK_CHECK_LAUNCH();
  return run_rmul(ctx, Q, cp, V, c, Mk, k, W, k, 0);
}

// Dense whitened third moment; optionally its sketches.
static int whitened_m3_impl(tsk_ctx* ctx, const Corpus& cps, const float* W, int k, double alpha0,
                            float* M3) {
  const int64_t D = cps.D, V = cps.V;
  const int kp = round_up(k, 8);
  const int nb = kp / 8;
  const int nu3 = count_units3(k, kp), nu2 = count_units2(k, kp);
  const int u3p = round_up(nu3, kUnitThreads), u2p = round_up(nu2, kUnitThreads);
  const int tile_split = 4096;
  const int S3d = (int)std::max<int64_t>(1, min64(256, (D + tile_split - 1) / tile_split));
  const int64_t per_d = round_up((int)((D + S3d - 1) / S3d), kTileItems);
  const int S3w = (int)std::max<int64_t>(1, min64(64, (V + 2047) / 2048));
  const int64_t per_w = round_up((int)((V + S3w - 1) / S3w), kTileItems);
  const int nproj = grid_for(ctx, D);
  // the document term of E3 on the tensor cores (3 x TF32, tcgen05) for k <= 160
  const bool tc = round_up(k, 16) <= kMoments3TcMaxN;
  Moments3TcArgs tca{};
  tca.k = k;
  tca.kp = kp;
  tca.N = round_up(k, 16);
  tca.npairs = (long long)k * (k + 1) / 2;
  tca.rows_pad = (tca.npairs + 127) / 128 * 128;
  tca.D = D;
  const int Stc = tc ? moments3_tc_splits((int)tca.npairs, ctx->num_sms, D) : 0;
  auto carve = [&](WsCarve& wc, float*& mdoc, unsigned long long*& counts, float*& Wp, float*& P,
                   float*& R, float*& ce, float*& qpart, int*& units3, int*& unit3_of, int*& units2,
                   int*& unit2_of, float*& part3d, float*& part3w, float*& part2d, float*& part2w,
                   double*& q, double*& E2) {
    mdoc = wc.take<float>(std::max<int64_t>(D, 1));
    counts = wc.take<unsigned long long>(3);
    Wp = wc.take<float>((size_t)V * kp);
    P = wc.take<float>((size_t)std::max<int64_t>(D, 1) * kp);
    R = wc.take<float>((size_t)V * kp);
    ce = wc.take<float>((size_t)V * 2);
    qpart = wc.take<float>((size_t)nproj * kp);
    units3 = wc.take<int>(u3p);
    unit3_of = wc.take<int>((size_t)nb * nb * kp);
    units2 = wc.take<int>(u2p);
    unit2_of = wc.take<int>((size_t)nb * kp);
    part3d = wc.take<float>(tc ? 64 : (size_t)S3d * 64 * u3p);
    tca.part = tc ? wc.take<double>((size_t)Stc * tca.rows_pad * tca.N) : nullptr;
    part3w = wc.take<float>((size_t)S3w * 64 * u3p);
    part2d = wc.take<float>((size_t)S3d * 8 * u2p);
    part2w = wc.take<float>((size_t)S3w * 8 * u2p);
    q = wc.take<double>(k);
    E2 = wc.take<double>((size_t)k * k);
  };
  float *mdoc, *Wp, *P, *R, *ce, *qpart, *part3d, *part3w, *part2d, *part2w;
  unsigned long long* counts;
  int *units3, *unit3_of, *units2, *unit2_of;
  double *q, *E2;
  WsCarve probe{nullptr, 0};
  carve(probe, mdoc, counts, Wp, P, R, ce, qpart, units3, unit3_of, units2, unit2_of, part3d, part3w,
        part2d, part2w, q, E2);
  int rc = tsk_ws_reserve(ctx, probe.off + 256);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  carve(wc, mdoc, counts, Wp, P, R, ce, qpart, units3, unit3_of, units2, unit2_of, part3d, part3w,
        part2d, part2w, q, E2);
  cudaStream_t st = ctx->stream;

  if ((rc = run_stats(ctx, cps, mdoc, counts, nullptr, nullptr)) != TSK_OK) return rc;
  TSK_CUDA(cudaMemsetAsync(Wp, 0, (size_t)V * kp * sizeof(float), st));
  TSK_CUDA(cudaMemcpy2DAsync(Wp, kp * sizeof(float), W, k * sizeof(float), k * sizeof(float), V,
                             cudaMemcpyDeviceToDevice, st));
  TSK_CUDA(cudaMemsetAsync(R, 0, (size_t)V * kp * sizeof(float), st));
  TSK_CUDA(cudaMemsetAsync(ce, 0, (size_t)V * 2 * sizeof(float), st));
  TSK_CUDA(cudaMemsetAsync(units3, 0, u3p * sizeof(int), st));
  TSK_CUDA(cudaMemsetAsync(units2, 0, u2p * sizeof(int), st));
  build_units_kernel<<<nb, 32, 0, st>>>(k, kp, units3, unit3_of, units2, unit2_of);
  TSK_CHECK_LAUNCH();
  if (D > 0) {
    if (kp <= 128) project_kernel<1><<<nproj, 256, 0, st>>>(cps, mdoc, Wp, kp, P, R, ce, qpart);
    else project_kernel<2><<<nproj, 256, 0, st>>>(cps, mdoc, Wp, kp, P, R, ce, qpart);
    TSK_CHECK_LAUNCH();
  } else {
    TSK_CUDA(cudaMemsetAsync(qpart, 0, (size_t)nproj * kp * sizeof(float), st));
  }
  // wedge accumulations
  const size_t smem1 = (size_t)(kTileItems * kp + kTileItems) * sizeof(float);
  const size_t smem2 = (size_t)(2 * kTileItems * kp + kTileItems) * sizeof(float);
  const size_t smem_max = (size_t)(2 * kTileItems * kMaxTopics + kTileItems) * sizeof(float);
  TSK_CUDA(tsk_smem_attr<moments_kernel<3, FROM_DOCS>>(smem_max));
  TSK_CUDA(tsk_smem_attr<moments_kernel<3, FROM_WORDS>>(smem_max));
  TSK_CUDA(tsk_smem_attr<moments_kernel<2, FROM_DOCS>>(smem_max));
  TSK_CUDA(tsk_smem_attr<moments_kernel<2, FROM_WORDS>>(smem_max));
  MomentArgs m3d{units3, u3p, P, nullptr, mdoc, D, per_d, kp, part3d};
  MomentArgs m3w{units3, u3p, Wp, R, ce, V, per_w, kp, part3w};
  MomentArgs m2d{units2, u2p, P, nullptr, mdoc, D, per_d, kp, part2d};
  MomentArgs m2w{units2, u2p, Wp, nullptr, ce, V, per_w, kp, part2w};
  if (tc) {
    tca.P = P;
    tca.mdoc = mdoc;
    tca.status = ctx->status;
    if ((rc = launch_moments3_tc(tca, Stc, st)) != TSK_OK) return rc;
  } else {
    moments_kernel<3, FROM_DOCS><<<dim3(u3p / kUnitThreads, S3d), kUnitThreads, smem1, st>>>(m3d);
    TSK_CHECK_LAUNCH();
  }
  moments_kernel<3, FROM_WORDS><<<dim3(u3p / kUnitThreads, S3w), kUnitThreads, smem2, st>>>(m3w);
  TSK_CHECK_LAUNCH();
  moments_kernel<2, FROM_DOCS><<<dim3(u2p / kUnitThreads, S3d), kUnitThreads, smem1, st>>>(m2d);
  TSK_CHECK_LAUNCH();
  moments_kernel<2, FROM_WORDS><<<dim3(u2p / kUnitThreads, S3w), kUnitThreads, smem1, st>>>(m2w);
  TSK_CHECK_LAUNCH();
  finalize2_kernel<<<k, 128, 0, st>>>(qpart, nproj, part2d, S3d, part2w, S3w, u2p, unit2_of, counts,
                                      k, kp, q, E2);
  TSK_CHECK_LAUNCH();
  finalize3_kernel<<<dim3(k, k), 128, 0, st>>>(part3d, S3d, part3w, S3w, u3p, unit3_of, counts, q,
                                               E2, k, kp, alpha0, M3, tca.part, Stc, tca.rows_pad,
                                               tca.N);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

extern "C" int lda_whitened_m3(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx,
                               const int32_t* cnt, int64_t D, int64_t V, const float* W, int k,
                               double alpha0, float* M3) {
  if (!ctx || !W || !M3) return TSK_EINVAL;
  Corpus cps{indptr, idx, cnt, D, V};
  int rc = check_corpus(cps);
  if (rc != TSK_OK) return rc;
  if (k < 1 || !(alpha0 > 0.0)) return TSK_EINVAL;
  if (k > kMaxTopics) return TSK_EUNSUPPORTED;
  return whitened_m3_impl(ctx, cps, W, k, alpha0, M3);
}

extern "C" int lda_sketch_m3(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx,
                             const int32_t* cnt, int64_t D, int64_t V, const float* W, int k,
                             double alpha0, const int32_t* h, const uint8_t* g, int B, int log2b,
                             float* M3, float* S) {
  if (!h || !g || !S) return TSK_EINVAL;
  int rc = lda_whitened_m3(ctx, indptr, idx, cnt, D, V, W, k, alpha0, M3);
  if (rc != TSK_OK) return rc;
  const int64_t dims[1] = {k};
  return sketch_tensor(ctx, M3, TSK_F32, 1, dims, h, g, B, log2b, S, TSK_C64, 0);
}

extern "C" int lda_recover(tsk_ctx* ctx, const float* W, int64_t V, int k, double alpha0,
                           const double* lambda, const float* Vv, double* alpha_hat,
                           float* mu_hat) {
  if (!ctx || !W || !lambda || !Vv || !alpha_hat || !mu_hat) return TSK_EINVAL;
  if (V < 1 || k < 1 || k > V || !(alpha0 > 0.0)) return TSK_EINVAL;
  if (k > kMaxWhitenCols) return TSK_EUNSUPPORTED;
  const int nblk = gram_blocks(ctx, V);
  WsCarve probe{nullptr, 0};
  probe.take<double>((size_t)nblk * k * k);
  for (int t = 0; t < 4; ++t) probe.take<double>((size_t)k * k);
  int rc = tsk_ws_reserve(ctx, probe.off + 256);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  double* part = wc.take<double>((size_t)nblk * k * k);
  double* G = wc.take<double>((size_t)k * k);
  double* Minv = wc.take<double>((size_t)k * k);
  double* Mrec = wc.take<double>((size_t)k * k);
  double* tmp = wc.take<double>((size_t)k * k);
  cudaStream_t st = ctx->stream;
  if ((rc = run_gram(ctx, W, k, W, k, V, k, GramWs{part, nblk}, G)) != TSK_OK) return rc;
  if ((rc = run_chol_inv(ctx, G, k, 0.0, Minv)) != TSK_OK) return rc;
  recover_small_kernel<<<1, 256, 0, st>>>(Minv, lambda, Vv, k, alpha0, alpha_hat, Mrec, tmp);
  TSK_CHECK_LAUNCH();
  return run_rmul(ctx, W, k, V, k, Mrec, k, mu_hat, (int)V, 1);
}
