// Asymmetric sketches of real tensors (Eq. 1): half spectra, the contraction T^(I,v,w) of
// Prop. 1 with two different vectors (the building block of the fast ALS of Alg. 2), the
// sketched CP loss with its adjoint, and the k x k solve of the ALS update (Eq. 15).
//
// All asymmetric sketches and count sketches are real, so their DFTs are Hermitian and only the
// half spectrum f = 0..b/2 is kept: a length-b real signal is transformed by a length-b/2 complex
// FFT (block_rfft / block_irfft), which also makes b = 2^15 fit one block's shared memory.
// Layouts: half spectra [.][b/2 + 1] complex; factor matrices are stored one component per row,
// X_j[r][i] (row r is the j-th factor vector of component r).
#include "common.cuh"
#include "fft.cuh"
#include "reduce.cuh"

namespace tsk {

constexpr int kMaxRank = 64;
constexpr int kMaxB64 = 64;

template <int LOGB>
constexpr int asym_threads() { return threads_for_logb(LOGB - 1); }

template <int LOGB>
constexpr size_t asym_smem_bytes() {
  return (size_t)(padded_len(1 << (LOGB - 1)) + 1) * sizeof(float2) + 64 * sizeof(float);
}

// Real count sketch s_j,x(t) = sum_{h_j(i) = t} xi_j(i) x_i (Sec. 3.1) into the zeroed signal X.
template <int NT>
__device__ __forceinline__ void scatter_real(float2* X, const float* x, int len, const int32_t* hrow,
                                             const uint8_t* grow, int mask, float scale) {
  for (int i = threadIdx.x; i < len; i += NT) {
    const float v = __ldg(x + i) * scale;
    atomicAdd(&real_at(X, hrow[i] & mask), (grow[i] & 1) ? -v : v);
  }
}

template <int LOGB>
__device__ __forceinline__ void zero_signal(float2* X, float2* last) {
  constexpr int NT = asym_threads<LOGB>();
  for (int i = threadIdx.x; i < padded_len(1 << (LOGB - 1)); i += NT) X[i] = make_float2(0.f, 0.f);
  if (threadIdx.x == 0) *last = make_float2(0.f, 0.f);
  __syncthreads();
}

template <int LOGB>
__device__ __forceinline__ void store_half(float2* dst, const float2* X, const float2* last) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int N = 1 << (LOGB - 1);
  for (int f = threadIdx.x; f < N; f += NT) dst[f] = X[pad_idx(f)];
  if (threadIdx.x == 0) dst[N] = *last;
}

// ------------------------------------------------------------------ half spectra of sketches
// Xh[m] = DFT of the real parts of S[m] (S: [B][b] complex, imaginary parts ignored).
template <int LOGB>
__global__ void __launch_bounds__(asym_threads<LOGB>(), 1) rfft_rows_kernel(const float2* S, float2* Xh) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int b = 1 << LOGB;
  constexpr int N = b / 2;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* last = smem + padded_len(N);
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const float2* src = S + (size_t)blockIdx.x * b;
  for (int t = threadIdx.x; t < N; t += NT)
    X[pad_idx(t)] = make_float2(src[2 * t].x, src[2 * t + 1].x);
  __syncthreads();
  block_rfft<LOGB, NT>(X, last, tw);
  store_half<LOGB>(Xh + (size_t)blockIdx.x * (N + 1), X, last);
}

// ------------------------------------------------------------------ T^(I,v,w), asymmetric
// For output mode o with the other modes p < q: per (vector pair r, sketch m)
//   g = F^-1( Xh o conj(F s_p,V[r]) o conj(F s_q,W[r]) ),  v_i = xi_o(i) g[h_o(i)]  (Prop. 1),
// then the median over the B sketches (Alg. 2) by the last block of r.
struct IvwArgs {
  const float2* Xh;        // [B][N+1] half spectra of the tensor sketches
  const int32_t* h;        // [B][3][nmax]
  const uint8_t* g;
  int nmax, B, K;
  int o, p, q;             // output mode and the two contracted modes
  int n_o, n_p, n_q;
  const float* V;          // [K][n_p]
  const float* W;          // [K][n_q]
  float2* spec;            // [K][B][N+1] workspace: F s_p,V[r]
  float* Vall;             // [K][B][n_o]
  float* Vmed;             // [K][n_o]
  unsigned* counters;      // [K]
};

template <int LOGB>
__global__ void __launch_bounds__(asym_threads<LOGB>(), 1) ivw_kernel(IvwArgs a) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int b = 1 << LOGB;
  constexpr int N = b / 2;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* last = smem + padded_len(N);
  __shared__ float2 tw[kTwEntries];
  __shared__ int s_last;
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, r = blockIdx.y;
  const int32_t* hm = a.h + (size_t)m * 3 * a.nmax;
  const uint8_t* gm = a.g + (size_t)m * 3 * a.nmax;
  float2* spec = a.spec + ((size_t)r * a.B + m) * (N + 1);
  const float2* Xh = a.Xh + (size_t)m * (N + 1);
  // F s_p,v  -> workspace
  zero_signal<LOGB>(X, last);
  scatter_real<NT>(X, a.V + (size_t)r * a.n_p, a.n_p, hm + (size_t)a.p * a.nmax, gm + (size_t)a.p * a.nmax, b - 1, 1.f);
  __syncthreads();
  block_rfft<LOGB, NT>(X, last, tw);
  store_half<LOGB>(spec, X, last);
  __syncthreads();
  // F s_q,w, then Y = Xh conj(F s_p F s_q) in place
  zero_signal<LOGB>(X, last);
  scatter_real<NT>(X, a.W + (size_t)r * a.n_q, a.n_q, hm + (size_t)a.q * a.nmax, gm + (size_t)a.q * a.nmax, b - 1, 1.f);
  __syncthreads();
  block_rfft<LOGB, NT>(X, last, tw);
  for (int f = threadIdx.x; f < N; f += NT)
    X[pad_idx(f)] = cmulconj(Xh[f], cmul(spec[f], X[pad_idx(f)]));
  if (threadIdx.x == 0) *last = cmulconj(Xh[N], cmul(spec[N], *last));
  __syncthreads();
  block_irfft<LOGB, NT, false>(X, last, tw);        // N z: the 1/N is applied at the read-off
  const int32_t* ho = hm + (size_t)a.o * a.nmax;
  const uint8_t* go = gm + (size_t)a.o * a.nmax;
  float* vout = a.Vall + ((size_t)r * a.B + m) * a.n_o;
  constexpr float invN = 1.f / (float)N;
  for (int i = threadIdx.x; i < a.n_o; i += NT) {
    const float v = real_at(X, ho[i] & (b - 1)) * invN;
    vout[i] = (go[i] & 1) ? -v : v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.counters[r], 1u) == (unsigned)(a.B - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // median over the B sketches; each thread sorts its values in a column of the (now free)
  // transform buffer rather than in a local-memory array
  float* scratch = reinterpret_cast<float*>(X);
  const int P = min(NT, 2 * padded_len(N) / a.B);
  if ((int)threadIdx.x < P) {
    float* x = scratch + threadIdx.x;
    for (int i = threadIdx.x; i < a.n_o; i += P) {
      for (int c = 0; c < a.B; ++c) x[c * P] = __ldcg(&a.Vall[((size_t)r * a.B + c) * a.n_o + i]);
      a.Vmed[(size_t)r * a.n_o + i] = small_median_strided(x, a.B, P);
    }
  }
  if (threadIdx.x == 0) a.counters[r] = 0u;
}

// ------------------------------------------------------------------ Alg. 1 as printed (three hashes)
// Rows of `in` ([rows][n]) scaled to unit length into `out` (may alias); a zero or non-finite
// norm is recorded as TSK_ENONFINITE and gives a zero row.  One block per row.
__global__ void __launch_bounds__(256) normalize_rows_kernel(const float* in, float* out, int n,
                                                             int* status) {
  __shared__ float red[33];
  const float* x = in + (size_t)blockIdx.x * n;
  float ss = 0.f;
  for (int i = threadIdx.x; i < n; i += 256) {
    const float v = __ldcg(x + i);
    ss += v * v;
  }
  ss = block_sum<256>(ss, red);
  float inv = 0.f;
  if (!(ss > 0.f) || !isfinite(ss)) {
    if (threadIdx.x == 0) tsk_set_status(status, TSK_ENONFINITE);
  } else {
    inv = 1.f / sqrtf(ss);
  }
  float* y = out + (size_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += 256) y[i] = __ldcg(x + i) * inv;
}

// Selection step: lambda^(m)_tau = sum_i u_i v^(m)_i (= T^(m)(u,u,u) by the linearity of
// Prop. 1) for every sketch m, and lam[tau] = their median.  One block per tau.
__global__ void __launch_bounds__(256) asym_select_kernel(const float* U, const float* Vall, int B,
                                                          int n, float* lam) {
  __shared__ float red[33];
  __shared__ float per[kMaxB64];
  const int tau = blockIdx.x;
  const float* u = U + (size_t)tau * n;
  for (int m = 0; m < B; ++m) {
    const float* v = Vall + ((size_t)tau * B + m) * n;
    float d = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) d += __ldcg(u + i) * __ldcg(v + i);
    d = block_sum<256>(d, red);
    if (threadIdx.x == 0) per[m] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) lam[tau] = small_median(per, B);
}

// tau* = first argmax of lam[0..L), then lambda[r] = lam[tau*], Vout[r] = U[tau*], tau_out[r],
// and the deflation weight defl = lam[tau*].  One block.
__global__ void __launch_bounds__(256) asym_pick_kernel(const float* lam, int L, const float* U,
                                                        int n, int r, double* lambda, float* Vout,
                                                        int32_t* tau_out, float* defl) {
  __shared__ int s_tau;
  if (threadIdx.x == 0) {
    int best = 0;
    float bv = __ldcg(lam);
    for (int t = 1; t < L; ++t) {
      const float v = __ldcg(lam + t);
      if (v > bv) { bv = v; best = t; }
    }
    s_tau = best;
    lambda[r] = (double)bv;
    if (tau_out) tau_out[r] = best;
    *defl = bv;
  }
  __syncthreads();
  const float* u = U + (size_t)s_tau * n;
  for (int i = threadIdx.x; i < n; i += 256) Vout[(size_t)r * n + i] = __ldcg(u + i);
}

// Deflation of sketch m = blockIdx.x in the frequency domain:
//   Xh[m] -= defl * F s_1,u o F s_2,u o F s_3,u   (Eq. 4; the half spectra of the real sketches),
// the product accumulated in dspec[m] ([B][N+1] workspace).
template <int LOGB>
__global__ void __launch_bounds__(asym_threads<LOGB>(), 1) asym_deflate_kernel(
    float2* Xh, const int32_t* h, const uint8_t* g, int nmax, const float* u, int n,
    const float* defl, float2* dspec) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int b = 1 << LOGB;
  constexpr int N = b / 2;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* last = smem + padded_len(N);
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x;
  const int32_t* hm = h + (size_t)m * 3 * nmax;
  const uint8_t* gm = g + (size_t)m * 3 * nmax;
  float2* P = dspec + (size_t)m * (N + 1);
  float2* Xm = Xh + (size_t)m * (N + 1);
  const float lam = __ldcg(defl);
  for (int j = 0; j < 3; ++j) {
    zero_signal<LOGB>(X, last);
    scatter_real<NT>(X, u, n, hm + (size_t)j * nmax, gm + (size_t)j * nmax, b - 1, 1.f);
    __syncthreads();
    block_rfft<LOGB, NT>(X, last, tw);
    for (int f = threadIdx.x; f <= N; f += NT) {
      const float2 z = f < N ? X[pad_idx(f)] : *last;
      if (j == 0) P[f] = z;
      else if (j == 1) P[f] = cmul(P[f], z);
      else Xm[f] = csub(Xm[f], cscale(cmul(P[f], z), lam));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ sketched CP loss
// L = (1/B) sum_m || s_T^(m) - sum_r lam_r s^(m)_{a_r (x) b_r (x) c_r} ||^2,
// s_{a(x)b(x)c} = s_1,a * s_2,b * s_3,c (Eq. 4).  With half spectra P_rj = F s_j,(X_j[r]),
// R = F s_T - sum_r lam_r P_r1 P_r2 P_r3, and Parseval with the Hermitian weights
// w_0 = w_{b/2} = 1, w_f = 2 otherwise:  L = (1/(B b)) sum_m sum_f w_f |R_f|^2.
// Adjoint: dL/dX_j[r][i] = -(2 lam_r / B) sum_m xi_j(i) (F^-1(R o conj(P_rj' P_rj'')))[h_j(i)],
//          dL/dlam_r     = -(2/(B b)) sum_m sum_f w_f Re(R_f conj(P_r1 P_r2 P_r3)_f).
struct CpArgs {
  const float2* Xh;        // [B][N+1] half spectra of the tensor sketches
  const int32_t* h;        // [B][3][nmax]
  const uint8_t* g;
  int nmax, B, R;
  int n[3];
  const float* lam;        // [R]
  const float* F[3];       // factors X_j: [R][n_j]
  float2* P;               // [R][B][3][N+1] workspace
  float2* Res;             // [B][N+1] workspace: residual spectra
  float* loss;             // [1] (accumulated)
  float* grad_lam;         // [R] (accumulated) or NULL
  float* grad[3];          // [R][n_j] (accumulated) or NULL
};

// P[r][m][j] = F s_j,(X_j[r]); grid (B, R, 3)
template <int LOGB>
__global__ void __launch_bounds__(asym_threads<LOGB>(), 1) cp_spectra_kernel(CpArgs a) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int b = 1 << LOGB;
  constexpr int N = b / 2;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* last = smem + padded_len(N);
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, r = blockIdx.y, j = blockIdx.z;
  zero_signal<LOGB>(X, last);
  scatter_real<NT>(X, a.F[j] + (size_t)r * a.n[j], a.n[j], a.h + ((size_t)m * 3 + j) * a.nmax,
                   a.g + ((size_t)m * 3 + j) * a.nmax, b - 1, 1.f);
  __syncthreads();
  block_rfft<LOGB, NT>(X, last, tw);
  store_half<LOGB>(a.P + (((size_t)r * a.B + m) * 3 + j) * (N + 1), X, last);
}

// Residual spectra and the loss; grid (B, chunks of the N + 1 frequencies), 256 threads.
__global__ void __launch_bounds__(256) cp_residual_kernel(CpArgs a, int N) {
  __shared__ float red[40];
  const int m = blockIdx.x;
  const float inv = 1.f / ((float)a.B * (float)(2 * N));
  float acc = 0.f;
  for (int f = blockIdx.y * blockDim.x + threadIdx.x; f <= N; f += gridDim.y * blockDim.x) {
    float2 M = make_float2(0.f, 0.f);
    for (int r = 0; r < a.R; ++r) {
      const float2* Pr = a.P + (((size_t)r * a.B + m) * 3) * (N + 1);
      const float2 prod = cmul(cmul(Pr[f], Pr[(N + 1) + f]), Pr[2 * (N + 1) + f]);
      M = cadd(M, cscale(prod, a.lam[r]));
    }
    const float2 Rf = csub(a.Xh[(size_t)m * (N + 1) + f], M);
    a.Res[(size_t)m * (N + 1) + f] = Rf;
    const float w = (f == 0 || f == N) ? 1.f : 2.f;
    acc += w * (Rf.x * Rf.x + Rf.y * Rf.y);
  }
  acc = block_sum<256>(acc, red);
  if (threadIdx.x == 0) atomicAdd(a.loss, acc * inv);
}

// Adjoint for mode j of component r against sketch m; grid (B, R, 3).
template <int LOGB>
__global__ void __launch_bounds__(asym_threads<LOGB>(), 1) cp_adjoint_kernel(CpArgs a) {
  constexpr int NT = asym_threads<LOGB>();
  constexpr int b = 1 << LOGB;
  constexpr int N = b / 2;
  extern __shared__ float2 smem[];
  float2* X = smem;
  float2* last = smem + padded_len(N);
  float* red = reinterpret_cast<float*>(last + 1);
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, r = blockIdx.y, j = blockIdx.z;
  const int j1 = j == 0 ? 1 : 0, j2 = j == 2 ? 1 : 2;
  const float2* Pr = a.P + (((size_t)r * a.B + m) * 3) * (N + 1);
  const float2* Rm = a.Res + (size_t)m * (N + 1);
  float dl = 0.f;
  for (int f = threadIdx.x; f <= N; f += NT) {
    const float2 Rf = Rm[f];
    const float2 pq = cmul(Pr[j1 * (N + 1) + f], Pr[j2 * (N + 1) + f]);
    const float2 Y = cmulconj(Rf, pq);
    if (f < N) X[pad_idx(f)] = Y; else *last = Y;
    if (j == 0 && a.grad_lam) {
      const float2 full = cmul(pq, Pr[f]);
      const float w = (f == 0 || f == N) ? 1.f : 2.f;
      dl += w * (Rf.x * full.x + Rf.y * full.y);           // Re(R conj(P1 P2 P3))
    }
  }
  __syncthreads();
  if (j == 0 && a.grad_lam) {
    dl = block_sum<NT>(dl, red);
    if (threadIdx.x == 0) atomicAdd(&a.grad_lam[r], -2.f * dl / ((float)a.B * (float)b));
  }
  block_irfft<LOGB, NT, false>(X, last, tw);        // N z: the 1/N goes into `scale`
  const int32_t* hj = a.h + ((size_t)m * 3 + j) * a.nmax;
  const uint8_t* gj = a.g + ((size_t)m * 3 + j) * a.nmax;
  const float scale = -2.f * a.lam[r] / ((float)a.B * (float)N);
  float* gr = a.grad[j] + (size_t)r * a.n[j];
  for (int i = threadIdx.x; i < a.n[j]; i += NT) {
    const float v = real_at(X, hj[i] & (b - 1));
    atomicAdd(&gr[i], scale * ((gj[i] & 1) ? -v : v));
  }
}

// ------------------------------------------------------------------ ALS solve (Eq. 15)
// out = G^-1 M with G = (P P^T) o (Q Q^T) (k x k, symmetric positive definite for independent
// factor columns), then lambda_r = ||out[r]|| and out[r] /= lambda_r.  M: [K][n] rows are the
// sketched T^(I, p_r, q_r).  One block; FP64 Gram matrix and Cholesky factorisation.
__global__ void __launch_bounds__(256) als_solve_kernel(const float* M, const float* P, const float* Q,
                                                        int K, int n, int np, int nq, float* out,
                                                        float* lam, int* status) {
  __shared__ double G[kMaxRank * kMaxRank];
  __shared__ double red[33];
  const int tid = threadIdx.x;
  for (int e = tid; e < K * K; e += blockDim.x) {
    const int r = e / K, s = e % K;
    double pp = 0.0, qq = 0.0;
    for (int i = 0; i < np; ++i) pp += (double)P[(size_t)r * np + i] * P[(size_t)s * np + i];
    for (int i = 0; i < nq; ++i) qq += (double)Q[(size_t)r * nq + i] * Q[(size_t)s * nq + i];
    G[e] = pp * qq;
  }
  __syncthreads();
  // Cholesky G = L L^T in place (lower triangle), column by column
  for (int c = 0; c < K; ++c) {
    if (tid == 0) {
      double d = G[c * K + c];
      for (int t = 0; t < c; ++t) d -= G[c * K + t] * G[c * K + t];
      if (!(d > 0.0)) {
        tsk_set_status(status, TSK_ENONFINITE);
        d = 1e-300;
      }
      G[c * K + c] = sqrt(d);
    }
    __syncthreads();
    for (int rr = c + 1 + tid; rr < K; rr += blockDim.x) {
      double v = G[rr * K + c];
      for (int t = 0; t < c; ++t) v -= G[rr * K + t] * G[c * K + t];
      G[rr * K + c] = v / G[c * K + c];
    }
    __syncthreads();
  }
  // solve G X = M column by column of M (each i independent)
  for (int i = tid; i < n; i += blockDim.x) {
    double y[kMaxRank];
    for (int r = 0; r < K; ++r) {
      double v = M[(size_t)r * n + i];
      for (int t = 0; t < r; ++t) v -= G[r * K + t] * y[t];
      y[r] = v / G[r * K + r];
    }
    for (int r = K - 1; r >= 0; --r) {
      double v = y[r];
      for (int t = r + 1; t < K; ++t) v -= G[t * K + r] * y[t];
      y[r] = v / G[r * K + r];
    }
    for (int r = 0; r < K; ++r) out[(size_t)r * n + i] = (float)y[r];
  }
  __syncthreads();
  __threadfence_block();
  for (int r = 0; r < K; ++r) {
    double ss = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
      const double v = out[(size_t)r * n + i];
      ss += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      red[32] = sqrt(tot);
      lam[r] = (float)red[32];
    }
    __syncthreads();
    const double nr = red[32];
    const float inv = nr > 0.0 ? (float)(1.0 / nr) : 0.f;
    for (int i = tid; i < n; i += blockDim.x) out[(size_t)r * n + i] *= inv;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ launch helpers

template <int LOGB>
static int launch_rfft_t(const float2* S, float2* Xh, int B, cudaStream_t st) {
  constexpr size_t smem = asym_smem_bytes<LOGB>();
  TSK_CUDA(tsk_smem_attr<rfft_rows_kernel<LOGB>>(smem));
  rfft_rows_kernel<LOGB><<<B, asym_threads<LOGB>(), smem, st>>>(S, Xh);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <int LOGB>
static int launch_ivw_t(const IvwArgs& a, cudaStream_t st) {
  constexpr size_t smem = asym_smem_bytes<LOGB>();
  TSK_CUDA(tsk_smem_attr<ivw_kernel<LOGB>>(smem));
  ivw_kernel<LOGB><<<dim3(a.B, a.K), asym_threads<LOGB>(), smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <int LOGB>
static int launch_cp_t(const CpArgs& a, bool with_grad, cudaStream_t st) {
  constexpr size_t smem = asym_smem_bytes<LOGB>();
  constexpr int N = 1 << (LOGB - 1);
  TSK_CUDA(tsk_smem_attr<cp_spectra_kernel<LOGB>>(smem));
  cp_spectra_kernel<LOGB><<<dim3(a.B, a.R, 3), asym_threads<LOGB>(), smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  const int chunks = (N + 1 + 255) / 256 < 64 ? (N + 1 + 255) / 256 : 64;
  cp_residual_kernel<<<dim3(a.B, chunks), 256, 0, st>>>(a, N);
  TSK_CHECK_LAUNCH();
  if (with_grad) {
    TSK_CUDA(tsk_smem_attr<cp_adjoint_kernel<LOGB>>(smem));
    cp_adjoint_kernel<LOGB><<<dim3(a.B, a.R, 3), asym_threads<LOGB>(), smem, st>>>(a);
    TSK_CHECK_LAUNCH();
  }
  return TSK_OK;
}

#define TSK_ASYM_DISPATCH(log2b, call)          \
  switch (log2b) {                               \
    case 9: return call<9>;                      \
    case 10: return call<10>;                    \
    case 11: return call<11>;                    \
    case 12: return call<12>;                    \
    case 13: return call<13>;                    \
    case 14: return call<14>;                    \
    case 15: return call<15>;                    \
    default: return TSK_EUNSUPPORTED;            \
  }

static int launch_rfft(int log2b, const float2* S, float2* Xh, int B, cudaStream_t st) {
  switch (log2b) {
    case 9: return launch_rfft_t<9>(S, Xh, B, st);
    case 10: return launch_rfft_t<10>(S, Xh, B, st);
    case 11: return launch_rfft_t<11>(S, Xh, B, st);
    case 12: return launch_rfft_t<12>(S, Xh, B, st);
    case 13: return launch_rfft_t<13>(S, Xh, B, st);
    case 14: return launch_rfft_t<14>(S, Xh, B, st);
    case 15: return launch_rfft_t<15>(S, Xh, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

static int launch_ivw(int log2b, const IvwArgs& a, cudaStream_t st) {
  switch (log2b) {
    case 9: return launch_ivw_t<9>(a, st);
    case 10: return launch_ivw_t<10>(a, st);
    case 11: return launch_ivw_t<11>(a, st);
    case 12: return launch_ivw_t<12>(a, st);
    case 13: return launch_ivw_t<13>(a, st);
    case 14: return launch_ivw_t<14>(a, st);
    case 15: return launch_ivw_t<15>(a, st);
    default: return TSK_EUNSUPPORTED;
  }
}

template <int LOGB>
static int launch_asym_deflate_t(float2* Xh, const int32_t* h, const uint8_t* g, int nmax,
                                 const float* u, int n, const float* defl, float2* dspec, int B,
                                 cudaStream_t st) {
  constexpr size_t smem = asym_smem_bytes<LOGB>();
  TSK_CUDA(tsk_smem_attr<asym_deflate_kernel<LOGB>>(smem));
  asym_deflate_kernel<LOGB><<<B, asym_threads<LOGB>(), smem, st>>>(Xh, h, g, nmax, u, n, defl, dspec);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

static int launch_asym_deflate(int log2b, float2* Xh, const int32_t* h, const uint8_t* g, int nmax,
                               const float* u, int n, const float* defl, float2* dspec, int B,
                               cudaStream_t st) {
  switch (log2b) {
    case 9: return launch_asym_deflate_t<9>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 10: return launch_asym_deflate_t<10>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 11: return launch_asym_deflate_t<11>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 12: return launch_asym_deflate_t<12>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 13: return launch_asym_deflate_t<13>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 14: return launch_asym_deflate_t<14>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    case 15: return launch_asym_deflate_t<15>(Xh, h, g, nmax, u, n, defl, dspec, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

static int launch_cp(int log2b, const CpArgs& a, bool with_grad, cudaStream_t st) {
  switch (log2b) {
    case 9: return launch_cp_t<9>(a, with_grad, st);
    case 10: return launch_cp_t<10>(a, with_grad, st);
    case 11: return launch_cp_t<11>(a, with_grad, st);
    case 12: return launch_cp_t<12>(a, with_grad, st);
    case 13: return launch_cp_t<13>(a, with_grad, st);
    case 14: return launch_cp_t<14>(a, with_grad, st);
    case 15: return launch_cp_t<15>(a, with_grad, st);
    default: return TSK_EUNSUPPORTED;
  }
}

}  // namespace tsk

using namespace tsk;

extern "C" int sketch_rfft(tsk_ctx* ctx, const float* S, float* Xh, int B, int log2b) {
  if (!ctx || !S || !Xh || B < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 9 || log2b > 15) return TSK_EUNSUPPORTED;
  return launch_rfft(log2b, reinterpret_cast<const float2*>(S), reinterpret_cast<float2*>(Xh), B,
                     ctx->stream);
}

extern "C" int contract_ivw(tsk_ctx* ctx, const float* Xh, const int32_t* h, const uint8_t* g,
                            int B, int log2b, const int64_t* dims_host, int mode, const float* V,
                            const float* W, int K, float* Vmed, float* Vall) {
  if (!ctx || !Xh || !h || !g || !dims_host || !V || !W || !Vmed) return TSK_EINVAL;
  if (B < 1 || K < 1 || mode < 0 || mode > 2 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 9 || log2b > 15 || B > 64 || K > 65535) return TSK_EUNSUPPORTED;
  int dims[3];
  int nmax = 0;
  for (int j = 0; j < 3; ++j) {
    if (dims_host[j] < 1) return TSK_EINVAL;
    if (dims_host[j] > 8192) return TSK_EUNSUPPORTED;
    dims[j] = (int)dims_host[j];
    nmax = dims[j] > nmax ? dims[j] : nmax;
  }
  IvwArgs a{};
  a.Xh = reinterpret_cast<const float2*>(Xh);
  a.h = h;
  a.g = g;
  a.nmax = nmax;
  a.B = B;
  a.K = K;
  a.o = mode;
  a.p = mode == 0 ? 1 : 0;
  a.q = mode == 2 ? 1 : 2;
  a.n_o = dims[a.o];
  a.n_p = dims[a.p];
  a.n_q = dims[a.q];
  a.V = V;
  a.W = W;
  a.Vmed = Vmed;
  const size_t N = (size_t)1 << (log2b - 1);
  const size_t need = ws_round((size_t)K * B * (N + 1) * sizeof(float2)) +
                      (Vall ? 0 : ws_round((size_t)K * B * a.n_o * sizeof(float))) +
                      ws_round((size_t)K * sizeof(unsigned));
  int rc = tsk_ws_reserve(ctx, need);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  a.spec = wc.take<float2>((size_t)K * B * (N + 1));
  a.Vall = Vall ? Vall : wc.take<float>((size_t)K * B * a.n_o);
  a.counters = wc.take<unsigned>(K);
  TSK_CUDA(cudaMemsetAsync(a.counters, 0, K * sizeof(unsigned), ctx->stream));
  return launch_ivw(log2b, a, ctx->stream);
}

extern "C" int cp_sketch_loss(tsk_ctx* ctx, const float* Xh, const int32_t* h, const uint8_t* g,
                              int B, int log2b, const int64_t* dims_host, int R, const float* lam,
                              const float* A, const float* Bf, const float* C, float* loss,
                              float* grad_lam, float* grad_A, float* grad_B, float* grad_C) {
  if (!ctx || !Xh || !h || !g || !dims_host || !lam || !A || !Bf || !C || !loss) return TSK_EINVAL;
  if (B < 1 || R < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  const bool with_grad = grad_lam || grad_A || grad_B || grad_C;
  if (with_grad && !(grad_lam && grad_A && grad_B && grad_C)) return TSK_EINVAL;
  if (log2b < 9 || log2b > 15 || R > 4096) return TSK_EUNSUPPORTED;
  CpArgs a{};
  int nmax = 0;
  for (int j = 0; j < 3; ++j) {
    if (dims_host[j] < 1) return TSK_EINVAL;
    if (dims_host[j] > 8192) return TSK_EUNSUPPORTED;
    a.n[j] = (int)dims_host[j];
    nmax = a.n[j] > nmax ? a.n[j] : nmax;
  }
  a.Xh = reinterpret_cast<const float2*>(Xh);
  a.h = h;
  a.g = g;
  a.nmax = nmax;
  a.B = B;
  a.R = R;
  a.lam = lam;
  a.F[0] = A;
  a.F[1] = Bf;
  a.F[2] = C;
  a.loss = loss;
  a.grad_lam = grad_lam;
  a.grad[0] = grad_A;
  a.grad[1] = grad_B;
  a.grad[2] = grad_C;
  const size_t N = (size_t)1 << (log2b - 1);
  const size_t need = ws_round((size_t)R * B * 3 * (N + 1) * sizeof(float2)) +
                      ws_round((size_t)B * (N + 1) * sizeof(float2));
  int rc = tsk_ws_reserve(ctx, need);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  a.P = wc.take<float2>((size_t)R * B * 3 * (N + 1));
  a.Res = wc.take<float2>((size_t)B * (N + 1));
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
  if (with_grad) {
    TSK_CUDA(cudaMemsetAsync(grad_lam, 0, R * sizeof(float), st));
    TSK_CUDA(cudaMemsetAsync(grad_A, 0, (size_t)R * a.n[0] * sizeof(float), st));
    TSK_CUDA(cudaMemsetAsync(grad_B, 0, (size_t)R * a.n[1] * sizeof(float), st));
    TSK_CUDA(cudaMemsetAsync(grad_C, 0, (size_t)R * a.n[2] * sizeof(float), st));
  }
  return launch_cp(log2b, a, with_grad, st);
}

extern "C" int cp_als_solve(tsk_ctx* ctx, const float* M, const float* P, const float* Q, int K,
                            int64_t n, int64_t np, int64_t nq, float* out, float* lam) {
  if (!ctx || !M || !P || !Q || !out || !lam || K < 1 || n < 1 || np < 1 || nq < 1)
    return TSK_EINVAL;
  if (K > kMaxRank || n > (1 << 24) || np > (1 << 24) || nq > (1 << 24)) return TSK_EUNSUPPORTED;
  als_solve_kernel<<<1, 256, 0, ctx->stream>>>(M, P, Q, K, (int)n, (int)np, (int)nq, out, lam,
                                               ctx->status);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

extern "C" int robust_power_method_asym(tsk_ctx* ctx, const float* S, const int32_t* h,
                                        const uint8_t* g, int B, int log2b, int64_t n, int k,
                                        int L, int T, const float* U0, double* lambda,
                                        float* Vout, int32_t* tau_star, float* lam_all_out,
                                        float* U_iters) {
  if (!ctx || !S || !h || !g) return TSK_EINVAL;
  if (k < 0 || T < 1 || B < 1 || L < 1 || n < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 9 || log2b > 15 || B > kMaxB64 || n > 8192 || L > 65535) return TSK_EUNSUPPORTED;
  if (k == 0) return TSK_OK;
  if (!U0 || !lambda || !Vout) return TSK_EINVAL;
  const size_t N = (size_t)1 << (log2b - 1);
  auto carve = [&](WsCarve& wc, float2*& Xh, float2*& spec, float2*& dspec, float*& Vall,
                   float*& Ua, float*& Ub, float*& lam, float*& defl, unsigned*& counters) {
    Xh = wc.take<float2>((size_t)B * (N + 1));
    spec = wc.take<float2>((size_t)L * B * (N + 1));
    dspec = wc.take<float2>((size_t)B * (N + 1));
    Vall = wc.take<float>((size_t)L * B * n);
    Ua = wc.take<float>((size_t)L * n);
    Ub = wc.take<float>((size_t)L * n);
    lam = lam_all_out ? lam_all_out : wc.take<float>((size_t)k * L);
    defl = wc.take<float>(1);
    counters = wc.take<unsigned>(L);
  };
  float2 *Xh, *spec, *dspec;
  float *Vall, *Ua, *Ub, *lam, *defl;
  unsigned* counters;
  WsCarve probe{nullptr, 0};
  carve(probe, Xh, spec, dspec, Vall, Ua, Ub, lam, defl, counters);
  int rc = tsk_ws_reserve(ctx, probe.off + 256);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  carve(wc, Xh, spec, dspec, Vall, Ua, Ub, lam, defl, counters);
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(counters, 0, L * sizeof(unsigned), st));
  if ((rc = launch_rfft(log2b, reinterpret_cast<const float2*>(S), Xh, B, st)) != TSK_OK) return rc;
  IvwArgs a{};
  a.Xh = Xh;
  a.h = h;
  a.g = g;
  a.nmax = (int)n;
  a.B = B;
  a.K = L;
  a.o = 0;
  a.p = 1;
  a.q = 2;
  a.n_o = a.n_p = a.n_q = (int)n;
  a.spec = spec;
  a.Vall = Vall;
  a.counters = counters;
  for (int r = 0; r < k; ++r) {
    normalize_rows_kernel<<<L, 256, 0, st>>>(U0 + (size_t)r * L * n, Ua, (int)n, ctx->status);
    TSK_CHECK_LAUNCH();
    const float* cur = Ua;
    for (int t = 0; t < T; ++t) {
      a.V = cur;
      a.W = cur;
      a.Vmed = Ub;
      if ((rc = launch_ivw(log2b, a, st)) != TSK_OK) return rc;
      float* next = U_iters ? U_iters + (((size_t)r * T + t) * L) * n : Ua;
      normalize_rows_kernel<<<L, 256, 0, st>>>(Ub, next, (int)n, ctx->status);
      TSK_CHECK_LAUNCH();
      cur = next;
    }
    // selection with the per-sketch values of the final iterates
    a.V = cur;
    a.W = cur;
    a.Vmed = Ub;
    if ((rc = launch_ivw(log2b, a, st)) != TSK_OK) return rc;
    float* lam_r = lam + (size_t)r * L;
    asym_select_kernel<<<L, 256, 0, st>>>(cur, Vall, B, (int)n, lam_r);
    TSK_CHECK_LAUNCH();
    asym_pick_kernel<<<1, 256, 0, st>>>(lam_r, L, cur, (int)n, r, lambda, Vout, tau_star, defl);
    TSK_CHECK_LAUNCH();
    if ((rc = launch_asym_deflate(log2b, Xh, h, g, (int)n, Vout + (size_t)r * n, (int)n, defl,
                                  dspec, B, st)) != TSK_OK)
      return rc;
  }
  return TSK_OK;
}
