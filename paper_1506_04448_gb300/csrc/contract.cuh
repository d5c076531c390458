// Fused sketched contractions against B colliding sketches (Prop. 1, App. B).
//
// One thread block handles one (vector tau, sketch m) pair entirely on chip:
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
// The last block to finish for a given tau (arrival counter) takes the median over the B
// sketches (Alg. 1) and, in a power step, normalises it into the next iterate.
//
// MODE_UUU evaluates T^(m)(u,u,u) directly (App. B, Eq. 13) after step 2:
//   (1/b) sum_f Re(FS[f] conj(U_f^3/6 + V'_f U_f/2)) + 1/3 Re(sum_i S[3h_i] conj(s_i)^3 u_i^3).
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
  unsigned* counters;    // [L]       arrival counters, zero between launches
  int* status;
};

template <int LOGB>
constexpr size_t contract_smem_bytes() {
  return (size_t)(padded_len(1 << LOGB) + padded_len(1 << (LOGB - 1))) * sizeof(float2) +
         64 * sizeof(float);
}

template <int LOGB, int MODE>
__global__ void __launch_bounds__(threads_for_logb(LOGB), 1) contract_kernel(ContractArgs a) {
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int b = 1 << LOGB;
  constexpr int hb = b / 2;
  extern __shared__ float2 smem[];
  float2* A = smem;                                  // padded, length b
  float2* Eb = smem + padded_len(b);                 // padded, length b/2
  float* red = reinterpret_cast<float*>(Eb + padded_len(hb));
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int m = blockIdx.x, tau = blockIdx.y;
  const int n = a.n;
  const int32_t* hm = a.h + (size_t)m * n;
  const uint8_t* gm = a.g + (size_t)m * n;
  const float* u = a.U + (size_t)tau * n;

  float uscale = 1.f;
  if (a.normalize_input) {
    float ss = 0.f;
    for (int i = tid; i < n; i += NT) ss += u[i] * u[i];
    ss = block_sum<NT>(ss, red);
    if (!(ss > 0.f) || !isfinite(ss)) {
      if (tid == 0) tsk_set_status(a.status, TSK_ENONFINITE);
      uscale = 0.f;
    } else {
      uscale = 1.f / sqrtf(ss);
    }
  }

  // 1. zero both buffers, then scatter the count sketches of u.
  for (int i = tid; i < padded_len(b); i += NT) A[i] = make_float2(0.f, 0.f);
  for (int i = tid; i < padded_len(hb); i += NT) Eb[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < n; i += NT) {
    const float x = u[i] * uscale;
    const int hi = hm[i] & (b - 1);
    const int gi = gm[i] & 3;
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hi)]);
    atomicAdd(slot + (gi & 1), (gi & 2) ? -x : x);
    atomicAdd(&Eb[pad_idx(hi & (hb - 1))].x, (gi & 1) ? -x * x : x * x);
  }
  __syncthreads();

  // 2. forward DFTs.
  block_fft<LOGB, NT, -1>(A);
  block_fft<LOGB - 1, NT, -1>(Eb);

  const float2* FSm = a.FS + (size_t)m * b;
  const float2* Sm = a.S + (size_t)m * b;
  constexpr float inv_b = 1.f / (float)b;

  if constexpr (MODE == MODE_IUU) {
    // 3. spectral products (each f < b/2 owns positions f and f + b/2 of A and f of Eb).
    for (int f = tid; f < hb; f += NT) {
      const float2 cu0 = cconj(A[pad_idx(f)]);
      const float2 cu1 = cconj(A[pad_idx(f + hb)]);
      const float2 cv = cconj(Eb[pad_idx(f)]);
      const float2 F0 = FSm[f];
      const float2 F1 = FSm[f + hb];
      A[pad_idx(f)] = cmul(F0, cadd(cmul(cu0, cu0), cv));
      A[pad_idx(f + hb)] = cmul(F1, cadd(cmul(cu1, cu1), cv));
      Eb[pad_idx(f)] = cadd(cmul(F0, cu0), cmul(F1, cu1));
    }
    __syncthreads();
    // 4. inverse DFTs and hashed read-off.
    block_fft<LOGB, NT, +1>(A);
    block_fft<LOGB - 1, NT, +1>(Eb);
    float lam = 0.f;
    float* vout = a.Vall + ((size_t)tau * a.B + m) * n;
    for (int i = tid; i < n; i += NT) {
      const float x = u[i] * uscale;
      const int hi = hm[i] & (b - 1);
      const int gi = gm[i] & 3;
      const float2 g12 = A[pad_idx(hi)];
      const float2 g0 = Eb[pad_idx(hi & (hb - 1))];
      const float2 s3 = Sm[(3 * hi) & (b - 1)];
      const float v = (re_ipow(g12, -gi) * (1.f / 6.f) + re_ipow(g0, -2 * gi) * x * (1.f / 3.f)) * inv_b +
                      re_ipow(s3, -3 * gi) * x * x * (1.f / 3.f);
      vout[i] = v;
      lam += x * v;
    }
    lam = block_sum<NT>(lam, red);
    if (tid == 0) a.lam_all[(size_t)tau * a.B + m] = lam;
  } else {
    float acc = 0.f;
    for (int f = tid; f < b; f += NT) {
      const float2 U = A[pad_idx(f)];
      const float2 V = Eb[pad_idx(f & (hb - 1))];
      const float2 U2 = cmul(U, U);
      const float2 Y = cadd(cscale(cmul(U2, U), 1.f / 6.f), cscale(cmul(V, U), 0.5f));
      const float2 F = FSm[f];
      acc += F.x * Y.x + F.y * Y.y;     // Re(F conj(Y))
    }
    acc *= inv_b;
    for (int i = tid; i < n; i += NT) {
      const float x = u[i] * uscale;
      const int hi = hm[i] & (b - 1);
      const int gi = gm[i] & 3;
      acc += re_ipow(Sm[(3 * hi) & (b - 1)], -3 * gi) * x * x * x * (1.f / 3.f);
    }
    acc = block_sum<NT>(acc, red);
    if (tid == 0) a.lam_all[(size_t)tau * a.B + m] = acc;
  }

  // 5. the last block of this tau takes the medians over the B sketches.
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(&a.counters[tau], 1u);
    s_last = (prev == (unsigned)(a.B - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int B = a.B;
  if (tid == 0) {
    float vals[kMaxB];
    for (int c = 0; c < B; ++c) vals[c] = __ldcg(&a.lam_all[(size_t)tau * B + c]);
    if (a.lam_med) a.lam_med[tau] = small_median(vals, B);
    a.counters[tau] = 0u;
  }
  if constexpr (MODE == MODE_IUU) {
    if (a.Vmed == nullptr && a.Unext == nullptr) return;
    float* dst = a.Vmed ? a.Vmed + (size_t)tau * n : a.Unext + (size_t)tau * n;
    float ss = 0.f;
    for (int i = tid; i < n; i += NT) {
      float vals[kMaxB];
      for (int c = 0; c < B; ++c) vals[c] = __ldcg(&a.Vall[((size_t)tau * B + c) * n + i]);
      const float med = small_median(vals, B);
      dst[i] = med;
      ss += med * med;
    }
    if (a.Unext) {
      ss = block_sum<NT>(ss, red);
      float inv = 0.f;
      if (!(ss > 0.f) || !isfinite(ss)) {
        if (tid == 0) tsk_set_status(a.status, TSK_ENONFINITE);
      } else {
        inv = 1.f / sqrtf(ss);
      }
      float* un = a.Unext + (size_t)tau * n;
      for (int i = tid; i < n; i += NT) un[i] = dst[i] * inv;
    }
  }
}

// Deflation of every sketch by the selected component (Alg. 1, deflation step), fused with the
// selection tau* = first argmax_tau lambda_tau.  One block per sketch m:
//   U = F s~_u,  D = lambda^ U^3  (= F of the sketch of lambda^ u(x)u(x)u, Sec. 3.3),
//   FS[m] -= D,  S[m] -= F^-1 D.
struct DeflateArgs {
  float2* FS;
  float2* S;
  const int32_t* h;
  const uint8_t* g;
  int n, B, L;
  const float* Ucur;      // [L][n] final iterates
  const float* lam_med;   // [L]
  int round;
  double* lambda_out;     // [k]
  float* Vout;            // [k][n]
  int32_t* tau_out;       // [k] or NULL
};

template <int LOGB>
constexpr size_t deflate_smem_bytes() {
  return (size_t)padded_len(1 << LOGB) * sizeof(float2);
}

template <int LOGB>
__global__ void __launch_bounds__(threads_for_logb(LOGB), 1) deflate_kernel(DeflateArgs a) {
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int b = 1 << LOGB;
  extern __shared__ float2 smem[];
  float2* A = smem;
  __shared__ int s_best;
  const int tid = threadIdx.x, m = blockIdx.x, n = a.n;
  if (tid == 0) {
    int best = 0;
    for (int t = 1; t < a.L; ++t)
      if (a.lam_med[t] > a.lam_med[best]) best = t;
    s_best = best;
  }
  for (int i = tid; i < padded_len(b); i += NT) A[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int best = s_best;
  const float lam = a.lam_med[best];
  const float* u = a.Ucur + (size_t)best * n;
  if (m == 0) {
    if (tid == 0) {
      a.lambda_out[a.round] = (double)lam;
      if (a.tau_out) a.tau_out[a.round] = best;
    }
    for (int i = tid; i < n; i += NT) a.Vout[(size_t)a.round * n + i] = u[i];
  }
  const int32_t* hm = a.h + (size_t)m * n;
  const uint8_t* gm = a.g + (size_t)m * n;
  for (int i = tid; i < n; i += NT) {
    const int gi = gm[i] & 3;
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hm[i] & (b - 1))]);
    atomicAdd(slot + (gi & 1), (gi & 2) ? -u[i] : u[i]);
  }
  __syncthreads();
  block_fft<LOGB, NT, -1>(A);
  float2* FSm = a.FS + (size_t)m * b;
  for (int f = tid; f < b; f += NT) {
    const float2 U = A[pad_idx(f)];
    const float2 D = cscale(cmul(cmul(U, U), U), lam);
    FSm[f] = csub(FSm[f], D);
    A[pad_idx(f)] = D;
  }
  __syncthreads();
  block_fft<LOGB, NT, +1>(A);
  float2* Sm = a.S + (size_t)m * b;
  constexpr float inv_b = 1.f / (float)b;
  for (int t = tid; t < b; t += NT) Sm[t] = csub(Sm[t], cscale(A[pad_idx(t)], inv_b));
}

// Host launchers (defined in contract.cu).
int launch_contract(int log2b, int mode, const ContractArgs& args, cudaStream_t st);
int launch_deflate(int log2b, const DeflateArgs& args, cudaStream_t st);

}  // namespace tsk
