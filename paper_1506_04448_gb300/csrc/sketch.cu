// Sketch construction: dense tensor sketches (Eq. 1, Eq. 7), batched DFTs of sketches and
// rank-1 sketches by FFT (Eq. 4).
//
// Dense build.  Each thread block owns one sketch m (and, for 64-bit accumulators, one of the
// two complex components) and a slab of the tensor; it privatises the b buckets in shared
// memory, streams its slab with coalesced loads and scatters with shared-memory atomics, then
// adds its histogram to the global sketch with one atomic per non-zero bucket.  Blocks of the
// same slab are adjacent in launch order, so the slab is read from DRAM once and from L2 by
// the other B-1 sketches.  For the colliding sketch only the wedge i <= j <= k is read, each
// entry weighted by kappa in {1, 3, 6} (Sec. 3.3); each entry lands in exactly one component
// because sigma_i sigma_j sigma_k = sqrt(-1)^((g_i + g_j + g_k) mod 4).
#include "common.cuh"
#include "fft.cuh"

namespace tsk {

// number of wedge entries (i <= j <= k < n) whose first index is < i: Tet(n) - Tet(n - i)
__device__ __forceinline__ long long tet(long long x) { return x * (x + 1) * (x + 2) / 6; }
__device__ __forceinline__ long long wedge_before_i(long long n, long long i) {
  return tet(n) - tet(n - i);
}
// linear position of the first entry of wedge row (i, j), j >= i
__device__ __forceinline__ long long wedge_row_start(long long n, long long i, long long j) {
  const long long d = j - i;
  return wedge_before_i(n, i) + d * n - d * (i + j - 1) / 2;
}

template <typename T>
__device__ __forceinline__ void acc_add(T* p, T v) {
  atomicAdd(p, v);
}
template <>
__device__ __forceinline__ void acc_add<long long>(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

struct SymSketchArgs {
  const void* T;
  int n;
  const int32_t* h;   // [B][n]
  const uint8_t* g;   // [B][n]
  int log2b;
  long long W;        // wedge size n(n+1)(n+2)/6
  int nslab;
  void* S;            // [B][b][2] accumulator type
  int log2r;          // the buckets are split into 2^log2r ranges, one block per range
};

template <typename TIn, typename Acc, int PARTS, bool RANGES = false>
__global__ void __launch_bounds__(1024, 1) sketch_sym_kernel(SymSketchArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_i0, s_j0, s_i1, s_j1;
  const int b = 1 << a.log2b;
  const int n = a.n;
  const int mask = b - 1;
  // this block's bucket range [rr br, (rr + 1) br): long sketches do not fit one block's shared
  // memory, so they are built by 2^log2r blocks that each keep the entries of their range
  const int R = RANGES ? 1 << a.log2r : 1;
  const int br = RANGES ? b >> a.log2r : b;
  const int hist_len = (PARTS == 1 ? 2 : 1) * br;
  Acc* hist = reinterpret_cast<Acc*>(sm_raw);
  // packed hash word q_k = 16 h_k + g_k: in q_i + q_j + q_k, bits 4.. carry h_i + h_j + h_k and
  // bits 0..3 carry g_i + g_j + g_k (at most 9), so one add gives bucket and sign exponent
  uint32_t* qs = reinterpret_cast<uint32_t*>(sm_raw + (size_t)hist_len * sizeof(Acc));
  const int m = blockIdx.x / (PARTS * R);
  const int part = (blockIdx.x / R) % PARTS;
  const int rr = blockIdx.x % R;
  const int shift_r = a.log2b - a.log2r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < hist_len; i += nt) hist[i] = (Acc)0;
  for (int i = tid; i < n; i += nt)
    qs[i] = ((uint32_t)(a.h[(size_t)m * n + i] & mask) << 4) | (uint32_t)(a.g[(size_t)m * n + i] & 3);

  // this block owns the wedge rows (i <= j) whose first entry lies in [e0, e1)
  const TIn* T = static_cast<const TIn*>(a.T);
  const long long per_slab = (a.W + a.nslab - 1) / a.nslab;
  const long long e0 = (long long)blockIdx.y * per_slab;
  const long long e1 = min(a.W, e0 + per_slab);
  if (tid < 2) {
    // first row whose start is >= e (e = e0 for thread 0, e1 for thread 1)
    const long long e = tid == 0 ? e0 : e1;
    int lo = 0, hi = n;  // largest i with wedge_before_i(i) <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wedge_before_i(n, mid) <= e) lo = mid; else hi = mid - 1;
    }
    int i = lo, jl = lo, jh = n;  // smallest j >= i with row_start(i, j) >= e
    while (jl < jh) {
      const int mid = (jl + jh) >> 1;
      if (wedge_row_start(n, i, mid) >= e) jh = mid; else jl = mid + 1;
    }
    int j = jl;
    if (j == n && i < n) { ++i; j = i; }   // (n, n) marks the end of the wedge
    if (tid == 0) { s_i0 = i; s_j0 = j; } else { s_i1 = i; s_j1 = j; }
  }
  __syncthreads();

  // rows are dealt to the warps round-robin (neighbouring rows have similar lengths); the
  // block's rows are those from (s_i0, s_j0) up to, not including, (s_i1, s_j1)
  const int nw = nt >> 5, w = tid >> 5, lane = tid & 31;
  const int i1 = s_i1, j1 = s_j1;
  int i = s_i0, j = s_j0;
  // advance (i, j) by `adv` rows in the order (0,0), (0,1), ..., (0,n-1), (1,1), ...
  auto advance = [n](int& ii, int& jj, int adv) {
    while (adv > 0 && ii < n) {
      const int left = n - jj;
      if (adv < left) { jj += adv; adv = 0; }
      else { adv -= left; ++ii; jj = ii; }
    }
  };
  advance(i, j, w);
  while (i < n && (i < i1 || (i == i1 && j < j1))) {
    const TIn* row = T + ((size_t)i * n + j) * (size_t)n;
    const uint32_t qij = qs[i] + qs[j];
    const Acc kap_diag = (Acc)((i == j) ? 1 : 3);   // kappa at k == j
    const Acc kap_off = (Acc)((i == j) ? 3 : 6);    // kappa at k > j
    constexpr int kU = 4;   // loads in flight per lane before the dependent atomics
    for (int k0 = j + lane; k0 < n; k0 += 32 * kU) {
      TIn x[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int k = k0 + 32 * q;
        x[q] = k < n ? __ldcg(row + k) : (TIn)0;
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int k = k0 + 32 * q;
        if (k >= n) break;
        const uint32_t sq = qij + qs[k];
        Acc v = (Acc)x[q] * (k == j ? kap_diag : kap_off);
        if (sq & 2) v = -v;
        const int t = (int)(sq >> 4) & mask;
        if (RANGES && (t >> shift_r) != rr) continue;
        const int tl = RANGES ? t & (br - 1) : t;
        if (PARTS == 1) {
          acc_add<Acc>(&hist[2 * tl + (int)(sq & 1)], v);
        } else if ((int)(sq & 1) == part) {
          acc_add<Acc>(&hist[tl], v);
        }
      }
    }
    advance(i, j, nw);
  }
  __syncthreads();
  Acc* Sg = static_cast<Acc*>(a.S) + (size_t)m * 2 * b + (size_t)2 * rr * br;
  for (int idx = tid; idx < hist_len; idx += nt) {
    const Acc v = hist[idx];
    if (v != (Acc)0) acc_add<Acc>(&Sg[PARTS == 1 ? idx : 2 * idx + part], v);
  }
}

struct AsymSketchArgs {
  const void* T;
  int n1, n2, n3, nmax;
  const int32_t* h;   // [B][3][nmax]
  const uint8_t* g;
  int log2b;
  long long rows;     // n1 * n2
  int nslab;
  void* S;            // [B][b][2]
};

template <typename TIn, typename Acc>
__global__ void __launch_bounds__(1024, 1) sketch_asym_kernel(AsymSketchArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int b = 1 << a.log2b;
  Acc* hist = reinterpret_cast<Acc*>(sm_raw);
  int* hs = reinterpret_cast<int*>(sm_raw + (size_t)b * sizeof(Acc));   // [3][nmax]
  uint8_t* gs = reinterpret_cast<uint8_t*>(hs + 3 * a.nmax);
  const int m = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < b; i += nt) hist[i] = (Acc)0;
  for (int i = tid; i < 3 * a.nmax; i += nt) {
    hs[i] = a.h[(size_t)m * 3 * a.nmax + i];
    gs[i] = a.g[(size_t)m * 3 * a.nmax + i] & 1;
  }
  __syncthreads();
  const TIn* T = static_cast<const TIn*>(a.T);
  const long long per_slab = (a.rows + a.nslab - 1) / a.nslab;
  const long long r0 = (long long)blockIdx.y * per_slab;
  const long long r1 = min(a.rows, r0 + per_slab);
  const int nw = nt >> 5, w = tid >> 5, lane = tid & 31;
  const int mask = b - 1;
  const int* h1 = hs;
  const int* h2 = hs + a.nmax;
  const int* h3 = hs + 2 * a.nmax;
  const uint8_t* g1 = gs;
  const uint8_t* g2 = gs + a.nmax;
  const uint8_t* g3 = gs + 2 * a.nmax;
  for (long long r = r0 + w; r < r1; r += nw) {
    const int i = (int)(r / a.n2), j = (int)(r % a.n2);
    const TIn* row = T + (size_t)r * a.n3;
    const int hij = h1[i] + h2[j];
    const int gij = g1[i] + g2[j];
    constexpr int kU = 4;
    for (int k0 = lane; k0 < a.n3; k0 += 32 * kU) {
      TIn x[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int k = k0 + 32 * q;
        x[q] = k < a.n3 ? __ldcg(row + k) : (TIn)0;
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int k = k0 + 32 * q;
        if (k >= a.n3) break;
        Acc v = (Acc)x[q];
        if ((gij + g3[k]) & 1) v = -v;
        acc_add<Acc>(&hist[(hij + h3[k]) & mask], v);
      }
    }
  }
  __syncthreads();
  Acc* Sg = static_cast<Acc*>(a.S) + (size_t)m * 2 * b;
  for (int idx = tid; idx < b; idx += nt) {
    const Acc v = hist[idx];
    if (v != (Acc)0) acc_add<Acc>(&Sg[2 * idx], v);
  }
}

template <typename TIn, typename Acc, int PARTS>
static int launch_sym(const SymSketchArgs& a0, int B, tsk_ctx* ctx) {
  SymSketchArgs a = a0;
  const int b = 1 << a.log2b;
  // fewest bucket ranges whose histogram fits the block's shared memory
  a.log2r = 0;
  size_t smem = 0;
  for (;; ++a.log2r) {
    smem = (size_t)(PARTS == 1 ? 2 : 1) * (b >> a.log2r) * sizeof(Acc) + (size_t)a.n * 4 + 16;
    if (smem <= (size_t)ctx->max_smem_optin || a.log2r >= 4) break;
  }
  const int R = 1 << a.log2r;
  if (smem > (size_t)ctx->max_smem_optin) return TSK_EUNSUPPORTED;
  auto kernel = a.log2r > 0 ? sketch_sym_kernel<TIn, Acc, PARTS, true>
                            : sketch_sym_kernel<TIn, Acc, PARTS, false>;
  TSK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 1024, smem));
  if (per_sm < 1) per_sm = 1;
  // one wave of blocks over the SMs, but no more slabs than ~16k entries each
  long long nslab = ((long long)ctx->num_sms * per_sm) / (B * PARTS * R);
  if (nslab < 1) nslab = 1;
  const long long cap = (a.W + 16383) / 16384;
  if (nslab > cap) nslab = cap < 1 ? 1 : cap;
  if (nslab > 65535) nslab = 65535;
  a.nslab = (int)nslab;
  dim3 grid(B * PARTS * R, (unsigned)nslab);
  kernel<<<grid, 1024, smem, ctx->stream>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <typename TIn, typename Acc>
static int launch_asym(const AsymSketchArgs& a0, int B, tsk_ctx* ctx) {
  AsymSketchArgs a = a0;
  const int b = 1 << a.log2b;
  const size_t smem = (size_t)b * sizeof(Acc) + (size_t)a.nmax * 15 + 16;
  if (smem > (size_t)ctx->max_smem_optin) return TSK_EUNSUPPORTED;
  TSK_CUDA(cudaFuncSetAttribute(sketch_asym_kernel<TIn, Acc>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_asym_kernel<TIn, Acc>,
                                                         1024, smem));
  if (per_sm < 1) per_sm = 1;
  long long nslab = ((long long)ctx->num_sms * per_sm) / B;
  if (nslab < 1) nslab = 1;
  const long long cap = (a.rows * a.n3 + 16383) / 16384;
  if (nslab > cap) nslab = cap < 1 ? 1 : cap;
  if (nslab > 65535) nslab = 65535;
  a.nslab = (int)nslab;
  dim3 grid(B, (unsigned)nslab);
  sketch_asym_kernel<TIn, Acc><<<grid, 1024, smem, ctx->stream>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

// ------------------------------------------------------------------ batched DFT of sketches
template <int LOGB>
__global__ void __launch_bounds__(threads_for_logb(LOGB)) fft_rows_kernel(const float2* in,
                                                                          float2* out, int inverse) {
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int b = 1 << LOGB;
  extern __shared__ float2 smem[];
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const float2* src = in + (size_t)blockIdx.x * b;
  float2* dst = out + (size_t)blockIdx.x * b;
  for (int t = threadIdx.x; t < b; t += NT) smem[pad_idx(t)] = src[t];
  __syncthreads();
  if (inverse) block_fft<LOGB, NT, +1>(smem, tw); else block_fft<LOGB, NT, -1>(smem, tw);
  const float s = inverse ? 1.f / (float)b : 1.f;
  for (int t = threadIdx.x; t < b; t += NT) dst[t] = cscale(smem[pad_idx(t)], s);
}

template <int LOGB>
static int launch_fft_t(const float2* in, float2* out, int B, int inverse, cudaStream_t st) {
  constexpr size_t smem = (size_t)padded_len(1 << LOGB) * sizeof(float2);
  TSK_CUDA(tsk_smem_attr<fft_rows_kernel<LOGB>>(smem));
  fft_rows_kernel<LOGB><<<B, threads_for_logb(LOGB), smem, st>>>(in, out, inverse);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

int launch_fft_batched(int log2b, const float2* in, float2* out, int B, int inverse, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_fft_t<8>(in, out, B, inverse, st);
    case 9: return launch_fft_t<9>(in, out, B, inverse, st);
    case 10: return launch_fft_t<10>(in, out, B, inverse, st);
    case 11: return launch_fft_t<11>(in, out, B, inverse, st);
    case 12: return launch_fft_t<12>(in, out, B, inverse, st);
    case 13: return launch_fft_t<13>(in, out, B, inverse, st);
    case 14: return launch_fft_t<14>(in, out, B, inverse, st);
    default: return TSK_EUNSUPPORTED;
  }
}

// ------------------------------------------------------------------ rank-1 sketches (Eq. 4)
struct Rank1Args {
  long long count;
  const float* w;
  const float* U;
  const float* V;
  const float* W;
  int M;
  int n1, n2, n3, nmax;
  const int32_t* h;   // [B][M][nmax]
  const uint8_t* g;
  int domain;         // 0 time, 1 frequency
  int accumulate;
  float2* S;          // [B][b]
  float2* acc;        // [B][b] workspace: running sum of the spectra
  float2* prod;       // [B][b] workspace: partial product (M = 3)
};

// Count sketch of x (length len) with hash row hrow / sign row grow into the zeroed buffer A.
// Colliding: sigma = sqrt(-1)^g.  Asymmetric: xi = 1 - 2 (g & 1).
template <int NT>
__device__ __forceinline__ void scatter_count_sketch(float2* A, const float* x, int len,
                                                     const int32_t* hrow, const uint8_t* grow,
                                                     float wscale, bool colliding, int mask) {
  for (int i = threadIdx.x; i < len; i += NT) {
    const float v = x[i] * wscale;
    const int gi = grow[i] & 3;
    float* slot = reinterpret_cast<float*>(&A[pad_idx(hrow[i] & mask)]);
    if (colliding) atomicAdd(slot + (gi & 1), (gi & 2) ? -v : v);
    else atomicAdd(slot, (gi & 1) ? -v : v);
  }
}

template <int LOGB>
__global__ void __launch_bounds__(threads_for_logb(LOGB)) rank1_kernel(Rank1Args a) {
  constexpr int NT = threads_for_logb(LOGB);
  constexpr int b = 1 << LOGB;
  extern __shared__ float2 smem[];
  float2* A = smem;
  __shared__ float2 tw[kTwEntries];
  fill_twiddles(tw, NT);
  const int m = blockIdx.x, tid = threadIdx.x;
  float2* acc = a.acc + (size_t)m * b;
  float2* prod = a.prod ? a.prod + (size_t)m * b : nullptr;
  const int32_t* hm = a.h + (size_t)m * a.M * a.nmax;
  const uint8_t* gm = a.g + (size_t)m * a.M * a.nmax;
  for (long long c = 0; c < a.count; ++c) {
    const float wc = a.w[c];
    const int modes = a.M == 1 ? 1 : 3;
    for (int j = 0; j < modes; ++j) {
      for (int i = tid; i < padded_len(b); i += NT) A[i] = make_float2(0.f, 0.f);
      __syncthreads();
      const float* x = j == 0 ? a.U + (size_t)c * a.n1 : (j == 1 ? a.V + (size_t)c * a.n2 : a.W + (size_t)c * a.n3);
      const int len = j == 0 ? a.n1 : (j == 1 ? a.n2 : a.n3);
      scatter_count_sketch<NT>(A, x, len, hm + (size_t)j * a.nmax, gm + (size_t)j * a.nmax,
                               (a.M == 3 && j == 0) ? wc : 1.f, a.M == 1, b - 1);
      __syncthreads();
      block_fft<LOGB, NT, -1>(A, tw);
      for (int f = tid; f < b; f += NT) {
        const float2 X = A[pad_idx(f)];
        float2 term;
        if (a.M == 1) {
          term = cscale(cmul(cmul(X, X), X), wc);   // w (F s~_u)^3
        } else if (j == 0) {
          prod[f] = X;
          continue;
        } else if (j == 1) {
          prod[f] = cmul(prod[f], X);
          continue;
        } else {
          term = cmul(prod[f], X);
        }
        acc[f] = (c == 0) ? term : cadd(acc[f], term);
      }
      __syncthreads();
    }
  }
  // final: frequency-domain sum -> requested domain, written into S
  for (int f = tid; f < b; f += NT) A[pad_idx(f)] = a.count > 0 ? acc[f] : make_float2(0.f, 0.f);
  __syncthreads();
  float s = 1.f;
  if (a.domain == 0) {
    block_fft<LOGB, NT, +1>(A, tw);
    s = 1.f / (float)b;
  }
  float2* Sm = a.S + (size_t)m * b;
  for (int t = tid; t < b; t += NT) {
    const float2 v = cscale(A[pad_idx(t)], s);
    Sm[t] = a.accumulate ? cadd(Sm[t], v) : v;
  }
}

template <int LOGB>
static int launch_rank1_t(const Rank1Args& a, int B, cudaStream_t st) {
  constexpr size_t smem = (size_t)padded_len(1 << LOGB) * sizeof(float2);
  TSK_CUDA(tsk_smem_attr<rank1_kernel<LOGB>>(smem));
  rank1_kernel<LOGB><<<B, threads_for_logb(LOGB), smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

static int launch_rank1(int log2b, const Rank1Args& a, int B, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_rank1_t<8>(a, B, st);
    case 9: return launch_rank1_t<9>(a, B, st);
    case 10: return launch_rank1_t<10>(a, B, st);
    case 11: return launch_rank1_t<11>(a, B, st);
    case 12: return launch_rank1_t<12>(a, B, st);
    case 13: return launch_rank1_t<13>(a, B, st);
    case 14: return launch_rank1_t<14>(a, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

}  // namespace tsk

using namespace tsk;

extern "C" int sketch_tensor(tsk_ctx* ctx, const void* T, int in_dtype, int M,
                             const int64_t* dims_host, const int32_t* h, const uint8_t* g, int B,
                             int log2b, void* S, int acc_dtype, int accumulate) {
  if (!ctx || !T || !dims_host || !h || !g || !S) return TSK_EINVAL;
  if (B < 1 || (M != 1 && M != 3) || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (in_dtype != TSK_F32 && in_dtype != TSK_F64 && in_dtype != TSK_I32) return TSK_EINVAL;
  if (acc_dtype != TSK_C64 && acc_dtype != TSK_C128 && acc_dtype != TSK_CI64) return TSK_EINVAL;
  if (acc_dtype == TSK_CI64 && in_dtype != TSK_I32) return TSK_EINVAL;
  if (acc_dtype == TSK_C128 && in_dtype == TSK_I32) return TSK_EINVAL;
  for (int j = 0; j < M; ++j)
    if (dims_host[j] < 0 || dims_host[j] > 8192) return dims_host[j] < 0 ? TSK_EINVAL : TSK_EUNSUPPORTED;
  const size_t b = (size_t)1 << log2b;
  const size_t elem = acc_dtype == TSK_C64 ? sizeof(float) : 8;
  if (!accumulate) TSK_CUDA(cudaMemsetAsync(S, 0, (size_t)B * b * 2 * elem, ctx->stream));
  if (M == 1) {
    const int n = (int)dims_host[0];
    if (n == 0) return TSK_OK;
    if (log2b > 16) return TSK_EUNSUPPORTED;
    SymSketchArgs a{T, n, h, g, log2b, (long long)n * (n + 1) * (n + 2) / 6, 1, S, 0};
    if (acc_dtype == TSK_C64) {
      if (in_dtype == TSK_F32) return launch_sym<float, float, 1>(a, B, ctx);
      if (in_dtype == TSK_F64) return launch_sym<double, float, 1>(a, B, ctx);
      return launch_sym<int32_t, float, 1>(a, B, ctx);
    }
    if (acc_dtype == TSK_C128) {
      if (in_dtype == TSK_F32) return launch_sym<float, double, 2>(a, B, ctx);
      return launch_sym<double, double, 2>(a, B, ctx);
    }
    return launch_sym<int32_t, long long, 2>(a, B, ctx);
  }
  const int n1 = (int)dims_host[0], n2 = (int)dims_host[1], n3 = (int)dims_host[2];
  if (n1 == 0 || n2 == 0 || n3 == 0) return TSK_OK;
  const int nmax = n1 > n2 ? (n1 > n3 ? n1 : n3) : (n2 > n3 ? n2 : n3);
  AsymSketchArgs a{T, n1, n2, n3, nmax, h, g, log2b, (long long)n1 * n2, 1, S};
  if (acc_dtype == TSK_C64) {
    if (log2b > 15) return TSK_EUNSUPPORTED;
    if (in_dtype == TSK_F32) return launch_asym<float, float>(a, B, ctx);
    if (in_dtype == TSK_F64) return launch_asym<double, float>(a, B, ctx);
    return launch_asym<int32_t, float>(a, B, ctx);
  }
  if (log2b > 14) return TSK_EUNSUPPORTED;
  if (acc_dtype == TSK_C128) {
    if (in_dtype == TSK_F32) return launch_asym<float, double>(a, B, ctx);
    return launch_asym<double, double>(a, B, ctx);
  }
  return launch_asym<int32_t, long long>(a, B, ctx);
}

extern "C" int sketch_fft(tsk_ctx* ctx, const float* S_in, float* S_out, int B, int log2b,
                          int inverse) {
  if (!ctx || !S_in || !S_out || B < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  return launch_fft_batched(log2b, reinterpret_cast<const float2*>(S_in),
                            reinterpret_cast<float2*>(S_out), B, inverse ? 1 : 0, ctx->stream);
}

extern "C" int sketch_rank1(tsk_ctx* ctx, int64_t count, const float* w, const float* U,
                            const float* V, const float* W, int M, const int64_t* dims_host,
                            const int32_t* h, const uint8_t* g, int B, int log2b, int domain,
                            float* S, int accumulate) {
  if (!ctx || !dims_host || !h || !g || !S || count < 0) return TSK_EINVAL;
  if ((M != 1 && M != 3) || B < 1 || log2b < 1 || log2b > 24 || (domain != 0 && domain != 1))
    return TSK_EINVAL;
  if (count > 0 && (!w || !U)) return TSK_EINVAL;
  if (M == 3 && count > 0 && (!V || !W)) return TSK_EINVAL;
  if (log2b < 8 || log2b > 14) return TSK_EUNSUPPORTED;
  Rank1Args a{};
  a.count = count;
  a.w = w;
  a.U = U;
  a.V = V;
  a.W = W;
  a.M = M;
  a.n1 = (int)dims_host[0];
  a.n2 = M == 3 ? (int)dims_host[1] : a.n1;
  a.n3 = M == 3 ? (int)dims_host[2] : a.n1;
  if (a.n1 < 0 || a.n2 < 0 || a.n3 < 0) return TSK_EINVAL;
  a.nmax = a.n1 > a.n2 ? (a.n1 > a.n3 ? a.n1 : a.n3) : (a.n2 > a.n3 ? a.n2 : a.n3);
  a.h = h;
  a.g = g;
  a.domain = domain;
  a.accumulate = accumulate;
  a.S = reinterpret_cast<float2*>(S);
  const size_t b = (size_t)1 << log2b;
  int rc = tsk_ws_reserve(ctx, (M == 3 ? 2 : 1) * ws_round((size_t)B * b * sizeof(float2)));
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  a.acc = wc.take<float2>((size_t)B * b);
  a.prod = M == 3 ? wc.take<float2>((size_t)B * b) : nullptr;
  return launch_rank1(log2b, a, B, ctx->stream);
}
