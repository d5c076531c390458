// Order-p symmetric (colliding) tensor sketches, p = 3..6: the builds (every entry, or the wedge of
// a symmetric tensor) and the C entry points.  The sketch, contraction and deflation formulas are
// stated at the top of orderp.cuh, which holds the contraction and deflation kernels; orderp_p3.cu
// .. orderp_p6.cu instantiate them one order per translation unit.
#include <stdio.h>

#include "orderp.cuh"

namespace tsk {

// dynamic shared memory of sketch_p_kernel: the b <= 2^14 histogram and two n <= 8192 tables
constexpr size_t kSketchPSmemMax = ((size_t)1 << 14) * sizeof(float2) + 2 * (size_t)8192 * sizeof(int);

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
      // kappa of this row's entries: y == x and y > x
      const float kdia = fact[p] / (x == v ? denom * fact[run + 2] : denom * fact[run] * 2.f);
      const float koff = fact[p] / (x == v ? denom * fact[run + 1] : denom * fact[run]);
      for (int y = x + lane; y < n; y += 32) {
        const float kappa = y == x ? kdia : koff;
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

static int launch_contract_p(int log2b, int p, const PArgs& a, int L, cudaStream_t st) {
  switch (p) {
    case 3: return launch_contract_p3(log2b, a, L, st);
    case 4: return launch_contract_p4(log2b, a, L, st);
    case 5: return launch_contract_p5(log2b, a, L, st);
    case 6: return launch_contract_p6(log2b, a, L, st);
    default: return TSK_EUNSUPPORTED;
  }
}

static int launch_deflate_p(int log2b, int p, float2* FS, float2* S, const int32_t* h,
                            const uint8_t* g, int n, int L, const float* Uf, const float* lm, int r,
                            double* lo, float* Vo, int32_t* to, int B, cudaStream_t st) {
  switch (p) {
    case 3: return launch_deflate_p3(log2b, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 4: return launch_deflate_p4(log2b, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 5: return launch_deflate_p5(log2b, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
    case 6: return launch_deflate_p6(log2b, FS, S, h, g, n, L, Uf, lm, r, lo, Vo, to, B, st);
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
