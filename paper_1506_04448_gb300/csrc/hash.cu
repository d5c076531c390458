// cs_hashes: hash functions h: [n] -> [b] and complex Rademacher signs for B sketches.
//
// The paper requires H = h1 + h2 + h3 to be 2-wise independent (Sec. 2) and, for the
// colliding sketch where h1 = h2 = h3 = h, h to be 6-wise independent (Prop. 2 with p = 3,
// q = 2); sigma is uniform on the 4th roots of unity (Sec. 3.3, m = 4).  This library uses
// Carter-Wegman polynomials over GF(2^61 - 1): degree 5 for h (6-wise independent) and degree
// 11 for the sign index g (12-wise), coefficients drawn from a counter-based SplitMix64 stream
// (Steele, Lea & Flood 2014).  All arithmetic is exact 64/128-bit integer arithmetic.
#include "common.cuh"

namespace tsk {

constexpr uint64_t kP61 = (1ull << 61) - 1;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t mod_p61(uint64_t v) {
  uint64_t r = (v & kP61) + (v >> 61);
  return r >= kP61 ? r - kP61 : r;
}

// a * b mod P for a, b < P: the 122-bit product is split at bit 61 (2^61 = 1 mod P).
__device__ __forceinline__ uint64_t mulmod_p61(uint64_t a, uint64_t b) {
  const uint64_t lo = a * b;
  const uint64_t hi = __umul64hi(a, b);
  uint64_t r = (lo & kP61) + ((hi << 3) | (lo >> 61));
  r = (r & kP61) + (r >> 61);
  return r >= kP61 ? r - kP61 : r;
}

// Coefficient e of table w for (sketch m, mode j): SplitMix64 output number
// ((m*M + j)*2 + w)*16 + e of the stream started at seed, reduced mod P.
__device__ __forceinline__ uint64_t coef(uint64_t seed, int m, int j, int M, int w, int e) {
  const uint64_t c = (uint64_t)(((m * M + j) * 2 + w) * 16 + e);
  return mod_p61(mix64(seed + (c + 1) * kGamma));
}

template <int DEG>
__device__ __forceinline__ uint64_t poly_eval(uint64_t seed, int m, int j, int M, int w, uint64_t x) {
  uint64_t acc = 0;
#pragma unroll
  for (int e = DEG; e >= 0; --e) {
    acc = mulmod_p61(acc, x) + coef(seed, m, j, M, w, e);
    if (acc >= kP61) acc -= kP61;
  }
  return acc;
}

struct HashDims {
  int d[3];
};

__global__ void hash_kernel(uint64_t seed, int B, int M, int nmax, int log2b, HashDims dims,
                            int32_t* h, uint8_t* g) {
  const long long total = (long long)B * M * nmax;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nmax);
    const int j = (int)((idx / nmax) % M);
    const int m = (int)(idx / ((long long)nmax * M));
    if (i >= dims.d[j]) {
      h[idx] = 0;
      g[idx] = 0;
      continue;
    }
    const uint64_t hv = poly_eval<5>(seed, m, j, M, 0, (uint64_t)i);
    const uint64_t gv = poly_eval<11>(seed, m, j, M, 1, (uint64_t)i);
    h[idx] = (int32_t)(hv & ((1ull << log2b) - 1));
    g[idx] = (uint8_t)(gv & 3ull);
  }
}

// Order-p colliding hashes (p = 3..6): h from the degree-(2p-1) polynomial of table 0, so that
// h is (2p)-wise independent and H = h(i_1) + ... + h(i_p) 2-wise independent (Prop. 2 with
// q = 2); the sign index from the degree-11 polynomial of table 1 reduced mod m, sigma uniform
// on the m-th roots of unity with m the smallest power of two above p (E[sigma^k] = 0 unless
// m | k, so no two distinct multisets of p indices alias, Sec. 3.3).  At p = 3 these are the
// hashes of cs_hashes with M = 1.
template <int DEG>
__global__ void hash_p_kernel(uint64_t seed, int B, int n, int log2b, int mroots, int32_t* h,
                              uint8_t* g) {
  const long long total = (long long)B * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n);
    const int m = (int)(idx / n);
    const uint64_t hv = poly_eval<DEG>(seed, m, 0, 1, 0, (uint64_t)i);
    const uint64_t gv = poly_eval<11>(seed, m, 0, 1, 1, (uint64_t)i);
    h[idx] = (int32_t)(hv & ((1ull << log2b) - 1));
    g[idx] = (uint8_t)(gv & (uint64_t)(mroots - 1));
  }
}

}  // namespace tsk

extern "C" int cs_hashes_p(tsk_ctx* ctx, uint64_t seed, int B, int log2b, int p, int64_t n,
                           int32_t* h, uint8_t* g) {
  if (!ctx || !h || !g) return TSK_EINVAL;
  if (B < 1 || log2b < 1 || log2b > 24 || n < 0 || n >= (1ll << 31)) return TSK_EINVAL;
  if (p < 3 || p > 6) return TSK_EUNSUPPORTED;
  if (n == 0) return TSK_OK;
  const int mroots = p < 4 ? 4 : 8;
  const long long total = (long long)B * n;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  const unsigned nb = (unsigned)blocks;
  switch (p) {
    case 3: tsk::hash_p_kernel<5><<<nb, threads, 0, ctx->stream>>>(seed, B, (int)n, log2b, mroots, h, g); break;
    case 4: tsk::hash_p_kernel<7><<<nb, threads, 0, ctx->stream>>>(seed, B, (int)n, log2b, mroots, h, g); break;
    case 5: tsk::hash_p_kernel<9><<<nb, threads, 0, ctx->stream>>>(seed, B, (int)n, log2b, mroots, h, g); break;
    default: tsk::hash_p_kernel<11><<<nb, threads, 0, ctx->stream>>>(seed, B, (int)n, log2b, mroots, h, g); break;
  }
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

extern "C" int cs_hashes(tsk_ctx* ctx, uint64_t seed, int B, int log2b, int M,
                         const int64_t* dims_host, int32_t* h, uint8_t* g) {
  if (!ctx || !dims_host || !h || !g) return TSK_EINVAL;
  if (B < 1 || (M != 1 && M != 3) || log2b < 1 || log2b > 24) return TSK_EINVAL;
  int nmax = 0;
  tsk::HashDims dims{{0, 0, 0}};
  for (int j = 0; j < M; ++j) {
    if (dims_host[j] < 0 || dims_host[j] >= (1ll << 31)) return TSK_EINVAL;
    dims.d[j] = (int)dims_host[j];
    if (dims.d[j] > nmax) nmax = dims.d[j];
  }
  if (nmax == 0) return TSK_OK;
  const long long total = (long long)B * M * nmax;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  tsk::hash_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(seed, B, M, nmax, log2b, dims, h, g);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}
