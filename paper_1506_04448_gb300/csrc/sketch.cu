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
#include <type_traits>

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
  long long W;        // wedge entries to build (those of the planes asked for)
  long long E0;       // wedge position of the first of them
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
  const long long e0 = a.E0 + (long long)blockIdx.y * per_slab;
  const long long e1 = min(a.E0 + a.W, e0 + per_slab);
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

// ------------------------------------------------------------------ colliding build, exact int32
//
// The FP32 colliding build of Eq. 7 in integer fixed point.  Shared-memory FP32 atomics run as a
// compare-and-swap loop on this part (about 9 SM cycles per random warp-wide add, measured);
// 32-bit integer adds are native (about 2.7 cycles, 4.7 with the returned old value).  So every
// entry is quantised once, q = rint(kappa x 2^(25-E)) with 2^E > max|T| over the wedge (a
// prepass), and the buckets are accumulated as wrapping int32 sums.  The returned old value
// tells the warp when an add may have wrapped past +-2^31; the exact check then adds the carry
// +-1 to a global int32 array, so every bucket's integer total is exact.  Block partials are
// written to a workspace and summed in int64 by a separate kernel, which scales by 2^(E-25)
// once.  The result is deterministic; its only roundings are the quantisation of each entry
// (at most 2^(E-26), below 6e-8 of max|T|) and the final conversion to float.

// rows before wedge row i: sum_{i' < i} (n - i') = i n - i (i - 1) / 2
__device__ __forceinline__ long long wedge_rows_before(long long n, long long i) {
  return i * n - i * (i - 1) / 2;
}

// |x| rounded up to float, as raw bits (ordered like the values for non-negative floats; NaN
// and infinity compare above every finite value)
__device__ __forceinline__ uint32_t absbits(float x) { return __float_as_uint(fabsf(x)); }
__device__ __forceinline__ uint32_t absbits(double x) {
  return __float_as_uint(__double2float_ru(fabs(x)));
}
__device__ __forceinline__ uint32_t absbits(int32_t x) {
  return __float_as_uint(__ll2float_ru(llabs((long long)x)));
}

constexpr int kMaxTileCols = 256;   // nc = ceil(n / 32) for n <= 8192

// Wedge tiles.  The wedge {i <= j <= k < n} is covered by tiles (rb, c, i): plane i, rows j in
// [32 rb, 32 rb + 32) with j >= i, columns k in [32 c, 32 c + 32) with k >= j, for
// rb <= c < nc = ceil(n / 32) and i < min(32 rb + 32, n).  One warp takes one tile: lane l owns
// column k = 32 c + l (one coalesced 128-byte row segment per row), so the column's hash words
// stay in registers while the warp walks the tile's rows.  Within a row block rb the tiles are
// numbered column-major over the planes that reach it.  The fixed-point build and its prepass
// place the same tiles on indices shifted by (-n) mod 32 (wedge_shift).

// Wedge tiles of the fixed-point build are 32 x 32 blocks of (j, k) in the shifted indices
// j' = j + off, k' = k + off with off = (-n) mod 32, so that the last column block ends exactly at
// n: a lane never stands beyond the tensor, and the one ragged block (shifted indices below off)
// is reached only by the planes i < 32 - off.
__host__ __device__ __forceinline__ int wedge_shift(int n) { return (32 - (n & 31)) & 31; }

// max |T_ijk| over the wedge i <= j <= k as float bits, into *maxbits (zeroed by the caller).
// Warps take the wedge's tiles (all planes, shifted like the build's) and load a tile's up to 32
// rows at once.
template <typename TIn>
__global__ void __launch_bounds__(256) wedge_absmax_kernel(const TIn* __restrict__ T, int n, int i0,
                                                           int i1, unsigned* maxbits) {
  // planes [i0, i1) in the shifted indices of wedge_shift: row blocks rb >= (i0 + off) / 32,
  // each with planes i0 .. min(i1 + off, 32 rb + 32) - off - 1
  __shared__ unsigned smax;
  __shared__ int pre[kMaxTileCols + 1];   // tiles before row block rb0 + q
  const int off = wedge_shift(n);
  const int nc = (n + 31) >> 5;
  const int rb0 = (i0 + off) >> 5, nrb = nc - rb0;
  if (threadIdx.x == 0) {
    smax = 0u;
    int acc = 0;
    for (int q = 0; q < nrb; ++q) {
      pre[q] = acc;
      const int rb = rb0 + q;
      acc += max(0, min(i1 + off, 32 * rb + 32) - (i0 + off)) * (nc - rb);
    }
    pre[nrb] = acc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  uint32_t mb = 0u;
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < pre[nrb]; it += nwarps) {
    int lo = 0, hi = nrb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= it) lo = mid; else hi = mid - 1;
    }
    const int rb = rb0 + lo;
    const int nir = min(i1 + off, 32 * rb + 32) - (i0 + off);
    const int local = it - pre[lo];
    const int c = rb + local / nir;
    const int i = i0 + local % nir;
    const int jlo = max(i, 32 * rb - off), jhi = 32 * rb + 32 - off;
    const int k = 32 * c + lane - off;
    const int jlim = rb == c ? min(k, jhi - 1) : jhi - 1;   // no rows for k < 0
    const TIn* col = T + ((size_t)i * n + jlo) * n + (k < 0 ? 0 : k);
    TIn x[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      x[r] = (TIn)0;
      if (jlo + r <= jlim) x[r] = __ldcg(col + (size_t)r * n);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) mb = max(mb, absbits(x[r]));
  }
  mb = __reduce_max_sync(0xffffffffu, mb);
  if (lane == 0) atomicMax(&smax, mb);
  __syncthreads();
  if (threadIdx.x == 0 && smax != 0u) atomicMax(maxbits, smax);
}

// Quantisation for max|T| bits `mb`: q = rint(kappa x 2^(25-E)) with 2^E > max|T|, so
// |q| < 6 2^25 < 2^28.  The factor 2^(25-E) is applied as sa (and sb, only when it is not a
// normal float by itself).
constexpr int kFixBits = 25;

struct FixScale {
  float sa, sb;
  int e;        // E
  bool finite;
};
__device__ __forceinline__ FixScale fix_scale(uint32_t mb) {
  FixScale f;
  f.finite = mb < 0x7f800000u;
  int e = 0;
  if (mb != 0u && f.finite) frexpf(__uint_as_float(mb), &e);   // max|T| < 2^e
  const int k = kFixBits - e;                                  // k in [-103, 174]
  const bool one = k >= -120 && k <= 120;
  f.sa = ldexpf(1.f, one ? k : k / 2);
  f.sb = one ? 1.f : ldexpf(1.f, k - k / 2);
  f.e = e;
  return f;
}

constexpr int kMaxFixParts = 256;

struct SymFixArgs {
  const void* T;
  int n;
  const int32_t* h;     // [B][n]
  const uint8_t* g;     // [B][n]
  int B;
  int log2b;
  int log2r;            // 2^log2r bucket ranges, one block each
  int nslab;            // partials per sketch: block s of a sketch takes tiles s, s + nslab, ...
  const unsigned* maxbits;
  int* carry;           // [B][2b]: wraps of the int32 sums past +-2^31
  int* part;            // [nslab][B][2b]: per-block integer partials
  int p0, p1;           // the planes [p0, p1) are built
};

// Packed hash word of index i for the fixed-point build: 8 h(i) + g(i) 2^30 (mod 2^32).  In the
// sum sq of the words of i, j, k, bits 3..20 carry 8 (h_i + h_j + h_k) < 2^21 and bits 30..31
// carry (g_i + g_j + g_k) mod 4, the exponent of sigma_i sigma_j sigma_k = sqrt(-1)^e: bit 31 is
// its sign and bit 30 picks the imaginary part.  So the byte offset 8 t + 4 (e & 1) of the
// bucket's re/im cell is (sq & 8 mask) | ((sq >> 28) & ~(8 mask)), and the sign is sq's top bit.
__device__ __forceinline__ uint32_t fix_word(int32_t h, uint8_t g, int mask) {
  return ((uint32_t)(h & mask) << 3) + ((uint32_t)(g & 3) << 30);
}

// One batch of 8 rows j0..j0+7 of a tile for every sketch of the block: y[r] is row j0 + r's
// entry already scaled by kappa 2^(25-E) (0 for a lane that has no entry there).  Each add goes
// to a valid cell even when its value is 0, so no lane is masked off; the adds go out back to
// back and their returned old values are checked for wraps afterwards.
template <int SK, bool RANGES>
__device__ __forceinline__ void sym_fix_batch(const SymFixArgs& a, int* hist, const uint32_t* qs,
                                              const uint32_t* qik, const float* y, int j0,
                                              int jhi, int m0, int rr) {
  const int n = a.n;
  const int b = 1 << a.log2b;
  const int mask = b - 1;
  const uint32_t m8 = 8u * (uint32_t)mask;
  const int br = RANGES ? b >> a.log2r : b;
  const int cells = 2 * br;
  const int shift_r = a.log2b - a.log2r;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < SK; ++s) {
    // lane r of the warp holds row j0 + r's word
    const uint32_t qrow = qs[s * n + min(j0 + (lane & 7), jhi - 1)];
    char* hb = reinterpret_cast<char*>(hist + s * cells);
    int v[8], old[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t sq = qik[s] + __shfl_sync(0xffffffffu, qrow, r);
      uint32_t off;
      v[r] = __float2int_rn(__uint_as_float(__float_as_uint(y[r]) ^ (sq & 0x80000000u)));
      if (RANGES) {
        const int t = (int)(sq >> 3) & mask;
        if ((t >> shift_r) != rr) v[r] = 0;
        off = 8u * (uint32_t)(t & (br - 1)) + ((sq >> 28) & 4u);
      } else {
        off = (sq & m8) | ((sq >> 28) & ~m8);
      }
      old[r] = atomicAdd(reinterpret_cast<int*>(hb + off), v[r]);
    }
    // |v| < 2^28, so an add can wrap only if |old| >= 2^30, i.e. old + 2^30 has its top bit set
    unsigned near = 0u;
#pragma unroll
    for (int r = 0; r < 8; ++r) near |= (unsigned)old[r] + 0x40000000u;
    // exact check, carry +-2^32 for each wrapped add (rare); entered by the whole warp, since the
    // row words come back by shuffles over all lanes
    if (__any_sync(0xffffffffu, (int)near < 0)) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int sum = (int)((unsigned)old[r] + (unsigned)v[r]);
        const uint32_t sq = qik[s] + __shfl_sync(0xffffffffu, qrow, r);
        if (((old[r] ^ sum) & (v[r] ^ sum)) < 0) {
          const int t = (int)(sq >> 3) & mask;
          atomicAdd(&a.carry[(size_t)(m0 + s) * 2 * b + 2 * t + (int)((sq >> 30) & 1)],
                    v[r] > 0 ? 1 : -1);
        }
      }
    }
  }
}

// Interior tile (no row j == i, no diagonal element k == j, kappa = 6) of whole 8-row batches:
// unconditional loads (a lane beyond the tensor reads column n - 1 and scales it by 0), the next
// batch's loads issued before the current batch's adds.
template <typename TIn, int SK, bool RANGES, bool TWO>
__device__ __forceinline__ void sym_fix_rows_interior(const SymFixArgs& a, const FixScale& fs,
                                                      int* hist, const uint32_t* qs,
                                                      const TIn* col, bool kin, int jlo, int jhi,
                                                      const uint32_t* qik, int m0, int rr) {
  const int n = a.n;
  const float ks = kin ? 6.f * fs.sa : 0.f;
  TIn xa[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) xa[r] = __ldcg(col + (size_t)r * n);
  for (int j0 = jlo; j0 < jhi; j0 += 8) {
    TIn xb[8];
    if (j0 + 8 < jhi) {
      const TIn* p = col + (size_t)(j0 + 8 - jlo) * n;
#pragma unroll
      for (int r = 0; r < 8; ++r) xb[r] = __ldcg(p + (size_t)r * n);
    }
    float y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      y[r] = (float)xa[r] * ks;
      if (TWO) y[r] *= fs.sb;
    }
    sym_fix_batch<SK, RANGES>(a, hist, qs, qik, y, j0, jhi, m0, rr);
#pragma unroll
    for (int r = 0; r < 8; ++r) xa[r] = xb[r];
  }
}

// Any tile: rows [jlo, jhi) 8 at a time, loads only where the lane has an entry (j <= jlim).
template <typename TIn, int SK, bool RANGES, bool TWO>
__device__ __forceinline__ void sym_fix_rows_edge(const SymFixArgs& a, const FixScale& fs,
                                                  int* hist, const uint32_t* qs, const TIn* col,
                                                  int i, int k, int jlo, int jhi, int jlim,
                                                  const uint32_t* qik, int m0, int rr) {
  const int n = a.n;
  const float ks1 = fs.sa, ks3 = 3.f * fs.sa, ks6 = 6.f * fs.sa;
  for (int j0 = jlo; j0 < jhi; j0 += 8) {
    const TIn* p = col + (size_t)(j0 - jlo) * n;
    float y[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int j = j0 + r;
      TIn x = (TIn)0;
      if (j <= jlim) x = __ldcg(p + (size_t)r * n);
      // kappa = number of orderings of (i, j, k): 6 when all differ, 3 when two agree
      const float ks = (j == i) ? (k == j ? ks1 : ks3) : (k == j ? ks3 : ks6);
      y[r] = (float)x * ks;
      if (TWO) y[r] *= fs.sb;
    }
    sym_fix_batch<SK, RANGES>(a, hist, qs, qik, y, j0, jhi, m0, rr);
  }
}

// The tiles of one block, in the shifted indices of wedge_shift: planes [i0, i1), row blocks
// rb >= rb0 = (i0 + off) / 32, columns c >= rb, planes i + off < 32 rb + 32 only.  For row block
// rb there are nir = min(i1 + off, 32 rb + 32) - (i0 + off) planes times (nc - rb) columns; pre[]
// holds the running counts and rcp[] the reciprocals 1 / nir.
// The block takes every stride-th tile from first on (the blocks of a sketch deal the tiles out
// round robin, so each gets an even share of every tile size).  A warp's items come from the
// block's counter in increasing order, so its row block only moves forward (a scan from the last
// one), and local / nir is a float product corrected to the exact quotient (local < 2^24).
template <typename TIn, int SK, bool RANGES, bool TWO>
__device__ __forceinline__ void sym_fix_tiles(const SymFixArgs& a, const FixScale& fs, int* hist,
                                              const uint32_t* qs, const int* pre,
                                              const float* rcp, int nrb, int* next, int i0,
                                              int i1, int first, int stride, int m0, int rr) {
  const int n = a.n;
  const int off = wedge_shift(n);
  const int rb0 = (i0 + off) >> 5;
  const int lane = threadIdx.x & 31;
  const TIn* T = static_cast<const TIn*>(a.T);
  const int items = pre[nrb];
  int lo = 0;   // row block of the warp's last item
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(next, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    const int it = first + stride * u;   // < items + 32 stride: no int overflow
    if (it >= items) break;
    while (pre[lo + 1] <= it) ++lo;   // row block: last with pre[.] <= it
    const int rb = rb0 + lo;
    const int nir = min(i1 + off, 32 * rb + 32) - (i0 + off);
    const int local = it - pre[lo];
    int cq = (int)((float)local * rcp[lo]);
    int ir = local - cq * nir;
    if (ir < 0) { --cq; ir += nir; } else if (ir >= nir) { ++cq; ir -= nir; }
    const int c = rb + cq;
    const int i = i0 + ir;
    // rows and column in tensor indices (jhi <= n and k < n, since 32 nc = n + off)
    const int jlo = max(i, 32 * rb - off), jhi = 32 * rb + 32 - off;
    const int k = 32 * c + lane - off;
    // last row this lane takes part in: the tile's last row, k itself on the diagonal block
    // (j <= k); none for a lane ahead of the tensor (k < 0 <= i, diagonal block only)
    const int jlim = rb == c ? min(k, jhi - 1) : jhi - 1;
    // a lane ahead of the tensor adds zeros; it takes the word of k mod n, so that its cells are
    // spread like everyone else's (one shared cell would serialise those adds)
    int kw = k;   // k mod n (k >= -31)
    while (kw < 0) kw += n;
    uint32_t qik[SK];
#pragma unroll
    for (int s = 0; s < SK; ++s) qik[s] = qs[s * n + i] + qs[s * n + kw];
    const TIn* col = T + ((size_t)i * n + jlo) * n + (k < 0 ? 0 : k);
    if (rb < c) {
      // off the diagonal block: the plane's first row (j = i, kappa 3) and enough rows after it
      // to leave whole 8-row batches go the per-row path, the batches the interior path
      // (kappa 6), a ragged tail the per-row path again
      int e = 0;
      if (jlo == i) {
        e = (jhi - i) & 7;
        if (e == 0) e = 8;
      }
      const int jmid = jlo + e;
      const int nint = (jhi - jmid) & ~7;
      if (e > 0)
        sym_fix_rows_edge<TIn, SK, RANGES, TWO>(a, fs, hist, qs, col, i, k, jlo, jmid,
                                                min(jlim, jmid - 1), qik, m0, rr);
      if (nint > 0)
        sym_fix_rows_interior<TIn, SK, RANGES, TWO>(a, fs, hist, qs, col + (size_t)e * n, k >= 0,
                                                    jmid, jmid + nint, qik, m0, rr);
      if (jmid + nint < jhi)
        sym_fix_rows_edge<TIn, SK, RANGES, TWO>(a, fs, hist, qs, col + (size_t)(e + nint) * n, i,
                                                k, jmid + nint, jhi, jlim, qik, m0, rr);
    } else {
      sym_fix_rows_edge<TIn, SK, RANGES, TWO>(a, fs, hist, qs, col, i, k, jlo, jhi, jlim, qik, m0, rr);
    }
  }
}

// Block (group of SK sketches, bucket range rr, partial s).  The block's warps take its share of
// the wedge tiles from a shared counter; per batch of 8 rows a warp has 8 loads in flight per lane,
// scales each entry by kappa 2^(25-E) and, per sketch, flips its sign, rounds it to int32 and
// adds it to the bucket's re or im cell.
template <typename TIn, int SK, bool RANGES>
__global__ void __launch_bounds__(1024, 1) sketch_sym_fix_kernel(SymFixArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_next;
  __shared__ int s_pre[kMaxTileCols + 1];
  __shared__ float s_rcp[kMaxTileCols];
  const FixScale fs = fix_scale(*a.maxbits);
  if (!fs.finite) return;   // the reduce kernel writes NaN
  const int b = 1 << a.log2b;
  const int n = a.n;
  const int mask = b - 1;
  const int R = RANGES ? 1 << a.log2r : 1;
  const int br = RANGES ? b >> a.log2r : b;
  const int cells = 2 * br;   // re/im interleaved, like the output
  int* hist = reinterpret_cast<int*>(sm_raw);                                  // [SK][cells]
  uint32_t* qs = reinterpret_cast<uint32_t*>(sm_raw + (size_t)SK * cells * sizeof(int));  // [SK][n]
  const int grp = blockIdx.x / R;
  const int rr = blockIdx.x % R;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m0 = grp * SK;
  const int i0 = a.p0, i1 = a.p1;
  const int off = wedge_shift(n);
  const int nc = (n + 31) >> 5;
  const int rb0 = (i0 + off) >> 5;
  const int nrb = nc - rb0;
  for (int i = tid; i < SK * cells; i += nt) hist[i] = 0;
  for (int s = 0; s < SK; ++s) {
    const int m = m0 + s;
    for (int i = tid; i < n; i += nt) qs[s * n + i] = fix_word(a.h[(size_t)m * n + i], a.g[(size_t)m * n + i], mask);
  }
  if (tid == 0) {
    s_next = 0;
    int acc = 0;
    for (int q = 0; q < nrb; ++q) {
      s_pre[q] = acc;
      const int rb = rb0 + q;
      const int nir = min(i1 + off, 32 * rb + 32) - (i0 + off);
      s_rcp[q] = 1.f / (float)nir;
      acc += nir * (nc - rb);
    }
    s_pre[nrb] = acc;
  }
  __syncthreads();
  if (fs.sb == 1.f)
    sym_fix_tiles<TIn, SK, RANGES, false>(a, fs, hist, qs, s_pre, s_rcp, nrb, &s_next, i0, i1,
                                          blockIdx.y, a.nslab, m0, rr);
  else
    sym_fix_tiles<TIn, SK, RANGES, true>(a, fs, hist, qs, s_pre, s_rcp, nrb, &s_next, i0, i1,
                                         blockIdx.y, a.nslab, m0, rr);
  __syncthreads();
  for (int s = 0; s < SK; ++s) {
    int* dst = a.part + ((size_t)blockIdx.y * a.B + (m0 + s)) * 2 * b + (size_t)2 * rr * br;
    for (int c = tid; c < cells; c += nt) dst[c] = hist[s * cells + c];
  }
}

// S[m][c] (+)= 2^(E-25) (sum over the partials of part[.][m][c] + 2^32 carry[m][c]); NaN if
// max|T| is not finite (also reported as TSK_ENONFINITE).  Four cells per thread with 16-byte
// loads (cells is a multiple of 4), so that one wave of threads has every partial's loads in
// flight.
__global__ void __launch_bounds__(256) sym_fix_reduce_kernel(const int* __restrict__ part,
                                                             const int* __restrict__ carry,
                                                             const unsigned* maxbits, int nslab,
                                                             long long cells, float* S,
                                                             int accumulate, int s_aligned,
                                                             int* status) {
  const FixScale fs = fix_scale(*maxbits);
  const long long quads = cells >> 2;
  for (long long c4 = (long long)blockIdx.x * blockDim.x + threadIdx.x; c4 < quads;
       c4 += (long long)gridDim.x * blockDim.x) {
    float v[4];
    if (fs.finite) {
      const int4 cr = __ldcg(reinterpret_cast<const int4*>(carry) + c4);
      long long acc[4] = {(long long)cr.x * 4294967296LL, (long long)cr.y * 4294967296LL,
                          (long long)cr.z * 4294967296LL, (long long)cr.w * 4294967296LL};
#pragma unroll 8
      for (int s = 0; s < nslab; ++s) {
        const int4 p = __ldcg(reinterpret_cast<const int4*>(part + (size_t)s * cells) + c4);
        acc[0] += p.x;
        acc[1] += p.y;
        acc[2] += p.z;
        acc[3] += p.w;
      }
      // one rounding (int64 -> float), then an exact power-of-two scaling
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = ldexpf(__ll2float_rn(acc[e]), fs.e - kFixBits);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = __int_as_float(0x7fc00000);
      if (c4 == 0) tsk_set_status(status, TSK_ENONFINITE);
    }
    if (s_aligned) {
      float4* S4 = reinterpret_cast<float4*>(S) + c4;
      if (accumulate) {
        const float4 o = *S4;
        *S4 = make_float4(o.x + v[0], o.y + v[1], o.z + v[2], o.w + v[3]);
      } else {
        *S4 = make_float4(v[0], v[1], v[2], v[3]);
      }
    } else {   // S is only 8-byte aligned (a complex-float array)
#pragma unroll
      for (int e = 0; e < 4; ++e) S[4 * c4 + e] = accumulate ? S[4 * c4 + e] + v[e] : v[e];
    }
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

template <typename TIn, int SK, bool RANGES>
static int launch_sym_fix_t(const SymFixArgs& a, int groups, size_t smem, tsk_ctx* ctx) {
  auto kernel = sketch_sym_fix_kernel<TIn, SK, RANGES>;
  TSK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(groups << a.log2r, (unsigned)a.nslab);
  kernel<<<grid, 1024, smem, ctx->stream>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <typename TIn>
static int launch_sym_fix(const void* T, int n, int p0, int p1, const int32_t* h, const uint8_t* g,
                          int B, int log2b, void* S, int accumulate, tsk_ctx* ctx) {
  const size_t b = (size_t)1 << log2b;
  const size_t smax = (size_t)ctx->max_smem_optin - 4096;   // the kernel's static tables (2.1 KB)
  auto smem_for = [&](int sk, int lr) {
    return (size_t)sk * 2 * (b >> lr) * sizeof(int) + (size_t)sk * n * sizeof(uint32_t) + 16;
  };
  // fewest bucket ranges whose histogram fits; then the most sketches per block (dividing B,
  // so every block does the same work) that still fit
  int log2r = 0;
  while (smem_for(1, log2r) > smax && log2r < 4) ++log2r;
  if (smem_for(1, log2r) > smax) return TSK_EUNSUPPORTED;
  int SK = 1;
  if (std::is_same<TIn, float>::value && log2r == 0) {
    if (B % 4 == 0 && smem_for(4, 0) <= smax) SK = 4;
    else if (B % 2 == 0 && smem_for(2, 0) <= smax) SK = 2;
  }
  const size_t smem = smem_for(SK, log2r);
  const int groups = B / SK;
  const int R = 1 << log2r;
  SymFixArgs a{};
  a.T = T;
  a.n = n;
  a.h = h;
  a.g = g;
  a.B = B;
  a.log2b = log2b;
  a.log2r = log2r;
  // one wave of 1024-thread blocks (one per SM): nslab partials per sketch, none with fewer than
  // ~16k wedge entries; only the planes [p0, p1) are built
  auto tet = [](long long x) { return x * (x + 1) * (x + 2) / 6; };
  const long long W = tet(n - p0) - tet(n - p1);
  long long nslab = (long long)ctx->num_sms / ((long long)groups * R);
  if (nslab < 1) nslab = 1;
  const long long cap = (W + 16383) / 16384;
  if (nslab > cap) nslab = cap;
  if (nslab < 1) nslab = 1;
  if (nslab > kMaxFixParts) nslab = kMaxFixParts;
  a.nslab = (int)nslab;
  a.p0 = p0;
  a.p1 = p1;
  const size_t cells = (size_t)B * 2 * b;
  const size_t head = ws_round(256) + ws_round(cells * sizeof(int));
  int rc = tsk_ws_reserve(ctx, head + ws_round((size_t)a.nslab * cells * sizeof(int)));
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  unsigned* maxbits = wc.take<unsigned>(64);
  a.carry = wc.take<int>(cells);
  a.part = wc.take<int>((size_t)a.nslab * cells);
  a.maxbits = maxbits;
  TSK_CUDA(cudaMemsetAsync(ctx->ws, 0, head, ctx->stream));
  wedge_absmax_kernel<TIn><<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(static_cast<const TIn*>(T), n,
                                                                    p0, p1, maxbits);
  TSK_CHECK_LAUNCH();
  if constexpr (std::is_same<TIn, float>::value) {
    if (SK == 4) rc = launch_sym_fix_t<TIn, 4, false>(a, groups, smem, ctx);
    else if (SK == 2) rc = launch_sym_fix_t<TIn, 2, false>(a, groups, smem, ctx);
  }
  if (SK == 1) {
    if (log2r == 0) rc = launch_sym_fix_t<TIn, 1, false>(a, groups, smem, ctx);
    else rc = launch_sym_fix_t<TIn, 1, true>(a, groups, smem, ctx);
  }
  if (rc != TSK_OK) return rc;
  long long blocks = ((long long)cells / 4 + 255) / 256;
  if (blocks > (long long)ctx->num_sms * 8) blocks = (long long)ctx->num_sms * 8;
  sym_fix_reduce_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(
      a.part, a.carry, maxbits, a.nslab, (long long)cells, static_cast<float*>(S), accumulate,
      (reinterpret_cast<uintptr_t>(S) & 15) == 0 ? 1 : 0, ctx->status);
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

// ------------------------------------------------------------------ asymmetric build, exact int32
// Complex-float asymmetric sketches (Eq. 1) by the colliding build's integer scheme: every entry
// is rounded once to the grid 2^(E-25), 2^E > max|T| over the whole tensor (dense_absmax_kernel),
// the real buckets are summed exactly in int32 shared memory with exact carries past 2^31, and
// the slab partials are added in int64 by a fixed-order reduce, so that the result does not
// depend on thread scheduling and the only other rounding is the final conversion to float.

// max |T| over n entries, as the bit pattern of a non-negative float (monotone as unsigned);
// NaN compares above every finite value, so a non-finite entry makes the result non-finite.
template <typename TIn>
__global__ void __launch_bounds__(256) dense_absmax_kernel(const TIn* T, long long count,
                                                           unsigned* maxbits) {
  unsigned m = 0u;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf((float)__ldcg(T + e))));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m != 0u) atomicMax(maxbits, m);
}

struct AsymFixArgs {
  const void* T;
  int n1, n2, n3, nmax;
  const int32_t* h;   // [B][3][nmax]
  const uint8_t* g;
  int B;
  int log2b;
  long long rows;     // n1 * n2
  int nslab;
  const unsigned* maxbits;
  int* carry;         // [B][b]: wraps of the int32 sums past +-2^31
  int* part;          // [nslab][B][b]
};

// Per-mode word of index i: bucket h & (b - 1) in the low bits, the sign bit g & 1 in bit 31;
// the sum of three words holds (h1 + h2 + h3) in its low 17 bits (b <= 2^15) and the parity of
// g1 + g2 + g3, i.e. the sign of xi1 xi2 xi3, in bit 31.
__device__ __forceinline__ uint32_t asym_word(int32_t h, uint8_t g, int mask) {
  return (uint32_t)(h & mask) | ((uint32_t)(g & 1) << 31);
}

template <typename TIn>
__global__ void __launch_bounds__(1024, 1) sketch_asym_fix_kernel(AsymFixArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const FixScale fs = fix_scale(*a.maxbits);
  if (!fs.finite) return;   // the reduce kernel writes NaN
  const int b = 1 << a.log2b;
  const int mask = b - 1;
  int* hist = reinterpret_cast<int*>(sm_raw);                                // [b]
  uint32_t* ws = reinterpret_cast<uint32_t*>(sm_raw + (size_t)b * sizeof(int));  // [3][nmax]
  const int m = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < b; i += nt) hist[i] = 0;
  for (int i = tid; i < 3 * a.nmax; i += nt)
    ws[i] = asym_word(a.h[(size_t)m * 3 * a.nmax + i], a.g[(size_t)m * 3 * a.nmax + i], mask);
  __syncthreads();
  const TIn* T = static_cast<const TIn*>(a.T);
  const long long per_slab = (a.rows + a.nslab - 1) / a.nslab;
  const long long r0 = (long long)blockIdx.y * per_slab;
  const long long r1 = min(a.rows, r0 + per_slab);
  const int nw = nt >> 5, w = tid >> 5, lane = tid & 31;
  const uint32_t* w1 = ws;
  const uint32_t* w2 = ws + a.nmax;
  const uint32_t* w3 = ws + 2 * a.nmax;
  const float sa = fs.sa, sb = fs.sb;
  int* carry = a.carry + (size_t)m * b;
  // The warp's work is a list of chunks (row r, kU 32-entry pieces of it), walked with
  // incremental cursors (no divisions in the loop); the loads of the next chunk are issued before
  // the adds of the current one, so that every lane keeps 2 kU loads in flight while it waits on
  // shared adds.  Rows number at most 8192^2, so int indices suffice.
  constexpr int kU = 4;
  const int cpr = (a.n3 + 32 * kU - 1) / (32 * kU);          // chunks per row
  const int rend = (int)r1;
  int r = (int)r0 + w, kc = 0;                                // chunk being processed
  int i = r / a.n2, jj = r % a.n2;                            // its row's (i, j)
  int rn = r, kcn = 0;                                        // chunk being loaded
  auto load_chunk = [&](int rr, int kk, TIn* x) {
    const TIn* row = T + (size_t)rr * a.n3;
    const int k0 = kk * 32 * kU + lane;
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int k = k0 + 32 * q;
      x[q] = k < a.n3 ? __ldcg(row + k) : (TIn)0;
    }
  };
  auto step = [&](int& rr, int& kk) {
    if (++kk == cpr) { kk = 0; rr += nw; }
  };
  TIn xc[kU];
  if (rn < rend) {
    load_chunk(rn, kcn, xc);
    step(rn, kcn);
  }
  while (r < rend) {
    TIn xn[kU];
    if (rn < rend) load_chunk(rn, kcn, xn);
    const uint32_t wij = w1[i] + w2[jj];
    const int k0 = kc * 32 * kU + lane;
    int v[kU], t[kU], old[kU];
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      const int k = k0 + 32 * q;
      const uint32_t sq = wij + w3[k < a.n3 ? k : 0];
      float y = (float)xc[q] * sa;
      if (sb != 1.f) y *= sb;
      v[q] = __float2int_rn(__uint_as_float(__float_as_uint(y) ^ (sq & 0x80000000u)));
      t[q] = (int)(sq & (uint32_t)mask);
    }
    // the chunk's adds back to back (lanes beyond the row issue none); the returned values are
    // examined after the last one
#pragma unroll
    for (int q = 0; q < kU; ++q) {
      old[q] = 0;
      if (k0 + 32 * q < a.n3) old[q] = atomicAdd(&hist[t[q]], v[q]);
    }
    // |v| < 2^25 < 2^30: an add can wrap only if |old| >= 2^30; then the exact test, and a
    // carry of +-2^32 to the global array (rare)
    unsigned near = 0u;
#pragma unroll
    for (int q = 0; q < kU; ++q) near |= (unsigned)old[q] + 0x40000000u;
    if ((int)near < 0) {
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int sum = (int)((unsigned)old[q] + (unsigned)v[q]);
        if (((old[q] ^ sum) & (v[q] ^ sum)) < 0) atomicAdd(&carry[t[q]], v[q] > 0 ? 1 : -1);
      }
    }
#pragma unroll
    for (int q = 0; q < kU; ++q) xc[q] = xn[q];
    // next chunk: the row's (i, j) move on by nw rows when the row changes
    if (++kc == cpr) {
      kc = 0;
      r += nw;
      jj += nw;
      while (jj >= a.n2) { jj -= a.n2; ++i; }
    }
    if (rn < rend) step(rn, kcn);
  }
  __syncthreads();
  int* dst = a.part + ((size_t)blockIdx.y * a.B + m) * b;
  for (int c = tid; c < b; c += nt) dst[c] = hist[c];
}

// S[m][t] (+)= 2^(E-25) (sum over slabs of part[.][m][t] + 2^32 carry[m][t]) as the real part;
// the imaginary part is 0 (or left as it is when accumulating).  NaN if max|T| is not finite
// (also reported as TSK_ENONFINITE).
__global__ void __launch_bounds__(256) asym_fix_reduce_kernel(const int* __restrict__ part,
                                                              const int* __restrict__ carry,
                                                              const unsigned* maxbits, int nslab,
                                                              long long cells, float2* S,
                                                              int accumulate, int* status) {
  const FixScale fs = fix_scale(*maxbits);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    float v;
    if (fs.finite) {
      long long acc = (long long)carry[c] * 4294967296LL;
#pragma unroll 8
      for (int s = 0; s < nslab; ++s) acc += __ldcg(part + (size_t)s * cells + c);
      v = ldexpf(__ll2float_rn(acc), fs.e - kFixBits);
    } else {
      v = __int_as_float(0x7fc00000);
      if (c == 0) tsk_set_status(status, TSK_ENONFINITE);
    }
    if (accumulate) {
      S[c].x += v;
    } else {
      S[c] = make_float2(v, 0.f);
    }
  }
}

template <typename TIn>
static int launch_asym_fix(const AsymSketchArgs& a0, int B, float2* S, int accumulate,
                           tsk_ctx* ctx) {
  const int b = 1 << a0.log2b;
  const size_t smem = (size_t)b * sizeof(int) + (size_t)3 * a0.nmax * sizeof(uint32_t);
  if (smem > (size_t)ctx->max_smem_optin) return TSK_EUNSUPPORTED;
  auto kernel = sketch_asym_fix_kernel<TIn>;
  TSK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TSK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 1024, smem));
  if (per_sm < 1) per_sm = 1;
  long long nslab = ((long long)ctx->num_sms * per_sm) / B;
  if (nslab < 1) nslab = 1;
  const long long cap = (a0.rows * a0.n3 + 16383) / 16384;
  if (nslab > cap) nslab = cap < 1 ? 1 : cap;
  if (nslab > 65535) nslab = 65535;
  AsymFixArgs a{a0.T, a0.n1, a0.n2, a0.n3, a0.nmax, a0.h, a0.g, B, a0.log2b, a0.rows,
                (int)nslab, nullptr, nullptr, nullptr};
  const size_t cells = (size_t)B * b;
  const size_t head = ws_round(256) + ws_round(cells * sizeof(int));
  int rc = tsk_ws_reserve(ctx, head + ws_round((size_t)a.nslab * cells * sizeof(int)));
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  unsigned* maxbits = wc.take<unsigned>(64);
  a.carry = wc.take<int>(cells);
  a.part = wc.take<int>((size_t)a.nslab * cells);
  a.maxbits = maxbits;
  TSK_CUDA(cudaMemsetAsync(ctx->ws, 0, head, ctx->stream));
  dense_absmax_kernel<TIn><<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(
      static_cast<const TIn*>(a0.T), a0.rows * a0.n3, maxbits);
  TSK_CHECK_LAUNCH();
  kernel<<<dim3(B, (unsigned)a.nslab), 1024, smem, ctx->stream>>>(a);
  TSK_CHECK_LAUNCH();
  long long blocks = ((long long)cells + 255) / 256;
  if (blocks > (long long)ctx->num_sms * 8) blocks = (long long)ctx->num_sms * 8;
  asym_fix_reduce_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(
      a.part, a.carry, maxbits, a.nslab, (long long)cells, S, accumulate, ctx->status);
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

// colliding sketches of the wedge entries whose first index lies in [p0, p1) (arguments checked
// by the callers)
static int sketch_sym_planes(tsk_ctx* ctx, const void* T, int in_dtype, int n, int p0, int p1,
                             const int32_t* h, const uint8_t* g, int B, int log2b, void* S,
                             int acc_dtype, int accumulate) {
  if (p1 > p0 && log2b > 16) return TSK_EUNSUPPORTED;
  const size_t b = (size_t)1 << log2b;
  if (acc_dtype == TSK_C64 && p1 > p0) {
    // complex-float sketches: exact int32 accumulation (writes or adds S itself)
    if (in_dtype == TSK_F32) return launch_sym_fix<float>(T, n, p0, p1, h, g, B, log2b, S, accumulate, ctx);
    if (in_dtype == TSK_F64) return launch_sym_fix<double>(T, n, p0, p1, h, g, B, log2b, S, accumulate, ctx);
    return launch_sym_fix<int32_t>(T, n, p0, p1, h, g, B, log2b, S, accumulate, ctx);
  }
  const size_t elem = acc_dtype == TSK_C64 ? sizeof(float) : 8;
  if (!accumulate) TSK_CUDA(cudaMemsetAsync(S, 0, (size_t)B * b * 2 * elem, ctx->stream));
  if (p1 <= p0) return TSK_OK;
  auto tet = [](long long x) { return x * (x + 1) * (x + 2) / 6; };
  const long long E0 = tet(n) - tet(n - p0);
  const long long W = tet(n - p0) - tet(n - p1);
  SymSketchArgs a{T, n, h, g, log2b, W, E0, 1, S, 0};
  if (acc_dtype == TSK_C128) {
    if (in_dtype == TSK_F32) return launch_sym<float, double, 2>(a, B, ctx);
    return launch_sym<double, double, 2>(a, B, ctx);
  }
  return launch_sym<int32_t, long long, 2>(a, B, ctx);
}

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
  if (M == 1) {
    const int n = (int)dims_host[0];
    return sketch_sym_planes(ctx, T, in_dtype, n, 0, n, h, g, B, log2b, S, acc_dtype, accumulate);
  }
  const int n1 = (int)dims_host[0], n2 = (int)dims_host[1], n3 = (int)dims_host[2];
  const int nmax = n1 > n2 ? (n1 > n3 ? n1 : n3) : (n2 > n3 ? n2 : n3);
  AsymSketchArgs a{T, n1, n2, n3, nmax, h, g, log2b, (long long)n1 * n2, 1, S};
  if (acc_dtype == TSK_C64 && n1 > 0 && n2 > 0 && n3 > 0) {
    // complex-float sketches: exact int32 accumulation (writes or adds S itself)
    if (log2b > 15) return TSK_EUNSUPPORTED;
    float2* Sf = static_cast<float2*>(S);
    if (in_dtype == TSK_F32) return launch_asym_fix<float>(a, B, Sf, accumulate, ctx);
    if (in_dtype == TSK_F64) return launch_asym_fix<double>(a, B, Sf, accumulate, ctx);
    return launch_asym_fix<int32_t>(a, B, Sf, accumulate, ctx);
  }
  if (!accumulate) TSK_CUDA(cudaMemsetAsync(S, 0, (size_t)B * b * 2 * elem, ctx->stream));
  if (n1 == 0 || n2 == 0 || n3 == 0) return TSK_OK;
  if (log2b > 14) return TSK_EUNSUPPORTED;
  if (acc_dtype == TSK_C128) {
    if (in_dtype == TSK_F32) return launch_asym<float, double>(a, B, ctx);
    return launch_asym<double, double>(a, B, ctx);
  }
  return launch_asym<int32_t, long long>(a, B, ctx);
}

extern "C" int sketch_tensor_planes(tsk_ctx* ctx, const void* T, int in_dtype, int n,
                                    int plane_begin, int plane_end, const int32_t* h,
                                    const uint8_t* g, int B, int log2b, void* S, int acc_dtype,
                                    int accumulate) {
  if (!ctx || (!T && plane_end > plane_begin) || !h || !g || !S) return TSK_EINVAL;
  if (B < 1 || log2b < 1 || log2b > 24 || n < 0) return TSK_EINVAL;
  if (plane_begin < 0 || plane_end < plane_begin || plane_end > n) return TSK_EINVAL;
  if (in_dtype != TSK_F32 && in_dtype != TSK_F64 && in_dtype != TSK_I32) return TSK_EINVAL;
  if (acc_dtype != TSK_C64 && acc_dtype != TSK_C128 && acc_dtype != TSK_CI64) return TSK_EINVAL;
  if (acc_dtype == TSK_CI64 && in_dtype != TSK_I32) return TSK_EINVAL;
  if (acc_dtype == TSK_C128 && in_dtype == TSK_I32) return TSK_EINVAL;
  if (n > 8192) return TSK_EUNSUPPORTED;
  // the kernels address plane i at (i n) n entries from the tensor's origin; T starts at plane
  // plane_begin, so the origin is moved back by that many planes (only planes >= plane_begin
  // are read)
  const size_t esz = in_dtype == TSK_F64 ? 8 : 4;
  const void* T0 = plane_end > plane_begin
                       ? reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(T) -
                                                       (uintptr_t)plane_begin * n * n * esz)
                       : nullptr;
  return sketch_sym_planes(ctx, T0, in_dtype, n, plane_begin, plane_end, h, g, B, log2b, S,
                           acc_dtype, accumulate);
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
