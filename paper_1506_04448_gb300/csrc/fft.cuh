// Block-wide power-of-two FFTs over shared memory (Stockham auto-sort, radix <= 16).
//
// The DFTs of Eq. 4 and Prop. 1 are computed by one thread block per transform.  The data live
// in shared memory in the padded layout of pad_idx(); each pass loads E = N/NT elements per
// thread into registers, applies twiddles and radix-R DFTs in registers, synchronises, and
// stores to the Stockham output positions -- so transforms run in place without a second
// buffer.  Output is in natural order.  DIR = -1 is the forward transform exp(-2 pi i f t/N),
// DIR = +1 the unnormalised inverse (callers apply 1/N).
//
// Pass structure (Stockham auto-sort): with NS = product of the radices already applied,
// butterfly j reads x[j + r N/R] (r < R), multiplies element r by w_{NS R}^{DIR r (j mod NS)},
// takes an R-point DFT and writes element r to x[(j / NS) NS R + (j mod NS) + r NS].
//
// Slot ownership: thread t runs butterflies j = t + q NT, so the first pass reads, and the last
// pass (NS = N/R, j < NS) writes, exactly the slots t + NT s (s < N/NT) -- whatever the radices.
// The last pass is therefore in place per thread and needs no barrier between its loads and
// stores, and a pointwise step between a forward and an inverse transform that touches only the
// thread's own slots t + NT s needs no barrier before or after it.
#pragma once

#include "common.cuh"

namespace tsk {

// z * (DIR * i)
template <int DIR>
TSK_HD float2 mul_dir_i(float2 z) {
  return DIR > 0 ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// z * (c + DIR * s * i) for constants c, s
template <int DIR>
TSK_HD float2 mul_const(float2 z, float c, float s) {
  const float sd = DIR > 0 ? s : -s;
  return make_float2(z.x * c - z.y * sd, z.x * sd + z.y * c);
}

// cos and sin of pi/8, pi/4 (exact decimal expansions of the mathematical constants)
#define TSK_C8 0.92387953251128675613f
#define TSK_S8 0.38268343236508977173f
#define TSK_R2 0.70710678118654752440f

// z * w16^e with w16 = exp(DIR 2 pi i / 16), e in [0, 8); e is a compile-time constant after
// unrolling, so the branches fold away.
template <int DIR>
TSK_HD float2 mul_w16(float2 z, int e) {
  switch (e) {
    case 0: return z;
    case 1: return mul_const<DIR>(z, TSK_C8, TSK_S8);
    case 2: return mul_const<DIR>(z, TSK_R2, TSK_R2);
    case 3: return mul_const<DIR>(z, TSK_S8, TSK_C8);
    case 4: return mul_dir_i<DIR>(z);
    case 5: return mul_const<DIR>(z, -TSK_S8, TSK_C8);
    case 6: return mul_const<DIR>(z, -TSK_R2, TSK_R2);
    default: return mul_const<DIR>(z, -TSK_C8, TSK_S8);
  }
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
// Reverse the low BITS (<= 4) bits of x, without recursion so that it folds after unrolling.
template <int BITS>
__host__ __device__ constexpr int bitrev(int x) {
  static_assert(BITS >= 0 && BITS <= 4, "up to 4 bits");
  const int r = ((x & 1) << 3) | ((x & 2) << 1) | ((x & 4) >> 1) | ((x & 8) >> 3);
  return r >> (4 - BITS);
}

// One radix-2 decimation-in-frequency stage with butterfly distance SPAN, then the next.
template <int R, int DIR, int SPAN>
TSK_HD void dif_stage(float2* v) {
#pragma unroll
  for (int gbase = 0; gbase < R; gbase += 2 * SPAN) {
#pragma unroll
    for (int s = 0; s < SPAN; ++s) {
      const float2 a = v[gbase + s], c = v[gbase + s + SPAN];
      v[gbase + s] = cadd(a, c);
      v[gbase + s + SPAN] = mul_w16<DIR>(csub(a, c), s * (8 / SPAN));
    }
  }
  if constexpr (SPAN > 1) dif_stage<R, DIR, SPAN / 2>(v);
}

// In-place radix-2 decimation-in-frequency DFT of R <= 16 points held in registers.
// X_s = sum_r v_r exp(DIR 2 pi i r s / R) ends up in v[bitrev<log2 R>(s)].
template <int R, int DIR>
TSK_HD void dft_dif(float2* v) {
  static_assert(R == 2 || R == 4 || R == 8 || R == 16, "radix");
  dif_stage<R, DIR, R / 2>(v);
}

// Twiddle table: w^m for w = exp(-2 pi i / 2^15) and m < 2^15 as the product of two tables,
// lo[m & 255] * hi[m >> 8].  It lives in shared memory (3 KB) and is filled once per block by
// fill_twiddles(); one lookup replaces a sincospif call per butterfly.  The 256 entries of lo are
// stored XOR-swizzled, entry i at tw_lo_slot(i) (the low four index bits XORed with the high
// four): a Stockham pass looks up i = s k for consecutive k and a power-of-two stride s, and in
// linear order those entries share a few banks (up to 16-way conflicts for s = 16); swizzled,
// every distinct entry of a half-warp's lookup falls in its own bank pair.
constexpr int kTwLog = 15;
constexpr int kTwLo = 256;
constexpr int kTwEntries = kTwLo + (1 << kTwLog) / kTwLo;

TSK_HD constexpr int tw_lo_slot(int i) { return (i & 0xF0) | ((i ^ (i >> 4)) & 0xF); }

__device__ __forceinline__ void fill_twiddles(float2* tw, int nt) {
  for (int j = threadIdx.x; j < kTwEntries; j += nt) {
    // tw_lo_slot is an involution: slot j < 256 holds lo entry tw_lo_slot(j)
    const int m = j < kTwLo ? tw_lo_slot(j) : (j - kTwLo) * kTwLo;
    float s, c;
    sincospif(-2.f * (float)m / (float)(1 << kTwLog), &s, &c);
    tw[j] = make_float2(c, s);
  }
  __syncthreads();
}

// exp(DIR * 2 pi i * k / span), span a power of two <= 2^15, 0 <= k < span.
TSK_HD float2 unit_root(const float2* tw, int k, int span, int dir) {
#ifdef __CUDA_ARCH__
  const int m = k * ((1 << kTwLog) / span);
  const float2 w = cmul(tw[tw_lo_slot(m & (kTwLo - 1))], tw[kTwLo + (m >> 8)]);
  return dir > 0 ? cconj(w) : w;
#else
  (void)tw;
  const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)span;
  return make_float2((float)cos(a), (float)(dir > 0 ? sin(a) : -sin(a)));
#endif
}

// exp(DIR * 2 pi i * k / span) for spans up to 2^16: a 2^16 root with an odd exponent is the
// table's 2^15 root times exp(DIR * 2 pi i / 2^16) (used by the sketch-length splits only).
__device__ __forceinline__ float2 unit_root_wide(const float2* tw, int k, int span, int dir) {
  if (span <= (1 << kTwLog)) return unit_root(tw, k, span, dir);
  const float2 w = unit_root(tw, k >> 1, span >> 1, dir);
  if (!(k & 1)) return w;
  // cos and sin of 2 pi / 2^16 (decimal expansions of the mathematical constants)
  const float2 r = make_float2(0.99999999540410766f, dir > 0 ? 9.5873799095977345e-5f
                                                             : -9.5873799095977345e-5f);
  return cmul(w, r);
}

// exp(dir * 2 pi i * k / 2^logspan), 0 <= k < 2^logspan <= 2^16, by sincospif of the exact
// argument 2k / 2^logspan instead of the shared table: for indices that differ randomly across a
// warp (hashed positions) each table lookup costs several shared-memory wavefronts.
__device__ __forceinline__ float2 unit_root_direct(int k, int logspan, int dir) {
  float s, c;
  sincospif((float)(dir > 0 ? 2 * k : -2 * k) / (float)(1 << logspan), &s, &c);
  return make_float2(c, s);
}

// v[r] *= w^r, w = exp(DIR 2 pi i k / span), r = 1..R-1.  w^2, w^4, w^8 are formed by
// squaring and the odd powers by one extra product, so at most four roundings separate any
// power from the table value of w.
template <int R, int DIR>
TSK_HD void twiddle(float2* v, const float2* tw, int k, int span) {
  const float2 w1 = unit_root(tw, k, span, DIR);
  v[1] = cmul(v[1], w1);
  if constexpr (R >= 4) {
    const float2 w2 = cmul(w1, w1);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], cmul(w2, w1));
    if constexpr (R >= 8) {
      const float2 w4 = cmul(w2, w2);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], cmul(w4, w1));
      const float2 w6 = cmul(w4, w2);
      v[6] = cmul(v[6], w6);
      v[7] = cmul(v[7], cmul(w6, w1));
      if constexpr (R >= 16) {
        const float2 w8 = cmul(w4, w4);
#pragma unroll
        for (int r = 8; r < 16; ++r) {
          float2 t = w8;
          if (r & 4) t = cmul(t, w4);
          if (r & 2) t = cmul(t, w2);
          if (r & 1) t = cmul(t, w1);
          v[r] = cmul(v[r], t);
        }
      }
    }
  }
}

template <int N, int NT, int R, int NS, int DIR>
struct StockhamPass {
  static constexpr int E = N / NT;
  static constexpr int NB = E / R;
  static_assert(NB * R == E, "elements per thread must be a multiple of the radix");

  static TSK_HD void load_compute(const float2* x, const float2* tw, int tid, float2* v) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tid + q * NT;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = x[pad_idx(j + r * (N / R))];
      if constexpr (NS > 1) twiddle<R, DIR>(v + q * R, tw, j & (NS - 1), NS * R);
      dft_dif<R, DIR>(v + q * R);
    }
  }
  static TSK_HD void store(float2* x, int tid, const float2* v) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tid + q * NT;
      const int k = j & (NS - 1);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[pad_idx(base + r * NS)] = v[q * R + bitrev<ilog2(R)>(r)];
    }
  }
};

template <int N, int NT, int NS, int DIR>
struct FftPasses {
  static constexpr int E = N / NT;
  static constexpr int REM = N / NS;
  static constexpr int RMAX = E > 16 ? 16 : E;
  static constexpr int R = REM >= RMAX ? RMAX : REM;
  static __device__ __forceinline__ void run(float2* x, const float2* tw) {
    float2 v[E];
    StockhamPass<N, NT, R, NS, DIR>::load_compute(x, tw, threadIdx.x, v);
    if constexpr (NS * R < N) __syncthreads();       // the last pass is in place per thread
    StockhamPass<N, NT, R, NS, DIR>::store(x, threadIdx.x, v);
    __syncthreads();
    if constexpr (NS * R < N) FftPasses<N, NT, NS * R, DIR>::run(x, tw);
  }
};

// Two independent in-place transforms (NA points at xa, NE points at xe, same direction) whose
// passes are interleaved: step p runs pass p of A (load, sync, store) and then pass p of E
// (load, sync, store).  E's barrier also orders A's stores before A's next loads, and A's next
// barrier orders E's stores before E's next loads, so a step costs two barriers where the two
// transforms run one after the other would cost four.  An extra barrier is taken only when a
// step lacks one of the two parts.  PREV_E: the previous step ended with an E part.  A final
// pass skips its own load/store barrier (it is in place per thread) unless that barrier also
// orders the other transform's accesses.  FINAL_SYNC = false leaves out the closing barrier, for
// callers that next touch only their own slots t + NT s.
template <int NA, int NE, int NT, int NSA, int NSE, int DIR, bool PREV_E = true,
          bool FINAL_SYNC = true>
struct FftPair {
  static constexpr int EA = NA / NT, EE = NE / NT;
  static constexpr int RMA = EA > 16 ? 16 : EA, RME = EE > 16 ? 16 : EE;
  static constexpr bool DO_A = NSA < NA, DO_E = NSE < NE;
  static constexpr int RA = !DO_A ? 1 : (NA / NSA >= RMA ? RMA : NA / NSA);
  static constexpr int RE = !DO_E ? 1 : (NE / NSE >= RME ? RME : NE / NSE);
  static constexpr bool A_FINAL = DO_A && NSA * RA == NA, E_FINAL = DO_E && NSE * RE == NE;
  static __device__ __forceinline__ void run(float2* xa, float2* xe, const float2* tw) {
    if constexpr (DO_A) {
      if constexpr (!PREV_E) __syncthreads();
      float2 v[EA];
      StockhamPass<NA, NT, RA, NSA, DIR>::load_compute(xa, tw, threadIdx.x, v);
      // also orders E's previous stores before E's loads below
      if constexpr (!A_FINAL || DO_E) __syncthreads();
      StockhamPass<NA, NT, RA, NSA, DIR>::store(xa, threadIdx.x, v);
    }
    if constexpr (DO_E) {
      if constexpr (!DO_A) __syncthreads();
      float2 w[EE];
      StockhamPass<NE, NT, RE, NSE, DIR>::load_compute(xe, tw, threadIdx.x, w);
      // also orders A's stores above before A's next loads
      if constexpr (!E_FINAL || (DO_A && !A_FINAL)) __syncthreads();
      StockhamPass<NE, NT, RE, NSE, DIR>::store(xe, threadIdx.x, w);
    }
    if constexpr (DO_A || DO_E) {
      FftPair<NA, NE, NT, NSA * RA, NSE * RE, DIR, DO_E, FINAL_SYNC>::run(xa, xe, tw);
    } else if constexpr (FINAL_SYNC) {
      __syncthreads();
    }
  }
};

// block_fft of two arrays at once (xa: 2^LOGA points, xe: 2^LOGE points), interleaved as above.
// FINAL_SYNC = false: the caller next touches only each thread's own slots t + NT s of xa and xe.
template <int LOGA, int LOGE, int NT, int DIR, bool FINAL_SYNC = true>
__device__ __forceinline__ void block_fft_pair(float2* xa, float2* xe, const float2* tw) {
  constexpr int NA = 1 << LOGA, NE = 1 << LOGE;
  static_assert(NA / NT >= 2 && NA / NT <= 32 && NE / NT >= 2 && NE / NT <= 32, "2..32 per thread");
  static_assert(LOGA <= kTwLog && LOGE <= kTwLog, "twiddle table covers transforms up to 2^15");
  FftPair<NA, NE, NT, 1, 1, DIR, true, FINAL_SYNC>::run(xa, xe, tw);
}

// In-place FFT of N = 2^LOGN complex values at x (padded layout) by a block of exactly NT
// threads, with the twiddle table tw (fill_twiddles).  Must be called by all NT threads;
// begins and ends with the data synchronised.
template <int LOGN, int NT, int DIR>
__device__ __forceinline__ void block_fft(float2* x, const float2* tw) {
  constexpr int N = 1 << LOGN;
  constexpr int E = N / NT;
  static_assert(E >= 2 && E <= 32 && (E & (E - 1)) == 0, "2..32 elements per thread");
  static_assert(LOGN <= kTwLog, "twiddle table covers transforms up to 2^15");
  FftPasses<N, NT, 1, DIR>::run(x, tw);
}

// ------------------------------------------------------------------ real signals of length b
// A real signal x of length b = 2N is held as N complex values z_t = (x_2t, x_2t+1) in the padded
// layout; its half spectrum X_0..X_N (X_f = sum_t x_t exp(-2 pi i f t / b), the rest follows by
// Hermitian symmetry) is held as X_0..X_{N-1} in the same slots plus X_N in `last`.

// Forward: z -> half spectrum, in place.  Z = DFT_N(z), then for f = 0..N
//   X_f = (Z_f + conj Z_{N-f})/2 - i w^f (Z_f - conj Z_{N-f})/2,  w = exp(-2 pi i / b),  Z_N = Z_0.
template <int LOGB, int NT>
__device__ __forceinline__ void block_rfft(float2* x, float2* last, const float2* tw) {
  constexpr int N = 1 << (LOGB - 1);
  block_fft<LOGB - 1, NT, -1>(x, tw);
  // pairs (f, N - f), f = 0..N/2, are independent: each thread owns whole pairs
  for (int f = threadIdx.x; f <= N / 2; f += NT) {
    const float2 zf = x[pad_idx(f)];
    const float2 zg = x[pad_idx(f == 0 ? 0 : N - f)];   // Z_{N-f}
    auto untangle = [&](float2 a, float2 c, int ff) {
      const float2 e = cscale(cadd(a, cconj(c)), 0.5f);
      const float2 d = cscale(csub(a, cconj(c)), 0.5f);
      const float2 w = unit_root(tw, ff, 2 * N, -1);
      const float2 wd = cmul(w, d);
      return make_float2(e.x + wd.y, e.y - wd.x);          // e - i w d
    };
    if (f == 0) {
      *last = make_float2(zf.x - zf.y, 0.f);               // X_N = Re Z_0 - Im Z_0
      x[pad_idx(0)] = make_float2(zf.x + zf.y, 0.f);       // X_0 = Re Z_0 + Im Z_0
    } else {
      const float2 Xf = untangle(zf, zg, f);
      const float2 Xg = untangle(zg, zf, N - f);
      x[pad_idx(f)] = Xf;
      x[pad_idx(N - f)] = Xg;
    }
  }
  __syncthreads();
}

// Inverse: half spectrum -> z (the real signal, including the 1/b factor), in place.
//   E_f = (X_f + conj X_{N-f})/2,  O_f = w^{-f} (X_f - conj X_{N-f})/2,  Z_f = E_f + i O_f,
//   z = DFT_N^{-1}(Z) / N.
// SCALE = false leaves out the final 1/N (one shared-memory pass) for callers that fold it into
// what they do with z; the result is then N z.
template <int LOGB, int NT, bool SCALE = true>
__device__ __forceinline__ void block_irfft(float2* x, const float2* last, const float2* tw) {
  constexpr int N = 1 << (LOGB - 1);
  const float2 xN = *last;
  for (int f = threadIdx.x; f <= N / 2; f += NT) {
    const float2 Xf = x[pad_idx(f)];
    const float2 Xg = f == 0 ? xN : x[pad_idx(N - f)];    // X_{N-f}
    auto tangle = [&](float2 a, float2 c, int ff) {
      const float2 e = cscale(cadd(a, cconj(c)), 0.5f);
      const float2 d = cscale(csub(a, cconj(c)), 0.5f);
      const float2 o = cmul(unit_root(tw, ff, 2 * N, +1), d);
      return make_float2(e.x - o.y, e.y + o.x);           // e + i o
    };
    if (f == 0) {
      x[pad_idx(0)] = tangle(Xf, Xg, 0);
    } else {
      const float2 Zf = tangle(Xf, Xg, f);
      const float2 Zg = tangle(Xg, Xf, N - f);
      x[pad_idx(f)] = Zf;
      x[pad_idx(N - f)] = Zg;
    }
  }
  __syncthreads();
  block_fft<LOGB - 1, NT, +1>(x, tw);
  if constexpr (SCALE) {
    constexpr float invN = 1.f / (float)N;
    for (int t = threadIdx.x; t < N; t += NT) x[pad_idx(t)] = cscale(x[pad_idx(t)], invN);
    __syncthreads();
  }
}

// Real element k of a signal held as complex pairs in the padded layout.
__device__ __forceinline__ float& real_at(float2* x, int k) {
  return reinterpret_cast<float*>(&x[pad_idx(k >> 1)])[k & 1];
}

// Resident blocks per SM that the contraction kernels ask the compiler to fit.  With 16 elements
// per thread, 1024 threads per SM (64 registers per thread) fit without spills, and shared
// memory (about 12.75 b bytes per block) allows that many blocks for every b.  One-warp blocks
// (b <= 2^9) ask for half as many, and blocks with 32 elements per thread for one (they need
// more than 128 registers per thread).
constexpr int contract_min_blocks(int logb, int nt) {
  return (1 << logb) / nt > 16 ? 1 : (nt <= 32 ? 16 : 1024 / nt);
}

// Threads per block used by the sketch-length-b kernels: b/16 (one radix-16 butterfly, 16
// elements, per thread and pass of a length-b transform), at least one warp, at most 1024.
constexpr int threads_for_logb(int logb) {
  return (1 << logb) / 16 < 32 ? 32 : ((1 << logb) / 16 > 1024 ? 1024 : (1 << logb) / 16);
}

}  // namespace tsk
