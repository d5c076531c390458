// Whitened third-moment accumulation on the tensor cores (App. D, Alg. 3: the sketch of
// M3(W,W,W) starts from the dense k x k x k moment).  For document weights w_d = 1 / (m_d (m_d - 1)
// (m_d - 2)) and whitened documents p_d = W^T n_d (rows of P), the wedge of
//   E3[a][b][c] = sum_d w_d p_da p_db p_dc
// is the product of X[(a,b)][d] = w_d p_da p_db (one row per pair a <= b) with P: a GEMM of
// k (k + 1) / 2 rows, k columns and D as the contraction dimension.  It runs as tcgen05.mma
// kind::tf32 with the FP32 operands split into TF32 hi + lo parts, both rounded to nearest, and
// three products per step (hi lo + lo hi first, then hi hi), which keeps each product to about
// 2^-22 relative without a bias of one sign; the accumulator lives in tensor memory.
//
// One CTA (512 build threads and one MMA warp) takes 128 pairs and one contiguous range of documents, 32 documents per
// step.  The step's rows of P arrive in shared memory by one bulk copy issued two steps ahead.
// Every warp builds a 32-row x 8-document block of X (its lanes' pairs, in registers) and writes
// it, split into TF32 hi and lo, to the step's A stage in tensor memory (rows = lanes); the warps
// also build P^T as the K-major B operand (8-row x 16-byte core matrices, no swizzle) in the
// step's shared-memory stage.  One thread issues the step's 12 MMAs (A from tensor memory, B from
// shared memory) and commits them to the stage's mbarrier; while they run, all warps add the
// previous step's accumulator into a running sum.  Each step accumulates into one of two
// tensor-memory accumulators from zero (the tensor cores' FP32 accumulation is not rounded to
// nearest, so its runs are kept to one step's 12 MMAs); the running sum is an FP32 add rounded
// to nearest in a third region.  Each CTA writes its sum in FP64 to its split's partial.
#include "common.cuh"
#include "moments_tc.cuh"

namespace tsk {
namespace {

constexpr int kTcRows = 128;         // pairs per CTA (MMA M)
constexpr int kTcDocs = 32;          // documents per step (4 MMA K-steps of 8)
constexpr int kTcColAcc1 = 128;      // tensor-memory column of the second step accumulator
constexpr int kTcColSum = 256;       // ... and of the running sum
constexpr int kTcTmemCols = 512;
constexpr long long kTcSpinLimit = 1ll << 22;   // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major without swizzle: start address, LBO (between core
// matrices adjacent along K) and SBO (between adjacent 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                  "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                  "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                  "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])));
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away from zero: adding
// half a unit of the 13 dropped bits to the magnitude bits and clearing them carries into the
// exponent when it should (finite x well below the float range).  The split x = hi + lo uses
// hi = tf32_rn(x) and lo = tf32_rn(x - hi): x - hi is exact in FP32 and at most 2^-11 |x|, and
// rounding it costs at most 2^-22 |x|.  Both roundings are to nearest, so that their errors do
// not add up with one sign over the many documents of a sum (truncation would: a bias of about
// 2^-21 per product, which the cancellation between the moment's terms magnifies).  Two integer
// operations, on the full-rate ALU.
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
               :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                  "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])));
}

constexpr int kTcWarps = 16;   // build and merge warps; warp 16 issues the MMAs
// Steps per accumulation run: a run's MMAs accumulate in one tensor-memory accumulator (the
// tensor cores' FP32 additions are not rounded to nearest), which is then folded into the FP32
// running sum with round-to-nearest.
constexpr int kTcRun = 2;
constexpr int kTcThreads = (kTcWarps + 1) * 32;
constexpr int kTcColA = 384;   // A operand stages: stage s hi at 384 + 64 s, lo 32 columns on

__global__ void __launch_bounds__(kTcThreads, 1) moments3_tc_kernel(Moments3TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t done[2];   // MMAs of a step (its stage, its accumulator) done
  __shared__ __align__(8) uint64_t full[2];   // operands of a step built
  __shared__ __align__(8) uint64_t pbar[2];   // rows of P of a step arrived
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(16) float wdoc[2][kTcDocs];
  __shared__ int s_abort;
  const int N = a.N, k = a.k, kp = a.kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bstage = 2 * N * kTcDocs * 4;                                // B hi + lo
  float* Ps0 = reinterpret_cast<float*>(sm + 2 * bstage);              // [2][kTcDocs][kp]
  const int tile = blockIdx.x, split = blockIdx.y;
  // this CTA's documents: steps [st0, st1) of 32 documents
  const long long steps_all = (a.D + kTcDocs - 1) / kTcDocs;
  const long long per = (steps_all + gridDim.y - 1) / gridDim.y;
  const long long st0 = (long long)split * per;
  const long long st1 = st0 + per < steps_all ? st0 + per : steps_all;
  const long long nsteps = st1 > st0 ? st1 - st0 : 0;
  // A: warp w writes tensor-memory lanes (rows) 32 q .. 32 q + 31, q = w mod 4, columns of
  // documents 8 ch .. 8 ch + 7, ch = w / 4; its lane's row is pair p = b (b + 1) / 2 + a
  const int q = warp & 3, ch = warp >> 2;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  int pa, pb;
  {
    const long long p = (long long)tile * kTcRows + 32 * q + lane;
    int bb = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((long long)(bb + 1) * (bb + 2) / 2 <= p) ++bb;
    while (bb > 0 && (long long)bb * (bb + 1) / 2 > p) --bb;
    const bool valid = p < a.npairs;
    pa = valid ? (int)(p - (long long)bb * (bb + 1) / 2) : -1;
    pb = valid ? bb : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&pbar[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  // document weights w_d = 1 / (m_d (m_d - 1) (m_d - 2)) (m_d >= 3), by the last warp: the
  // lengths of step i are loaded into a register two steps ahead
  const bool wwarp = warp == kTcWarps - 1;
  auto length = [&](long long i) {
    const long long d = (st0 + i) * kTcDocs + lane;
    return (wwarp && i < nsteps && d < a.D) ? __ldg(a.mdoc + d) : 0.f;
  };
  auto weights = [&](float m, int buf) {
    if (wwarp) wdoc[buf][lane] = m >= 3.f ? 1.f / (m * (m - 1.f) * (m - 2.f)) : 0.f;
  };
  weights(length(0), 0);
  float mnext = length(1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // rows of P of local step i: one bulk copy of the step's contiguous [rows][kp] block
  long long last_fetch[2] = {-1, -1};
  auto fetch_rows = [&](long long i) {
    const long long d0 = (st0 + i) * kTcDocs;
    const long long rows = a.D - d0 < kTcDocs ? a.D - d0 : kTcDocs;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk_copy_g2s(smem_u32(Ps0 + (size_t)(i & 1) * kTcDocs * kp), a.P + d0 * kp,
                  (uint32_t)(rows * kp * sizeof(float)), smem_u32(&pbar[i & 1]));
    last_fetch[i & 1] = i;
  };
  if (tid == 0)
    for (long long i = 0; i < 2 && i < nsteps; ++i) fetch_rows(i);
  // running sum: warp w owns lanes 32 q .. and columns [ch N / 4, (ch + 1) N / 4)
  const int qcols = N / 4, c0 = ch * qcols;
  {
    const float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (warp < kTcWarps)
      for (int c = c0; c < c0 + qcols; c += 4) tmem_st4(tmem + lane_base + kTcColSum + c, z);
    asm volatile("tcgen05.wait::st.sync.aligned;");
  }
  // add the accumulator of the run ending at local step j (finished) into the running sum
  // (FP32, round to nearest)
  auto merge = [&](long long j) -> bool {
    bool ok = !*(volatile int*)&s_abort &&
              mbar_wait(smem_u32(&done[j & 1]), (uint32_t)((j >> 1) & 1));
    ok = __all_sync(0xffffffffu, ok);   // the tensor-memory accesses below are warp-wide
    if (!ok) return false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t accol = (uint32_t)((j / kTcRun) & 1) * kTcColAcc1;
    // 16 columns at a time (qcols <= 32): the loads first (4 columns each), one wait, the stores
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      if (h < qcols) {
        float acc[16], sum[16];
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
          if (h + c < qcols) {
            tmem_ld4(tmem + lane_base + accol + c0 + h + c, acc + c);
            tmem_ld4(tmem + lane_base + kTcColSum + c0 + h + c, sum + c);
          }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
          if (h + c < qcols) {
#pragma unroll
            for (int e = 0; e < 4; ++e) sum[c + e] += acc[c + e];
            tmem_st4(tmem + lane_base + kTcColSum + c0 + h + c, sum + c);
          }
        }
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
    return true;
  };
  // kind::tf32, D f32, A (tensor memory) and B tf32 and K-major, N, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                         ((uint32_t)(kTcRows >> 4) << 24);
  // B items it = tid, tid + 512 (< N 8): 16-byte column kc = it / N of row c = it % N
  int bkc[2], bc[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int it = tid + kTcWarps * 32 * j;
    bkc[j] = it < N * (kTcDocs / 4) ? it / N : -1;
    bc[j] = it < N * (kTcDocs / 4) ? it % N : 0;
  }
  long long issued = 0;
  if (warp == kTcWarps) {
    // ---------------- MMA warp: step i's 12 MMAs once its operands are built, A from tensor
    // memory, B from shared memory, into accumulator (i / kTcRun) mod 2, from zero at the start
    // of each run of kTcRun steps
    if (lane == 0) {
      const uint32_t bbytes = (uint32_t)(N * kTcDocs * 4);
      for (long long i = 0; i < nsteps; ++i) {
        const int stg = (int)(i & 1);
        const bool ok = !*(volatile int*)&s_abort &&
                        mbar_wait(smem_u32(&full[stg]), (uint32_t)((i >> 1) & 1));
        if (!ok) { atomicExch(&s_abort, 1); break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t bb = smem_u32(sm + stg * bstage);
        const uint32_t dcol = tmem + (uint32_t)((i / kTcRun) & 1) * kTcColAcc1;
        const uint32_t acol = tmem + kTcColA + 64u * stg;
        // the small terms (hi lo, lo hi) first, then hi hi: the accumulator's FP32 additions are
        // not rounded to nearest, and an addition costs up to one unit in the last place of the
        // accumulator, so the adds made while it is still small cost little
#pragma unroll
        for (int pass = 1; pass < 4; ++pass) {
#pragma unroll
          for (int ks = 0; ks < kTcDocs / 8; ++ks) {
            const uint32_t at = acol + (pass == 2 ? 32u : 0u) + 8u * ks;
            const uint64_t bd = smem_desc(bb + (pass == 1 ? bbytes : 0u) + ks * 256, 128, 1024);
            const uint32_t acc = (ks == 0 && pass == 1 && (i % kTcRun) == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
                :: "r"(dcol), "r"(at), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
            :: "r"(smem_u32(&done[stg])));
      }
    }
    __syncwarp();
  } else for (long long i = 0; i < nsteps; ++i) {
    const int stg = (int)(i & 1);
    unsigned char* bbase = sm + stg * bstage;
    const float* Ps = Ps0 + (size_t)stg * kTcDocs * kp;
    const long long d0 = (st0 + i) * kTcDocs;
    const int nv = (int)(a.D - d0 < kTcDocs ? a.D - d0 : kTcDocs);   // documents of this step
    // this step's rows (fetched two steps ahead), and its stage, released by step i - 2's MMAs
    if (!*(volatile int*)&s_abort && !mbar_wait(smem_u32(&pbar[stg]), (uint32_t)((i >> 1) & 1)))
      atomicExch(&s_abort, 1);
    if (i >= 2 && !*(volatile int*)&s_abort &&
        !mbar_wait(smem_u32(&done[stg]), (uint32_t)(((i - 2) >> 1) & 1)))
      atomicExch(&s_abort, 1);
    // A: X[m][d] = w_d p_da p_db (0 past the last document) -> tensor memory, tf32 hi and lo
    {
      const float4 w0 = reinterpret_cast<const float4*>(wdoc[stg])[2 * ch];
      const float4 w1 = reinterpret_cast<const float4*>(wdoc[stg])[2 * ch + 1];
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      float hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = 8 * ch + j;
        const float x = (pa >= 0 && d < nv) ? w[j] * Ps[d * kp + pa] * Ps[d * kp + pb] : 0.f;
        hi[j] = tf32_rn(x);
        lo[j] = tf32_rn(x - hi[j]);
      }
      const uint32_t acol = tmem + lane_base + kTcColA + 64u * stg + 8u * ch;
      tmem_st8(acol, hi);
      tmem_st8(acol + 32u, lo);
    }
    // B: P^T[c][d] (c < k and d < nv, zero elsewhere) -> shared memory, slot ((c / 8) 8 + kc) 8
    // + c % 8 of 16 bytes; a warp covers one 4-document column and consecutive c
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (bkc[j] < 0) continue;
      const int kc = bkc[j], c = bc[j];
      const int slot = ((c >> 3) * 8 + kc) * 8 + (c & 7);
      float y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int d = 4 * kc + e;
        y[e] = (c < k && d < nv) ? Ps[d * kp + c] : 0.f;
      }
      const float4 hi = make_float4(tf32_rn(y[0]), tf32_rn(y[1]), tf32_rn(y[2]), tf32_rn(y[3]));
      reinterpret_cast<float4*>(bbase)[slot] = hi;
      reinterpret_cast<float4*>(bbase + N * kTcDocs * 4)[slot] =
          make_float4(tf32_rn(y[0] - hi.x), tf32_rn(y[1] - hi.y), tf32_rn(y[2] - hi.z),
                      tf32_rn(y[3] - hi.w));
    }
    // the next step's weights (their buffer was last read in step i - 1); the lengths of
    // step i + 2 start loading
    if (i + 1 < nsteps) weights(mnext, stg ^ 1);
    mnext = length(i + 2);
    asm volatile("tcgen05.wait::st.sync.aligned;");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("bar.sync 1, %0;" :: "r"(kTcWarps * 32) : "memory");
    if (*(volatile int*)&s_abort) break;
    // operands of step i built: the MMA warp may go; then the rows of step i + 2 into the
    // buffer this step has finished with
    if (tid == 0) {
      mbar_arrive(smem_u32(&full[stg]));
      if (i + 2 < nsteps) fetch_rows(i + 2);
    }
    issued = i + 1;
    // while these MMAs run: fold the previous run's accumulator (ending at step i - 1) into the
    // running sum, which releases it for the run starting at step i + kTcRun
    if (i >= kTcRun && (i % kTcRun) == 0 && !merge(i - 1)) atomicExch(&s_abort, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (warp < kTcWarps && !*(volatile int*)&s_abort && issued > 0 && !merge(issued - 1))
    atomicExch(&s_abort, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*(volatile int*)&s_abort) {
    // copies and MMAs in flight get a bounded chance to land before the memory is released
    if (tid == 0) {
      for (int s = 0; s < 2; ++s)
        if (last_fetch[s] >= 0) mbar_wait(smem_u32(&pbar[s]), (uint32_t)((last_fetch[s] >> 1) & 1));
      if (issued > 0) mbar_wait(smem_u32(&done[(issued - 1) & 1]), (uint32_t)(((issued - 1) >> 1) & 1));
      tsk_set_status(a.status, TSK_ETIMEOUT);
    }
  } else if (warp < kTcWarps) {
    // the running sum, in FP64, to this split's partial [split][pair row][column]
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = 32 * q + lane;
    double* out = a.part + ((size_t)split * a.rows_pad + (size_t)tile * kTcRows + row) * N;
    for (int c = c0; c < c0 + qcols; c += 4) {
      float sum[4];
      tmem_ld4(tmem + lane_base + kTcColSum + c, sum);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int e = 0; e < 4; ++e) out[c + e] = (double)sum[e];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcTmemCols));
}

}  // namespace

size_t moments3_tc_smem(int N, int kp) {
  return 2 * (size_t)(2 * N * kTcDocs * 4) + 2 * (size_t)kTcDocs * kp * sizeof(float);
}

int moments3_tc_splits(int npairs, int num_sms, long long D) {
  const int tiles = (npairs + kTcRows - 1) / kTcRows;
  // a whole number of waves of one CTA per SM when possible, at least 1024 documents a split
  int g = num_sms, t = tiles;
  while (t) { const int r = g % t; g = t; t = r; }
  long long S = num_sms / g;
  while (S * tiles < num_sms) S += num_sms / g;
  const long long cap = (D + 1023) / 1024;
  if (S > cap) S = cap;
  return (int)(S < 1 ? 1 : S);
}

int launch_moments3_tc(const Moments3TcArgs& a, int splits, cudaStream_t st) {
  const size_t smem = moments3_tc_smem(a.N, a.kp);
  TSK_CUDA(cudaFuncSetAttribute(moments3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  const int tiles = (int)(a.rows_pad / kTcRows);
  moments3_tc_kernel<<<dim3(tiles, splits), kTcThreads, smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

}  // namespace tsk
