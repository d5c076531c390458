/*
 * tsk.h -- C ABI of the GB300 (sm_103a) tensor-sketch library.
 *
 * Implements the hot path of the sketched robust tensor power method of Wang, Tung, Smola and
 * Anandkumar, "Fast and Guaranteed Tensor Decomposition via Sketching" (NIPS 2015):
 * colliding count sketches of symmetric tensors (Sec. 3.3), rank-1 sketches by FFT (Eq. 4),
 * the sketched contractions T^(I,u,u) and T^(u,u,u) read from inverse FFTs at hashed
 * positions (Prop. 1, App. B), the median over B sketches and deflation (Alg. 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers are DEVICE pointers owned by the caller unless the argument says "host".
 *   The library never frees or retains caller memory.
 * - Every call is asynchronous on the stream bound to the context (tsk_ctx_set_stream);
 *   results are valid once that stream has been synchronised.
 * - Argument errors are detected on the host before anything is enqueued: the call returns
 *   TSK_EINVAL (or TSK_EUNSUPPORTED for a valid but unimplemented size) and enqueues nothing.
 * - Errors found on the device (a zero or non-finite norm in a power update) are recorded
 *   in a status word of the context; tsk_ctx_status() synchronises and returns/clears it.
 * - A launch or allocation failure of the CUDA runtime returns TSK_ECUDA / TSK_ENOMEM.
 * - The only memory the library allocates is the context's scratch workspace (grown on
 *   demand, freed by tsk_ctx_destroy).
 * - b = 2^log2b is the sketch length.  Sketches are stored as [B][b] arrays of
 *   interleaved complex numbers (re, im).  DFTs are unnormalised forward
 *   F(x)_f = sum_t x_t exp(-2 pi i f t / b); inverse transforms carry 1/b.
 * - Hash tables: h int32 [B][M][nmax] with values in [0, b); g uint8 [B][M][nmax] with values
 *   in {0,1,2,3}.  M = 1 (colliding, symmetric sketch) or M = 3 (asymmetric sketch).  The
 *   complex sign is sigma(i) = sqrt(-1)^g(i) (Sec. 3.3, m = 4); the real sign of the
 *   asymmetric sketch is xi(i) = 1 - 2 (g(i) & 1) (Eq. 1).
 */
#ifndef TSK_H_
#define TSK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsk_ctx tsk_ctx;

enum tsk_status {
  TSK_OK = 0,
  TSK_EINVAL = -1,        /* bad argument (null pointer, size out of range, bad dtype) */
  TSK_ENOMEM = -2,        /* workspace allocation failed */
  TSK_ECUDA = -3,         /* CUDA runtime error (launch, copy, device query) */
  TSK_ETIMEOUT = -4,      /* reserved: a bounded device-side wait gave up */
  TSK_ENONFINITE = -5,    /* power update met ||v_bar|| = 0 or a non-finite norm */
  TSK_EUNSUPPORTED = -6   /* valid request outside the implemented sizes */
};

enum tsk_dtype {
  TSK_F32 = 0,   /* float */
  TSK_F64 = 1,   /* double */
  TSK_I32 = 2,   /* int32 */
  TSK_C64 = 3,   /* complex float, interleaved (re, im) */
  TSK_C128 = 4,  /* complex double, interleaved */
  TSK_CI64 = 5   /* complex int64, interleaved: exact integer sketches */
};

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` bound to `stream` (a cudaStream_t; NULL = legacy
 * default stream).  *out receives the handle.  Returns TSK_OK or TSK_ECUDA/TSK_EINVAL. */
int tsk_ctx_create(int device, void* stream, tsk_ctx** out);

/* Free the context's workspace and the context itself.  Synchronises its stream first. */
int tsk_ctx_destroy(tsk_ctx* ctx);

/* Re-bind the context to another stream of the same device (no host synchronisation).  The
 * context's workspace and status word are shared by the streams it is bound to, so work
 * enqueued after the re-binding waits on the device for the work already enqueued on the
 * previous stream (an event recorded there).  While either stream is being captured into a CUDA
 * graph nothing is recorded: the capturing caller orders its streams itself. */
int tsk_ctx_set_stream(tsk_ctx* ctx, void* stream);

/* Synchronise the context's stream, then return and clear the first device-side error
 * recorded since the last call (TSK_OK if none). */
int tsk_ctx_status(tsk_ctx* ctx);

/* Static, human-readable text for a status code. */
const char* tsk_strerror(int status);

/* ---------------------------------------------------------------- measured roofs (no counterpart in the paper) */

/* Micro-kernels for the roofs the kernels are measured against.  TSK_PEAK_FMA: FP32 FMA issue
 * (8 independent chains per thread, work in flops); TSK_PEAK_SMEM: conflict-free 16-byte shared
 * loads (work in bytes); TSK_PEAK_ATOMS: random-bucket int32 shared-memory adds that return the
 * old value, into a 128 KB histogram per SM as in the colliding build (work in adds).
 * tsk_peak_launch enqueues one launch of `iters` iterations on the context's stream (sink: a
 * device scratch word the kernels never actually write); the caller times it with events and
 * divides tsk_peak_work's figure for the same (kind, iters) by the time. */
enum tsk_peak_kind { TSK_PEAK_FMA = 0, TSK_PEAK_SMEM = 1, TSK_PEAK_ATOMS = 2 };
int tsk_peak_launch(tsk_ctx* ctx, int kind, int iters, void* sink);
int tsk_peak_work(tsk_ctx* ctx, int kind, int iters, double* work);

/* ---------------------------------------------------------------- hashing (Sec. 2, Sec. 3.3, Prop. 2) */

/* Draw the hash tables of B independent sketches.  For sketch m and mode j (j < M):
 *   h[m][j][i] = ((a_0 + a_1 i + ... + a_5 i^5) mod P) mod b      (6-wise independent, Prop. 2)
 *   g[m][j][i] = ((c_0 + c_1 i + ... + c_11 i^11) mod P) mod 4    (12-wise independent)
 * with P = 2^61 - 1 and coefficient e of table w (0 = h, 1 = g) equal to output number
 * ((m*M + j)*2 + w)*16 + e of the SplitMix64 stream started at `seed`, reduced mod P.
 * dims_host: host array of M mode sizes; nmax = max(dims_host).  Entries i >= dims[j] are
 * written as 0.  Requires 1 <= B, M in {1,3}, 1 <= log2b <= 24, 0 <= dims[j] < 2^31. */
int cs_hashes(tsk_ctx* ctx, uint64_t seed, int B, int log2b, int M, const int64_t* dims_host,
              int32_t* h, uint8_t* g);

/* ---------------------------------------------------------------- sketch construction (Eq. 1, Eq. 7) */

/* Tensor sketches of a dense row-major tensor T.
 * M = 1: colliding sketch of a SYMMETRIC n x n x n tensor (Eq. 7):
 *     S[m][t] = sum over ordered (i,j,k) with (h(i)+h(j)+h(k)) mod b = t of sigma_i sigma_j sigma_k T_ijk,
 *   computed from the entries with i <= j <= k only, each weighted by kappa in {1,3,6}
 *   (Sec. 3.3: all permutations of an entry collide); T must be symmetric.
 * M = 3: asymmetric sketch of an n1 x n2 x n3 tensor (Eq. 1), real-valued, stored with
 *   zero imaginary part: S[m][t] = sum_{(h1+h2+h3) mod b = t} xi1 xi2 xi3 T_ijk.
 * in_dtype: TSK_F32 | TSK_F64 | TSK_I32.  acc_dtype: TSK_C64 (complex float result, any input),
 *   TSK_C128 (double accumulation, F64 input) or TSK_CI64 (exact int64, I32 input).
 * TSK_C64 (M = 1 and M = 3): every entry read is rounded once to the integer grid 2^(E-25), where
 *   2^E is the smallest power of two above max|T| over the entries read (the wedge for M = 1,
 *   the whole tensor for M = 3), and the buckets are summed exactly in integers; the only other
 *   rounding is the final conversion to float.  The result does not depend on thread scheduling
 *   (two calls give identical bits).  A non-finite entry (or an FP64 entry beyond the float range)
 *   makes every value of S NaN and is reported by tsk_ctx_status() as TSK_ENONFINITE.  Uses
 *   context workspace of about (P + 1) * B * 2b * 4 bytes (M = 1) or (P + 1) * B * b * 4 bytes
 *   (M = 3), where P <= the number of SMs is the number of block partials per sketch.
 * S: [B][b] of acc_dtype.  accumulate = 0 overwrites S, 1 adds to it.
 * Limits: symmetric path log2b <= 16 (M = 1; above 2^14 the buckets are built in 2 or 4
 * ranges by separate blocks), asymmetric path log2b <= 15, n <= 8192. */
int sketch_tensor(tsk_ctx* ctx, const void* T, int in_dtype, int M, const int64_t* dims_host,
                  const int32_t* h, const uint8_t* g, int B, int log2b,
                  void* S, int acc_dtype, int accumulate);

/* Colliding sketches (M = 1) of the wedge entries i <= j <= k of a symmetric n x n x n tensor
 * whose first index i lies in [plane_begin, plane_end): the part of sketch_tensor's sum over
 * those planes.  Sketches are linear in the tensor (Sec. 3.1), so the sum of the sketches of a
 * partition of 0..n-1 into plane ranges, built on different devices and added (e.g. by an
 * all-reduce), is the sketch of the whole tensor: exactly with TSK_CI64, up to float rounding
 * with TSK_C64 (each part is rounded on its own grid, set by max|T| over its planes).
 * T: planes plane_begin .. plane_end - 1 only, [plane_end - plane_begin][n][n] row-major, i.e.
 *   the slice T[plane_begin:plane_end] of the full tensor (no other entries are read); may be
 *   NULL when the range is empty.
 * h, g: [B][n] hash tables as for sketch_tensor with M = 1.  Other arguments, workspace use,
 * status reporting and limits as for sketch_tensor with M = 1.  An empty range writes zeros
 * (accumulate = 0) or leaves S unchanged.
 * Returns TSK_EINVAL unless 0 <= plane_begin <= plane_end <= n. */
int sketch_tensor_planes(tsk_ctx* ctx, const void* T, int in_dtype, int n, int plane_begin,
                         int plane_end, const int32_t* h, const uint8_t* g, int B, int log2b,
                         void* S, int acc_dtype, int accumulate);

/* Batched length-b DFT of B complex float vectors (S_in, S_out: [B][b] TSK_C64; may alias).
 * inverse = 0: unnormalised forward transform; 1: inverse transform including 1/b. */
int sketch_fft(tsk_ctx* ctx, const float* S_in, float* S_out, int B, int log2b, int inverse);

/* Rank-1 sketches by FFT (Eq. 4, Sec. 3.1 linearity).  For every sketch m:
 *   M = 1 (colliding):  S[m] (+)= sum_c w[c] * (s~_{u_c} * s~_{u_c} * s~_{u_c})
 *   M = 3 (asymmetric): S[m] (+)= sum_c w[c] * (s_{1,u_c} * s_{2,v_c} * s_{3,w_c})
 * computed as F^{-1}(sum_c w_c F(s_1) o F(s_2) o F(s_3)).
 * w: [count] float; U: [count][n1], V: [count][n2], W: [count][n3] float (V, W only for M = 3);
 * dims_host: M mode sizes.  domain = 0 writes the time-domain sketch, 1 its DFT.
 * S: [B][b] TSK_C64; accumulate = 0 overwrites, 1 adds.  Uses count*B FFTs.
 * Limits: log2b in [8, 14]. */
int sketch_rank1(tsk_ctx* ctx, int64_t count, const float* w, const float* U, const float* V,
                 const float* W, int M, const int64_t* dims_host, const int32_t* h,
                 const uint8_t* g, int B, int log2b, int domain, float* S, int accumulate);

/* ---------------------------------------------------------------- contractions (Prop. 1, App. B) */

/* Sketched T^(I,u,u) for L vectors against B colliding sketches (M = 1).  For sketch m and
 * vector u = U[l] (used as given):
 *   v_i^(m) = Re[ 1/6 conj(sigma_i) (g_2 + g_1)[h_i] + 1/3 conj(sigma_i)^2 u_i g_0[2 h_i mod b]
 *               + 1/3 conj(sigma_i)^3 u_i^2 S[3 h_i mod b] ]
 * where g_0 = F^-1(FS o conj F s~_u), g_1 = F^-1(FS o conj F s~_{2,u o u}),
 *       g_2 = F^-1(FS o conj(F s~_u)^2)  (App. B, Eq. 14 with coefficients 1/3,1/6,1/6,1/3
 *       -- the printed 1 and 1 on the outer terms give a biased estimate).
 * FS: [B][b] TSK_C64 = DFT of S; S: [B][b] TSK_C64 time-domain sketch; U: [L][n] float.
 * Vmed: [L][n] float, median over m of v^(m) (mean of the two middle values for even B).
 * Vall: optional [L][B][n] float, every v^(m).  Without it the call may split each sketch's
 *   frequencies over several blocks as robust_power_method does (same result).
 * Limits: log2b in [8, 14], 1 <= B <= 64, 1 <= n <= 8192. */
int contract_iuu(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                 const uint8_t* g, int B, int log2b, const float* U, int L, int64_t n,
                 float* Vmed, float* Vall);

/* contract_iuu for callers that cannot allocate device memory.  The paper has no counterpart:
 * this is a deployment variant of contract_iuu with the same arguments and result (Vmed only).
 * Callers whose device memory belongs to another allocator, or whose loops forbid allocation
 * after start-up, cannot let the library cudaMalloc its workspace; this entry point allocates
 * nothing and needs no context.  Its scratch (per-sketch values, per-sketch
 * eigenvalue estimates, arrival counters) lives in one static device array of 4 MiB compiled
 * into the library, which every GPU that loads the library holds until the process exits.
 * stream: the cudaStream_t to enqueue on (NULL = legacy default stream); the current device is
 * used.  The first call on a device looks up the array's device address (cudaGetSymbolAddress).  Returns TSK_EUNSUPPORTED when the scratch,
 * L*B*n*4 + L*B*4 + L*4 bytes with each part rounded up to 256, would exceed 4 MiB.  All calls
 * share the array: calls whose kernels overlap on the GPU (e.g. on two streams) race.  Having no
 * context, it records no device status: a zero or non-finite input vector is not reported (its
 * output row is computed from it as given). */
int contract_iuu_static(const float* FS, const float* S, const int32_t* h, const uint8_t* g,
                        int B, int log2b, const float* U, int L, int64_t n, float* Vmed,
                        void* stream);

/* Sketched T^(u,u,u) (App. B, Eq. 13, all terms as time-domain inner products):
 *   lambda^(m) = Re[ 1/6 <S, s~_u * s~_u * s~_u> + 1/2 <S, s~_{2,u o u} * s~_u> + 1/3 <S, s~_{3,u o u o u}> ]
 * evaluated as (1/b) sum_f FS[f] conj(U_f^3/6 + V_f U_f/2) plus the sparse third term.
 * lam_med: [L] float, median over the B sketches; lam_all: optional [L][B] float.
 * Same limits as contract_iuu. */
int contract_uuu(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                 const uint8_t* g, int B, int log2b, const float* U, int L, int64_t n,
                 float* lam_med, float* lam_all);

/* ---------------------------------------------------------------- asymmetric sketches (Eq. 1, Alg. 2) */

/* Half spectra of real sketches: Xh[m][f] = sum_t Re(S[m][t]) exp(-2 pi i f t / b), f = 0..b/2.
 * S: [B][b] TSK_C64 (imaginary parts ignored, e.g. the asymmetric sketch of sketch_tensor with
 * M = 3); Xh: [B][b/2 + 1] TSK_C64.  Limits: log2b in [9, 15]. */
int sketch_rfft(tsk_ctx* ctx, const float* S, float* Xh, int B, int log2b);

/* Sketched T^(I,v,w) of an asymmetric sketch (Prop. 1 with two different vectors; the columns of
 * T_(1)(C (.) B) in Alg. 2).  For output mode `mode` (0, 1, 2) and the other modes p < q:
 *   v^(m)_i = xi_mode(i) [F^-1(Xh^(m) o conj F s_p,V[r] o conj F s_q,W[r])]_{h_mode(i)},
 * Vmed[r] = median over the B sketches.  Xh: [B][b/2+1] half spectra (sketch_rfft); h, g:
 * [B][3][nmax]; dims_host: the three mode sizes; V: [K][dims[p]], W: [K][dims[q]] float;
 * Vmed: [K][dims[mode]]; Vall: optional [K][B][dims[mode]].  Limits: log2b in [9, 15], B <= 64. */
int contract_ivw(tsk_ctx* ctx, const float* Xh, const int32_t* h, const uint8_t* g, int B,
                 int log2b, const int64_t* dims_host, int mode, const float* V, const float* W,
                 int K, float* Vmed, float* Vall);

/* Sketched CP loss and its adjoint (the paper's Eq. 2 inner-product estimator and the
 * linearity of Sec. 3.1 applied to a rank-R model; derived, not printed in the paper):
 *   loss = (1/B) sum_m || s_T^(m) - sum_r lam_r s^(m)_{A[r] (x) Bf[r] (x) C[r]} ||^2,
 * with s_{a(x)b(x)c} = s_1,a * s_2,b * s_3,c (Eq. 4).  The gradient with respect to a factor
 * row is a sketched T(I,v,w) contraction of the residual sketch:
 *   dloss/dA[r][i] = -(2 lam_r / B) sum_m xi_1(i) [F^-1(F R^(m) o conj F s_2,Bf[r] o conj F s_3,C[r])]_{h_1(i)}
 * (likewise Bf, C) and dloss/dlam_r = -(2/B) sum_m <R^(m), s^(m)_r>.
 * Xh: [B][b/2+1] half spectra of the tensor sketches; lam: [R]; A: [R][n1], Bf: [R][n2],
 * C: [R][n3] float (one component per row).  loss: one float (device).  The four gradient
 * outputs are all NULL (loss only) or all given (same shapes as lam, A, Bf, C).
 * Limits: log2b in [9, 15], R <= 4096. */
int cp_sketch_loss(tsk_ctx* ctx, const float* Xh, const int32_t* h, const uint8_t* g, int B,
                   int log2b, const int64_t* dims_host, int R, const float* lam, const float* A,
                   const float* Bf, const float* C, float* loss, float* grad_lam, float* grad_A,
                   float* grad_B, float* grad_C);

/* ALS update of one factor (Eq. 15): out = G^-1 M with G = (P P^T) o (Q Q^T) (FP64 Cholesky),
 * then lam[r] = ||out[r]|| and out[r] /= lam[r] (Alg. 2).  M: [K][n] rows = sketched
 * T(I, p_r, q_r) (contract_ivw); P: [K][np], Q: [K][nq]; out: [K][n]; lam: [K].  A singular G
 * is reported by tsk_ctx_status() as TSK_ENONFINITE.  Limits: K <= 64. */
int cp_als_solve(tsk_ctx* ctx, const float* M, const float* P, const float* Q, int K, int64_t n,
                 int64_t np, int64_t nq, float* out, float* lam);

/* Alg. 1 exactly as printed: three independent hashes and B asymmetric sketches (Eq. 1) of a
 * symmetric n x n x n tensor.  S: [B][b] TSK_C64, real parts used (sketch_tensor with M = 3,
 * dims {n, n, n}); h, g: [B][3][n].  For r = 0..k-1 and every tau < L:
 *   T power updates  v^(m)_i = xi_1(i) [F^-1(F s_T o conj F s_2,u o conj F s_3,u)]_{h_1(i)},
 *                    u <- median_m Re v^(m) / ||.||;
 *   selection        lambda^(m)_tau = sum_i u_i v^(m)_i(u) (= T^(m)(u,u,u), Prop. 1),
 *                    lambda_tau = median_m, tau* = first argmax;
 *   deflation        every sketch loses lambda^ s_1,u^ * s_2,u^ * s_3,u^ (Eq. 4), applied to
 *                    the half spectra that all later contractions use.
 * Outputs as robust_power_method: lambda [k] double, Vout [k][n], tau_star [k] (may be NULL),
 * lam_all optional [k][L], U_iters optional [k][T][L][n].  A zero/non-finite norm is reported by
 * tsk_ctx_status() as TSK_ENONFINITE.  Limits: log2b in [9, 15], B <= 64, n <= 8192, T >= 1. */
int robust_power_method_asym(tsk_ctx* ctx, const float* S, const int32_t* h, const uint8_t* g,
                             int B, int log2b, int64_t n, int k, int L, int T, const float* U0,
                             double* lambda, float* Vout, int32_t* tau_star, float* lam_all,
                             float* U_iters);

/* ---------------------------------------------------------------- spectral LDA (App. D, Alg. 3) */

/* Corpora are CSR word counts on the device: indptr int64 [D+1] (indptr[0] = 0, nondecreasing),
 * idx int32 [nnz] word ids in [0, V), cnt int32 [nnz] counts >= 1, nnz = indptr[D]; document d
 * has length m_d = sum of its counts.  The empirical moments average per-document unbiased
 * estimates over DISTINCT token positions (App. D):
 *   M1^ = mean over documents with m_d >= 1 of n_d / m_d                        (Eq. moment1)
 *   E2^ = mean over m_d >= 2 of (n_d n_d^T - diag n_d) / (m_d (m_d - 1))
 *   E3^ = mean over m_d >= 3 of N_d, the ordered distinct-position triple counts
 *         (n_i n_j n_k off the diagonals, n_i (n_i - 1) n_k on one, n_i (n_i-1)(n_i-2) on all)
 *         / (m_d (m_d - 1)(m_d - 2))
 *   M2^ = E2^ - alpha0/(alpha0+1) M1^ M1^T                                       (Eq. moment2)
 *   M3^ = E3^ - alpha0/(alpha0+2) (E2^ (x) M1^ + the two other placements)
 *         + 2 alpha0^2/((alpha0+1)(alpha0+2)) M1^ (x) M1^ (x) M1^                (Eq. moment3)
 * Word ids outside [0, V) and counts < 1 are skipped and reported by tsk_ctx_status() as
 * TSK_EINVAL. */

/* Y = M2^ X without forming M2^.  X, Y: [V][c] float row-major.  Limits: 1 <= c <= 256. */
int lda_m2_apply(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx, const int32_t* cnt,
                 int64_t D, int64_t V, double alpha0, const float* X, int c, float* Y);

/* Whitening (Alg. 3, line 3): the k leading eigenpairs (U, sigma) of M2^ by randomized
 * subspace iteration from the start block Omega ([V][c] float, c = k + oversampling; random
 * numbers are the caller's), power_iters extra applications of M2^, Cholesky-QR
 * orthonormalisation, and a Rayleigh-Ritz step solved by FP64 Jacobi; then
 * W[i][j] = U[i][j] / sqrt(sigma_j), so that W^T M2^ W = I_k.
 * Outputs: W [V][k] float, sigma [k] double (descending), M1_out optional [V] float (M1^).
 * Fewer than k positive Ritz values is reported by tsk_ctx_status() as TSK_EINVAL, a
 * Cholesky breakdown as TSK_ENONFINITE.  Limits: 1 <= k <= c <= min(V, 128), power_iters <= 64. */
int lda_whiten(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx, const int32_t* cnt,
               int64_t D, int64_t V, int k, double alpha0, const float* Omega, int c,
               int power_iters, float* W, double* sigma, float* M1_out);

/* The whitened third moment M3^(W, W, W) (k x k x k, dense, symmetric, float) of Alg. 3,
 * line 4, with each document entering through p_d = W^T n_d (Eq. td):
 *   N_d(W,W,W) = p^(x)3 - sum_i n_i (w_i w_i p + w_i p w_i + p w_i w_i) + 2 sum_i n_i w_i^(x)3,
 * w_i = row i of W, and E2^(W, W) (x) q with q = W^T M1^ for the alpha0 terms (Eq. applda_exxm).
 * W: [V][k] float.  Accumulates in FP32 over at most ~4096 documents, then in FP64.
 * Limits: 1 <= k <= 256. */
int lda_whitened_m3(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx, const int32_t* cnt,
                    int64_t D, int64_t V, const float* W, int k, double alpha0, float* M3);

/* B colliding sketches of M3^(W, W, W) (Alg. 3, line 4): lda_whitened_m3 into M3 (caller's
 * [k][k][k] float, also an output), then sketch_tensor with M = 1 into S ([B][b] TSK_C64).
 * h, g: [B][k] hash tables (cs_hashes with M = 1, dims = {k}).  Limits: k <= 256, log2b <= 14. */
int lda_sketch_m3(tsk_ctx* ctx, const int64_t* indptr, const int32_t* idx, const int32_t* cnt,
                  int64_t D, int64_t V, const float* W, int k, double alpha0, const int32_t* h,
                  const uint8_t* g, int B, int log2b, float* M3, float* S);

/* Recovery (Alg. 3, line 6): alpha_hat[i] = 4 alpha0 (alpha0+1) / ((alpha0+2)^2 lambda_i^2) and
 * mu_hat[i] = (alpha0+2)/2 lambda_i (W^+)^T v_i, with W^+ = (W^T W)^-1 W^T (FP64 Cholesky).
 * W: [V][k] float; lambda: [k] double; Vv: [k][k] float, row i = v_i (robust_power_method's
 * Vout); alpha_hat: [k] double; mu_hat: [k][V] float, row i = topic i.  Limits: k <= 128. */
int lda_recover(tsk_ctx* ctx, const float* W, int64_t V, int k, double alpha0,
                const double* lambda, const float* Vv, double* alpha_hat, float* mu_hat);

/* ---------------------------------------------------------------- Alg. 1 */

/* Fast robust tensor power method (Alg. 1) on B colliding sketches of a symmetric tensor.
 * S: [B][b] TSK_C64 time-domain sketches (read only).  U0: [k][L][n] float initial vectors of
 * every deflation round (normalised on the device before use).  For r = 0..k-1:
 *   T power updates u <- median_m T^(m)(I,u,u) / ||.|| for all L vectors;
 *   lambda_tau = median_m T^(m)(u,u,u); tau* = first argmax; (lambda^, u^) = (lambda_tau*, u_tau*);
 *   deflation: every sketch loses lambda^ * s~_{u^ (x) u^ (x) u^}.
 * Outputs: lambda [k] double, Vout [k][n] float, tau_star [k] int32 (may be NULL),
 * S_deflated: optional [B][b] TSK_C64 receiving the sketches after the k-th deflation,
 * lam_all: optional [k][L] float, lambda_tau of every initial vector of every round,
 * U_iters: optional [k][T][L][n] float, every iterate u_1..u_T of every round (diagnostics;
 *   lets a caller re-check each power update and selection independently).
 * A zero/non-finite norm in an update is reported by tsk_ctx_status() as TSK_ENONFINITE.
 * Sketch lengths above 2^14 (log2b 15, 16) are split by frequency class f mod P over
 * P = b / 2^14 blocks per (vector, sketch): block c scatters each nonzero of the count sketch
 * with the twiddle w_b^(c p) into a length-b/P transform, and the read-off sums the P classes'
 * inverses with w_b^(-c t) (an exact rewriting of the length-b DFT).
 * Limits: log2b in [8, 16], 1 <= B <= 64, 1 <= n <= 8192, 1 <= L <= 4096, T >= 1, k >= 0. */
int robust_power_method(tsk_ctx* ctx, const float* S, const int32_t* h, const uint8_t* g,
                        int B, int log2b, int64_t n, int k, int L, int T, const float* U0,
                        double* lambda, float* Vout, int32_t* tau_star, float* S_deflated,
                        float* lam_all, float* U_iters);

/* Number of kernel launches robust_power_method makes for these sizes on ctx's device (one DFT
 * of the sketches, then per round G groups x (T power steps + 1 selection) + 1 deflation (+1 to
 * assemble the time-domain update when the frequencies are split over several blocks per
 * contraction, which depends on n and b), where G = min(L, 8) is the number of helper-stream
 * groups the L chains are split into).  -1 on bad sizes. */
int64_t robust_power_method_launches(tsk_ctx* ctx, int B, int log2b, int64_t n, int k, int L,
                                     int T);

/* ---------------------------------------------------------------- order-p symmetric sketches */

/* The colliding sketch of Sec. 3.3 for symmetric tensors of order p = 3..6 (the paper states
 * the extension to higher order without details; the readings here are this library's).
 * Signs: sigma uniform on the m-th roots of unity, m = 4 for p = 3 and 8 for p = 4..6 (Sec. 3.3:
 * E[sigma^k] = 0 unless m | k, so with m > p no two multisets of p indices alias).
 * Hash (Prop. 2 with q = 2): h (2p)-wise independent, the Carter-Wegman polynomial of degree
 * 2p - 1 over GF(2^61 - 1) with cs_hashes' coefficient stream; g from the degree-11 polynomial
 * reduced mod m.  At p = 3 the hashes equal cs_hashes(M = 1).
 * h: [B][n] int32 in [0, b); g: [B][n] uint8 in [0, m).  TSK_EUNSUPPORTED for p outside 3..6. */
int cs_hashes_p(tsk_ctx* ctx, uint64_t seed, int B, int log2b, int p, int64_t n, int32_t* h,
                uint8_t* g);

/* Order-p colliding sketch (Eq. 7 with p indices) of a dense FP32 tensor T (row-major, n^p
 * entries): S[m][t] = sum over ordered p-tuples with (h(i_1)+...+h(i_p)) mod b = t of
 * T_{i_1..i_p} sigma(i_1)...sigma(i_p).  symmetric = 0: every entry is read; symmetric = 1: T is
 * taken as symmetric and only i_1 <= ... <= i_p is read, each entry weighted by its number of
 * orderings p!/prod(run lengths)! (n^p/p! reads; Sec. 3.3).  S: [B][b] TSK_C64, overwritten.
 * Limits: p in 3..6, log2b <= 14, B <= 64, n <= 8192. */
int sketch_tensor_p(tsk_ctx* ctx, const float* T, int p, int64_t n, const int32_t* h,
                    const uint8_t* g, int B, int log2b, int symmetric, float* S);

/* Sketched T(I,u,...,u) and T(u,...,u) for order p.  The colliding sketch counts each multiset
 * of indices once per ordering, so T(u,...,u) is estimated by pairing S with the sketch of the
 * complete homogeneous polynomial h_p = sum over partitions lambda of p of p_lambda / z_lambda,
 * the power sum p_k being the count sketch s_k[(k h(i)) mod b] += sigma(i)^k u_i^k:
 *   T^(u,...,u) = Re < S, sum_lambda (1/z_lambda) s_{lambda_1} * ... * s_{lambda_l} >,
 * and T^(I,u,...,u) is its gradient divided by p (at p = 3: App. B, Eq. 13 and Eq. 14).
 * FS = DFT of S, both [B][b] TSK_C64; U: [L][n].  Outputs (each may be NULL, not all):
 * Vall [L][B][n] per-sketch T^(m)(I,u,...,u); Vmed [L][n] their median over the sketches;
 * lam_all [L][B] per-sketch T^(m)(u,...,u); lam_med [L] their median.
 * Limits: p in 3..6, log2b in [8, 12], B <= 64, n <= 8192, L <= 65535. */
int contract_p(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h, const uint8_t* g,
               int B, int log2b, int p, const float* U, int L, int64_t n, float* Vmed, float* Vall,
               float* lam_med, float* lam_all);

/* Alg. 1 for order p: as robust_power_method, with the power update
 * u <- median_m T^(m)(I,u,...,u) / ||.||, the selection lambda_tau = median_m T^(m)(u,...,u),
 * tau* = first argmax, and the deflation S <- S - lambda^ s_1^{*p} (the sketch of u^{(x)p} is the
 * p-fold circular convolution of the count sketch s_1 of u).  Arguments and outputs as
 * robust_power_method's; limits as contract_p's, L <= 4096, T >= 1. */
int robust_power_method_p(tsk_ctx* ctx, const float* S, const int32_t* h, const uint8_t* g,
                          int B, int log2b, int p, int64_t n, int k, int L, int T, const float* U0,
                          double* lambda, float* Vout, int32_t* tau_star, float* S_deflated,
                          float* lam_all, float* U_iters);

/* Kernel launches of robust_power_method_p: one DFT of the sketches, then per round T power
 * steps and the selection (one launch each: the contraction, whose last-arriving block per vector
 * takes the medians) and the deflation.  -1 on bad sizes. */
int64_t robust_power_method_p_launches(tsk_ctx* ctx, int p, int k, int T);

/* ---------------------------------------------------------------- many independent problems */

/* One decomposition of a batch (all pointers device memory; see robust_power_method). */
typedef struct tsk_problem {
  const float* S;      /* [B][b] TSK_C64 time-domain colliding sketches (read only) */
  const int32_t* h;    /* [B][n] */
  const uint8_t* g;    /* [B][n] */
  const float* U0;     /* [k][L][n] initial vectors (NULL allowed when k = 0) */
  int64_t n;           /* dimension, 1..8192 */
  int k;               /* deflation rounds, >= 0 */
  int log2b;           /* sketch length 2^log2b, 10..14 */
  double* lambda;      /* out [k] */
  float* V;            /* out [k][n] */
  int32_t* tau;        /* out [k] or NULL */
  float* lam_all;      /* out [k][L] or NULL: lambda_tau of every round */
  float* U_iters;      /* out [k][T][L][n] or NULL: every iterate */
} tsk_problem;

typedef struct tsk_batch tsk_batch;

/* Plan Alg. 1 for P independent problems sharing B, L and T (the batch pattern of many
 * decompositions of uneven size; the paper runs one decomposition at a time).  Problems are
 * grouped by sketch length; each group's power steps are single launches over all its active
 * problems, groups run on helper streams of the context.  The plan allocates its own workspace
 * (device memory, freed by tsk_batch_destroy) and copies the problem descriptors to the device;
 * autotune = 1 times each compiled block size (FFT elements per thread) of every group on its
 * first power step and keeps the fastest.  The problem arrays must stay valid until the plan
 * is destroyed. */
int tsk_batch_create(tsk_ctx* ctx, const tsk_problem* problems, int P, int B, int L, int T,
                     int autotune, tsk_batch** out);
/* Enqueue the whole batch on the context's stream (sketch copies, DFTs, all rounds of every
 * problem).  Allocates nothing and synchronises nothing, so it can be captured into one CUDA
 * graph and replayed; each run starts from the problems' S and U0 again. */
int tsk_batch_run(tsk_ctx* ctx, tsk_batch* batch);
int tsk_batch_destroy(tsk_batch* batch);   /* TSK_EINVAL for NULL */
/* Block size chosen for the group of sketch length 2^log2b (0 if the plan has no such group,
 * TSK_EINVAL for a NULL plan). */
int tsk_batch_block_size(const tsk_batch* batch, int log2b);
/* create (without autotuning) + run + synchronise + destroy. */
int robust_power_method_batched(tsk_ctx* ctx, const tsk_problem* problems, int P, int B, int L,
                                int T);

#ifdef __cplusplus
}
#endif

#endif /* TSK_H_ */
