// Launchers and C entry points for the sketched contractions (contract_iuu, contract_uuu) and
// the fast robust tensor power method (Alg. 1).
#include <stdio.h>

#include "contract.cuh"

namespace tsk {

// Valid (log2 b, log2 P) pairs: one block per (vector, sketch) up to b = 2^14, or the
// frequencies split into P classes whose transforms have length b / P = 2^13 or 2^14.
constexpr bool split_ok(int logb, int logp) {
  return logp >= 0 && logb - logp >= 8 && logb - logp <= 14 && (logp == 0 || logb - logp >= 12);
}

template <int LOGB, int LOGP, int MODE>
static int launch_contract_t(const ContractArgs& a, cudaStream_t st) {
  constexpr int NT = threads_for_logb(LOGB - LOGP);
  constexpr size_t smem = contract_smem_bytes<LOGB - LOGP>();
  TSK_CUDA(tsk_smem_attr<contract_kernel<LOGB, MODE, LOGP>>(smem));
  dim3 grid(a.B << LOGP, a.L);
  contract_kernel<LOGB, MODE, LOGP><<<grid, NT, smem, st>>>(a);
  TSK_CHECK_LAUNCH();
  return TSK_OK;
}

template <int LOGB, int LOGP>
static int launch_contract_p(int mode, const ContractArgs& a, cudaStream_t st) {
  if constexpr (split_ok(LOGB, LOGP)) {
    return mode == MODE_IUU ? launch_contract_t<LOGB, LOGP, MODE_IUU>(a, st)
                            : launch_contract_t<LOGB, LOGP, MODE_UUU>(a, st);
  } else {
    return TSK_EUNSUPPORTED;
  }
}

template <int LOGB>
static int launch_contract_b(int logp, int mode, const ContractArgs& a, cudaStream_t st) {
  switch (logp) {
    case 0: return launch_contract_p<LOGB, 0>(mode, a, st);
    case 1: return launch_contract_p<LOGB, 1>(mode, a, st);
    case 2: return launch_contract_p<LOGB, 2>(mode, a, st);
    case 3: return launch_contract_p<LOGB, 3>(mode, a, st);
    default: return TSK_EUNSUPPORTED;
  }
}

int launch_contract(int log2b, int logp, int mode, const ContractArgs& a, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_contract_b<8>(logp, mode, a, st);
    case 9: return launch_contract_b<9>(logp, mode, a, st);
    case 10: return launch_contract_b<10>(logp, mode, a, st);
    case 11: return launch_contract_b<11>(logp, mode, a, st);
    case 12: return launch_contract_b<12>(logp, mode, a, st);
    case 13: return launch_contract_b<13>(logp, mode, a, st);
    case 14: return launch_contract_b<14>(logp, mode, a, st);
    case 15: return launch_contract_b<15>(logp, mode, a, st);
    case 16: return launch_contract_b<16>(logp, mode, a, st);
    default: return TSK_EUNSUPPORTED;
  }
}

template <int LOGB, int LOGP>
static int launch_deflate_t(const DeflateArgs& a, int B, cudaStream_t st) {
  if constexpr (split_ok(LOGB, LOGP)) {
    constexpr int NT = threads_for_logb(LOGB - LOGP);
    constexpr size_t smem = (size_t)padded_len(1 << (LOGB - LOGP)) * sizeof(float2);
    TSK_CUDA(tsk_smem_attr<deflate_kernel<LOGB, LOGP>>(smem));
    deflate_kernel<LOGB, LOGP><<<B << LOGP, NT, smem, st>>>(a);
    TSK_CHECK_LAUNCH();
    if constexpr (LOGP > 0) {
      deflate_combine_kernel<LOGB, LOGP><<<dim3(16, B), 256, 0, st>>>(a.S, a.G);
      TSK_CHECK_LAUNCH();
    }
    return TSK_OK;
  } else {
    return TSK_EUNSUPPORTED;
  }
}

template <int LOGB>
static int launch_deflate_b(int logp, const DeflateArgs& a, int B, cudaStream_t st) {
  switch (logp) {
    case 0: return launch_deflate_t<LOGB, 0>(a, B, st);
    case 1: return launch_deflate_t<LOGB, 1>(a, B, st);
    case 2: return launch_deflate_t<LOGB, 2>(a, B, st);
    case 3: return launch_deflate_t<LOGB, 3>(a, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

int launch_deflate(int log2b, int logp, const DeflateArgs& a, int B, cudaStream_t st) {
  switch (log2b) {
    case 8: return launch_deflate_b<8>(logp, a, B, st);
    case 9: return launch_deflate_b<9>(logp, a, B, st);
    case 10: return launch_deflate_b<10>(logp, a, B, st);
    case 11: return launch_deflate_b<11>(logp, a, B, st);
    case 12: return launch_deflate_b<12>(logp, a, B, st);
    case 13: return launch_deflate_b<13>(logp, a, B, st);
    case 14: return launch_deflate_b<14>(logp, a, B, st);
    case 15: return launch_deflate_b<15>(logp, a, B, st);
    case 16: return launch_deflate_b<16>(logp, a, B, st);
    default: return TSK_EUNSUPPORTED;
  }
}

template <int LOGB, int LOGP>
static int launch_fft_split_t(const float2* S, float2* FS, int B, cudaStream_t st, int cm) {
  if constexpr (LOGP > 0 && split_ok(LOGB, LOGP)) {
    constexpr int LOGM = LOGB - LOGP;
    constexpr size_t smem = (size_t)padded_len(1 << LOGM) * sizeof(float2);
    TSK_CUDA(tsk_smem_attr<fft_split_kernel<LOGB, LOGP>>(smem));
    fft_split_kernel<LOGB, LOGP><<<B << LOGP, threads_for_logb(LOGM), smem, st>>>(S, FS, cm);
    TSK_CHECK_LAUNCH();
    return TSK_OK;
  } else {
    return TSK_EUNSUPPORTED;
  }
}

int launch_fft_split(int log2b, int logp, const float2* S, float2* FS, int B, cudaStream_t st,
                     int cm) {
  switch (log2b * 4 + logp) {
    case 13 * 4 + 1: return launch_fft_split_t<13, 1>(S, FS, B, st, cm);
    case 14 * 4 + 1: return launch_fft_split_t<14, 1>(S, FS, B, st, cm);
    case 14 * 4 + 2: return launch_fft_split_t<14, 2>(S, FS, B, st, cm);
    case 15 * 4 + 1: return launch_fft_split_t<15, 1>(S, FS, B, st, cm);
    case 15 * 4 + 2: return launch_fft_split_t<15, 2>(S, FS, B, st, cm);
    case 15 * 4 + 3: return launch_fft_split_t<15, 3>(S, FS, B, st, cm);
    case 16 * 4 + 2: return launch_fft_split_t<16, 2>(S, FS, B, st, cm);
    case 16 * 4 + 3: return launch_fft_split_t<16, 3>(S, FS, B, st, cm);
    default: return TSK_EUNSUPPORTED;
  }
}

int launch_fft_batched(int log2b, const float2* in, float2* out, int B, int inverse, cudaStream_t st);

}  // namespace tsk

using namespace tsk;

// Alg. 1 (and contract_iuu / contract_uuu without per-sketch outputs) splits each (vector, sketch) contraction's frequencies over 2^logp blocks (see
// contract_one): smaller blocks fit more of them per SM and hide each other's barriers, but
// every block repeats the work that grows with n (scatter, read-off, the sum of the shares).
// The blocks' transform length M = b / 2^logp is kept at >= 8 n, >= 2^12 and <= 2^14, with at
// most 8 blocks; measured on n = 100, 400 and 1000 for b = 2^12 .. 2^16 this choice was the
// fastest or within 3 % of it (2^11-point blocks were 10 % slower at n = 100).
static int rpm_split_log(int log2b, int64_t n) {
  int logm = 12;
  while (logm < 14 && ((int64_t)1 << logm) < 8 * n) ++logm;
  if (logm >= log2b) return 0;
  int lp = log2b - logm;
  if (lp > 3) lp = 3;
  return lp;
}


static int check_contract_args(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                               const uint8_t* g, int B, int log2b, const float* U, int L, int64_t n) {
  if (!ctx || !FS || !S || !h || !g || !U) return TSK_EINVAL;
  if (B < 1 || L < 1 || n < 1) return TSK_EINVAL;
  if (log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 8 || log2b > 14 || B > kMaxB || n > 8192 || L > 65535) return TSK_EUNSUPPORTED;
  return TSK_OK;
}

extern "C" int contract_iuu(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                            const uint8_t* g, int B, int log2b, const float* U, int L, int64_t n,
                            float* Vmed, float* Vall) {
  int rc = check_contract_args(ctx, FS, S, h, g, B, log2b, U, L, n);
  if (rc != TSK_OK) return rc;
  if (!Vmed) return TSK_EINVAL;
  // per-sketch values requested: one block per (vector, sketch); otherwise the split of Alg. 1
  const int logp = Vall ? 0 : rpm_split_log(log2b, n);
  const int P = 1 << logp;
  const size_t vall_bytes = Vall ? 0 : ws_round((size_t)L * B * P * n * sizeof(float));
  const size_t need = vall_bytes + ws_round((size_t)L * B * P * sizeof(float)) +
                      ws_round((size_t)L * sizeof(unsigned));
  if ((rc = tsk_ws_reserve(ctx, need)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  ContractArgs a{};
  a.Vall = Vall ? Vall : wc.take<float>((size_t)L * B * P * n);
  a.lam_all = wc.take<float>((size_t)L * B * P);
  a.counters = wc.take<unsigned>(L);
  TSK_CUDA(cudaMemsetAsync(a.counters, 0, L * sizeof(unsigned), ctx->stream));
  a.FS = reinterpret_cast<const float2*>(FS);
  a.S = reinterpret_cast<const float2*>(S);
  a.h = h;
  a.g = g;
  a.U = U;
  a.n = (int)n;
  a.B = B;
  a.L = L;
  a.normalize_input = 0;
  a.Vmed = Vmed;
  a.Unext = nullptr;
  a.lam_med = nullptr;
  a.status = ctx->status;
  return launch_contract(log2b, logp, MODE_IUU, a, ctx->stream);
}

extern "C" int contract_uuu(tsk_ctx* ctx, const float* FS, const float* S, const int32_t* h,
                            const uint8_t* g, int B, int log2b, const float* U, int L, int64_t n,
                            float* lam_med, float* lam_all) {
  int rc = check_contract_args(ctx, FS, S, h, g, B, log2b, U, L, n);
  if (rc != TSK_OK) return rc;
  if (!lam_med) return TSK_EINVAL;
  const int logp = lam_all ? 0 : rpm_split_log(log2b, n);
  const int P = 1 << logp;
  const size_t need = (lam_all ? 0 : ws_round((size_t)L * B * P * sizeof(float))) +
                      ws_round((size_t)L * sizeof(unsigned));
  if ((rc = tsk_ws_reserve(ctx, need)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  ContractArgs a{};
  a.lam_all = lam_all ? lam_all : wc.take<float>((size_t)L * B * P);
  a.counters = wc.take<unsigned>(L);
  TSK_CUDA(cudaMemsetAsync(a.counters, 0, L * sizeof(unsigned), ctx->stream));
  a.FS = reinterpret_cast<const float2*>(FS);
  a.S = reinterpret_cast<const float2*>(S);
  a.h = h;
  a.g = g;
  a.U = U;
  a.n = (int)n;
  a.B = B;
  a.L = L;
  a.normalize_input = 0;
  a.Vall = nullptr;
  a.Vmed = nullptr;
  a.Unext = nullptr;
  a.lam_med = lam_med;
  a.status = ctx->status;
  return launch_contract(log2b, logp, MODE_UUU, a, ctx->stream);
}

// The L power-iteration chains are independent until the selection, so they are split into
// G = min(L, 8) groups, each enqueued on its own stream: while one group's step finishes its
// last wave of blocks and its last-arriving blocks take the medians, the other groups' steps
// fill the idle SMs (a single B x L grid per step would leave the SMs partly idle at the end of
// every step).  Eight groups measured at least as fast as fewer for every sketch length, and
// sixteen were 11 % slower for n = 400, b = 2^14, L = 50.
static long long rpm_groups(int L) {
  return L < kCtxAuxStreams ? L : kCtxAuxStreams;
}

extern "C" int64_t robust_power_method_launches(tsk_ctx* ctx, int B, int log2b, int64_t n, int k,
                                                int L, int T) {
  if (!ctx || k < 0 || B < 1 || L < 1 || T < 1 || log2b < 8 || log2b > 16) return -1;
  if (k == 0) return 0;
  const long long G = rpm_groups(L);
  const int split = rpm_split_log(log2b, n) > 0 ? 1 : 0;   // deflation adds a combine launch
  return 1 + (int64_t)k * (G * (T + 1) + 1 + split);
}

extern "C" int robust_power_method(tsk_ctx* ctx, const float* S, const int32_t* h,
                                   const uint8_t* g, int B, int log2b, int64_t n, int k, int L,
                                   int T, const float* U0, double* lambda, float* Vout,
                                   int32_t* tau_star, float* S_deflated, float* lam_all_out,
                                   float* U_iters) {
  if (!ctx || !S || !h || !g) return TSK_EINVAL;
  if (k < 0 || T < 0 || B < 1 || L < 1 || n < 1) return TSK_EINVAL;
  if (log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 8 || log2b > 16 || B > kMaxB || n > 8192 || L > 4096 || T < 1)
    return TSK_EUNSUPPORTED;
  const size_t b = (size_t)1 << log2b;
  if (k == 0) {
    if (S_deflated && S_deflated != S)
      TSK_CUDA(cudaMemcpyAsync(S_deflated, S, (size_t)B * b * sizeof(float2),
                               cudaMemcpyDeviceToDevice, ctx->stream));
    return TSK_OK;
  }
  if (!U0 || !lambda || !Vout) return TSK_EINVAL;
  // sketch lengths above 2^14 are split over P blocks per (vector, sketch): per-sketch values
  // and eigenvalues are kept as P shares, and deflation needs a [B][b] staging buffer
  const int logp = rpm_split_log(log2b, n);
  const int P = 1 << logp;
  const size_t need = 2 * ws_round(B * b * sizeof(float2)) + ws_round((size_t)L * B * P * n * 4) +
                      ws_round((size_t)L * B * P * 4) + ws_round(2 * (size_t)L * n * 4) +
                      ws_round((size_t)k * L * 4) + ws_round((size_t)k * L * sizeof(double)) +
                      ws_round((size_t)L * 4) +
                      (P > 1 ? ws_round(B * b * sizeof(float2)) : 0);
  int rc = tsk_ws_reserve(ctx, need);
  if (rc != TSK_OK) return rc;
  const long long G = rpm_groups(L);
  if ((rc = tsk_ctx_aux_streams(ctx, (int)G)) != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(ctx->ws), 0};
  float2* Sw = wc.take<float2>(B * b);
  float2* FSw = wc.take<float2>(B * b);
  float* Vall = wc.take<float>((size_t)L * B * P * n);
  float* lam_all = wc.take<float>((size_t)L * B * P);
  float* Ubuf = wc.take<float>(2 * (size_t)L * n);
  float* lam_med = lam_all_out ? lam_all_out : wc.take<float>((size_t)k * L);
  double* lam_med64 = wc.take<double>((size_t)k * L);   // selection and deflation in FP64
  unsigned* counters = wc.take<unsigned>(L);
  float2* Gdefl = P > 1 ? wc.take<float2>(B * b) : nullptr;
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaMemsetAsync(counters, 0, L * sizeof(unsigned), st));
  TSK_CUDA(cudaMemcpyAsync(Sw, S, B * b * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if (P == 1) {
    if ((rc = launch_fft_batched(log2b, Sw, FSw, B, 0, st)) != TSK_OK) return rc;
  } else {
    // the workspace spectra are kept class-major (each class's frequencies contiguous)
    if ((rc = launch_fft_split(log2b, logp, Sw, FSw, B, st, 1)) != TSK_OK) return rc;
  }

  ContractArgs a{};
  a.FS = FSw;
  a.S = Sw;
  a.h = h;
  a.g = g;
  a.n = (int)n;
  a.B = B;
  a.status = ctx->status;
  a.fs_class_major = P > 1;
  DeflateArgs d{};
  d.FS = FSw;
  d.S = Sw;
  d.h = h;
  d.g = g;
  d.n = (int)n;
  d.L = L;
  d.lambda_out = lambda;
  d.Vout = Vout;
  d.tau_out = tau_star;
  d.G = Gdefl;
  d.fs_class_major = P > 1;
  for (int r = 0; r < k; ++r) {
    TSK_CUDA(cudaEventRecord(ctx->ev_fork, st));
    for (int s = 0; s < G; ++s) {
      const int tau0 = (int)((long long)L * s / G);
      const int Ls = (int)((long long)L * (s + 1) / G) - tau0;
      cudaStream_t gs = ctx->aux[s];
      TSK_CUDA(cudaStreamWaitEvent(gs, ctx->ev_fork, 0));
      a.L = Ls;
      a.Vall = Vall + (size_t)tau0 * B * P * n;
      a.lam_all = lam_all + (size_t)tau0 * B * P;
      a.counters = counters + tau0;
      const float* cur = U0 + ((size_t)r * L + tau0) * n;
      for (int t = 0; t < T; ++t) {
        float* next = U_iters ? U_iters + (((size_t)r * T + t) * L + tau0) * n
                              : Ubuf + ((size_t)((t + 1) & 1) * L + tau0) * n;
        a.U = cur;
        a.normalize_input = (t == 0);
        a.Unext = next;
        a.Vmed = nullptr;
        a.lam_med = nullptr;
        a.lam_med64 = nullptr;
        if ((rc = launch_contract(log2b, logp, MODE_IUU, a, gs)) != TSK_OK) return rc;
        cur = next;
      }
      // selection: lambda_tau = median_m T^(m)(u_tau, u_tau, u_tau)
      a.U = cur;
      a.normalize_input = 0;
      a.Unext = nullptr;
      a.lam_med = lam_med + (size_t)r * L + tau0;
      a.lam_med64 = lam_med64 + (size_t)r * L + tau0;
      if ((rc = launch_contract(log2b, logp, MODE_UUU, a, gs)) != TSK_OK) return rc;
      TSK_CUDA(cudaEventRecord(ctx->ev_join[s], gs));
      TSK_CUDA(cudaStreamWaitEvent(st, ctx->ev_join[s], 0));
    }
    d.Ufinal = U_iters ? U_iters + ((size_t)r * T + (T - 1)) * L * n : Ubuf + (size_t)(T & 1) * L * n;
    d.lam_med = lam_med64 + (size_t)r * L;
    d.round = r;
    if ((rc = launch_deflate(log2b, logp, d, B, st)) != TSK_OK) return rc;
  }
  if (S_deflated)
    TSK_CUDA(cudaMemcpyAsync(S_deflated, Sw, B * b * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  return TSK_OK;
}
