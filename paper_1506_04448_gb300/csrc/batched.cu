// Plans for many independent decompositions (Alg. 1): grouping, workspace, block-size autotuning
// and the launch sequence (see batched.cuh).
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "batched.cuh"

namespace tsk {

int launch_fft_batched(int log2b, const float2* in, float2* out, int B, int inverse, cudaStream_t st);

namespace {

// Block sizes compiled for each sketch length (first = default: 16 elements per thread).
void block_sizes(int log2b, int* sizes, int* count) {
  *count = 0;
  switch (log2b) {
    case 10: sizes[0] = 64; sizes[1] = 32; *count = 2; break;
    case 11: sizes[0] = 128; sizes[1] = 64; *count = 2; break;
    case 12: sizes[0] = 256; sizes[1] = 128; *count = 2; break;
    case 13: sizes[0] = 512; sizes[1] = 256; *count = 2; break;
    case 14: sizes[0] = 1024; *count = 1; break;
    default: break;
  }
}

int launch(int log2b, int nt, int kind, const BatchProblem* probs, int B, int L, int T, int t, int r,
           int nprob, int* status, cudaStream_t st) {
  int rc = batch_launch_lo(log2b, nt, kind, probs, B, L, T, t, r, nprob, status, st);
  if (rc == TSK_EUNSUPPORTED) rc = batch_launch_hi(log2b, nt, kind, probs, B, L, T, t, r, nprob, status, st);
  return rc;
}

}  // namespace

struct BatchGroup {
  int log2b = 0;
  int nt = 0;
  std::vector<int> order;          // problem indices, decreasing k
  std::vector<int> ks;             // k in that order
  std::vector<const float2*> src;  // input sketches in that order
  BatchProblem* d_probs = nullptr;
  float2* S_ws = nullptr;          // [nprob][B][b]
  float2* FS_ws = nullptr;
  unsigned* counters = nullptr;    // [nprob][L]
  int tuned_times = 0;
};

}  // namespace tsk

struct tsk_batch {
  int B, L, T, P;
  std::vector<tsk::BatchGroup> groups;
  void* mem;
};

using namespace tsk;

static int check_problem(const tsk_problem& p) {
  if (!p.S || !p.h || !p.g || p.k < 0 || p.n < 1) return TSK_EINVAL;
  if (p.k > 0 && (!p.U0 || !p.lambda || !p.V)) return TSK_EINVAL;   // k = 0: nothing is read or written
  if (p.log2b < 1 || p.log2b > 24) return TSK_EINVAL;
  if (p.log2b < 10 || p.log2b > 14 || p.n > 8192) return TSK_EUNSUPPORTED;
  return TSK_OK;
}

extern "C" int tsk_batch_destroy(tsk_batch* batch) {
  if (!batch) return TSK_EINVAL;
  if (batch->mem) cudaFree(batch->mem);
  delete batch;
  return TSK_OK;
}

extern "C" int tsk_batch_create(tsk_ctx* ctx, const tsk_problem* problems, int P, int B, int L, int T,
                                int autotune, tsk_batch** out) {
  if (!ctx || !problems || !out || P < 1 || B < 1 || L < 1) return TSK_EINVAL;
  if (T < 1 || B > kMaxB || L > 65535 || P > 65535) return TSK_EUNSUPPORTED;
  *out = nullptr;
  for (int i = 0; i < P; ++i) {
    const int rc = check_problem(problems[i]);
    if (rc != TSK_OK) return rc;
  }
  tsk_batch* bt = new tsk_batch{B, L, T, P, {}, nullptr};
  for (int lb = 10; lb <= 14; ++lb) {
    BatchGroup g;
    g.log2b = lb;
    for (int i = 0; i < P; ++i)
      if (problems[i].log2b == lb && problems[i].k > 0) g.order.push_back(i);
    if (g.order.empty()) continue;
    std::stable_sort(g.order.begin(), g.order.end(),
                     [&](int a, int c) { return problems[a].k > problems[c].k; });
    for (int i : g.order) {
      g.ks.push_back(problems[i].k);
      g.src.push_back(reinterpret_cast<const float2*>(problems[i].S));
    }
    int sizes[4], cnt = 0;
    block_sizes(lb, sizes, &cnt);
    g.nt = sizes[0];
    bt->groups.push_back(g);
  }
  if ((int)bt->groups.size() > kCtxAuxStreams) {
    delete bt;
    return TSK_EUNSUPPORTED;
  }
  // workspace: descriptors, sketch copies and per-problem scratch in one allocation
  size_t bytes = 0;
  for (auto& g : bt->groups) {
    const size_t b = (size_t)1 << g.log2b, np = g.order.size();
    bytes += ws_round(np * sizeof(BatchProblem)) + 2 * ws_round(np * B * b * sizeof(float2)) +
             ws_round(np * L * sizeof(unsigned));
    for (int i : g.order) {
      const tsk_problem& p = problems[i];
      bytes += ws_round((size_t)L * B * p.n * 4) + ws_round((size_t)L * B * 4) +
               ws_round(2 * (size_t)L * p.n * 4) + (p.lam_all ? 0 : ws_round((size_t)p.k * L * 4)) +
               ws_round((size_t)p.k * L * sizeof(double));
    }
  }
  cudaError_t e = cudaMalloc(&bt->mem, bytes ? bytes : 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete bt;
    return TSK_ENOMEM;
  }
  WsCarve wc{static_cast<char*>(bt->mem), 0};
  int rc = TSK_OK;
  for (auto& g : bt->groups) {
    const size_t b = (size_t)1 << g.log2b, np = g.order.size();
    g.d_probs = wc.take<BatchProblem>(np);
    g.S_ws = wc.take<float2>(np * B * b);
    g.FS_ws = wc.take<float2>(np * B * b);
    g.counters = wc.take<unsigned>(np * L);
    std::vector<BatchProblem> host(np);
    for (size_t q = 0; q < np; ++q) {
      const tsk_problem& p = problems[g.order[q]];
      BatchProblem& d = host[q];
      d.FS = g.FS_ws + q * B * b;
      d.S = g.S_ws + q * B * b;
      d.h = p.h;
      d.g = p.g;
      d.U0 = p.U0;
      d.Vall = wc.take<float>((size_t)L * B * p.n);
      d.lam_all = wc.take<float>((size_t)L * B);
      d.Ubuf = wc.take<float>(2 * (size_t)L * p.n);
      d.lam_med = p.lam_all ? p.lam_all : wc.take<float>((size_t)p.k * L);
      d.lam_med64 = wc.take<double>((size_t)p.k * L);
      d.counters = g.counters + q * L;
      d.lambda = p.lambda;
      d.V = p.V;
      d.tau = p.tau;
      d.U_iters = p.U_iters;
      d.n = (int)p.n;
      d.k = p.k;
    }
    if ((e = cudaMemcpy(g.d_probs, host.data(), np * sizeof(BatchProblem), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(g.counters, 0, np * L * sizeof(unsigned))) != cudaSuccess) {
      rc = tsk_from_cuda(e);
      break;
    }
  }
  if (rc == TSK_OK && autotune) {
    // time each compiled block size on the group's first power step (its result is discarded:
    // a run starts again from U0 and from fresh copies of the sketches)
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TSK_ECUDA;
    for (auto& g : bt->groups) {
      if (rc != TSK_OK) break;
      const size_t b = (size_t)1 << g.log2b, np = g.order.size();
      for (size_t q = 0; q < np && rc == TSK_OK; ++q)
        if (cudaMemcpyAsync(g.S_ws + q * B * b, g.src[q], B * b * sizeof(float2), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
          rc = TSK_ECUDA;
      if (rc == TSK_OK) rc = launch_fft_batched(g.log2b, g.S_ws, g.FS_ws, (int)(np * B), 0, st);
      int sizes[4], cnt = 0;
      block_sizes(g.log2b, sizes, &cnt);
      float best_ms = 1e30f;
      for (int c = 0; c < cnt && rc == TSK_OK; ++c) {
        float ms = 0.f;
        for (int rep = 0; rep < 3 && rc == TSK_OK; ++rep) {
          cudaEventRecord(e0, st);
          rc = launch(g.log2b, sizes[c], BATCH_STEP, g.d_probs, B, L, T, 0, 0, (int)np, ctx->status, st);
          cudaEventRecord(e1, st);
          if (rc == TSK_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;      // the first launch pays for module loading
          }
        }
        if (rc == TSK_OK && ms < best_ms) {
          best_ms = ms;
          g.nt = sizes[c];
        }
      }
      g.tuned_times = cnt;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  if (rc != TSK_OK) {
    tsk_batch_destroy(bt);
    return rc;
  }
  *out = bt;
  return TSK_OK;
}

extern "C" int tsk_batch_run(tsk_ctx* ctx, tsk_batch* bt) {
  if (!ctx || !bt) return TSK_EINVAL;
  const int B = bt->B, L = bt->L, T = bt->T;
  int rc = tsk_ctx_aux_streams(ctx, (int)bt->groups.size());
  if (rc != TSK_OK) return rc;
  cudaStream_t st = ctx->stream;
  TSK_CUDA(cudaEventRecord(ctx->ev_fork, st));
  for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
    BatchGroup& g = bt->groups[gi];
    cudaStream_t gs = ctx->aux[gi];
    const size_t b = (size_t)1 << g.log2b, np = g.order.size();
    TSK_CUDA(cudaStreamWaitEvent(gs, ctx->ev_fork, 0));
    for (size_t q = 0; q < np; ++q)
      TSK_CUDA(cudaMemcpyAsync(g.S_ws + q * B * b, g.src[q], B * b * sizeof(float2), cudaMemcpyDeviceToDevice, gs));
    if ((rc = launch_fft_batched(g.log2b, g.S_ws, g.FS_ws, (int)(np * B), 0, gs)) != TSK_OK) return rc;
    TSK_CUDA(cudaMemsetAsync(g.counters, 0, np * L * sizeof(unsigned), gs));
    const int max_k = g.ks.empty() ? 0 : g.ks[0];
    for (int r = 0; r < max_k; ++r) {
      int nact = 0;
      while (nact < (int)np && g.ks[nact] > r) ++nact;
      for (int t = 0; t < T; ++t)
        if ((rc = launch(g.log2b, g.nt, BATCH_STEP, g.d_probs, B, L, T, t, r, nact, ctx->status, gs)) != TSK_OK) return rc;
      if ((rc = launch(g.log2b, g.nt, BATCH_SELECT, g.d_probs, B, L, T, T, r, nact, ctx->status, gs)) != TSK_OK) return rc;
      if ((rc = launch(g.log2b, g.nt, BATCH_DEFLATE, g.d_probs, B, L, T, T, r, nact, ctx->status, gs)) != TSK_OK) return rc;
    }
    TSK_CUDA(cudaEventRecord(ctx->ev_join[gi], gs));
    TSK_CUDA(cudaStreamWaitEvent(st, ctx->ev_join[gi], 0));
  }
  return TSK_OK;
}

extern "C" int tsk_batch_block_size(const tsk_batch* bt, int log2b) {
  if (!bt) return TSK_EINVAL;
  for (const auto& g : bt->groups)
    if (g.log2b == log2b) return g.nt;
  return 0;
}

extern "C" int robust_power_method_batched(tsk_ctx* ctx, const tsk_problem* problems, int P, int B,
                                           int L, int T) {
  tsk_batch* bt = nullptr;
  int rc = tsk_batch_create(ctx, problems, P, B, L, T, 0, &bt);
  if (rc != TSK_OK) return rc;
  rc = tsk_batch_run(ctx, bt);
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  tsk_batch_destroy(bt);
  if (rc != TSK_OK) return rc;
  return tsk_from_cuda(e);
}
