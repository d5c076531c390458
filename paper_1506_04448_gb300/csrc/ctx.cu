// Context management: stream binding, scratch workspace and the device status word.
#include <stdlib.h>

#include "common.cuh"

namespace {

// Run the body with ctx->device current, restoring the caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

int tsk_ws_reserve(tsk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return TSK_OK;
  // the old buffer may still be read by work queued on the stream
  TSK_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t grow = bytes + bytes / 2;
  grow = (grow + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TSK_ENOMEM;
  }
  ctx->ws = p;
  ctx->ws_bytes = grow;
  return TSK_OK;
}

int tsk_ctx_aux_streams(tsk_ctx* ctx, int count) {
  if (count > kCtxAuxStreams) return TSK_EUNSUPPORTED;
  if (ctx->n_aux == 0) TSK_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  while (ctx->n_aux < count) {
    const int i = ctx->n_aux;
    TSK_CUDA(cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
    TSK_CUDA(cudaEventCreateWithFlags(&ctx->ev_join[i], cudaEventDisableTiming));
    ctx->n_aux = i + 1;
  }
  return TSK_OK;
}

extern "C" int tsk_ctx_create(int device, void* stream, tsk_ctx** out) {
  if (!out) return TSK_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return TSK_ECUDA;
  }
  DeviceGuard guard(device);
  if (!guard.ok) return TSK_ECUDA;
  tsk_ctx* c = static_cast<tsk_ctx*>(calloc(1, sizeof(tsk_ctx)));
  if (!c) return TSK_ENOMEM;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
    if (c->status) cudaFree(c->status);
    free(c);
    cudaGetLastError();
    return TSK_ECUDA;
  }
  *out = c;
  return TSK_OK;
}

extern "C" int tsk_ctx_destroy(tsk_ctx* ctx) {
  if (!ctx) return TSK_EINVAL;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < ctx->n_aux; ++i) {
    cudaStreamSynchronize(ctx->aux[i]);
    cudaStreamDestroy(ctx->aux[i]);
    cudaEventDestroy(ctx->ev_join[i]);
  }
  if (ctx->n_aux > 0) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_switch) cudaEventDestroy(ctx->ev_switch);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->status) cudaFree(ctx->status);
  free(ctx);
  return TSK_OK;
}

extern "C" int tsk_ctx_set_stream(tsk_ctx* ctx, void* stream) {
  if (!ctx) return TSK_EINVAL;
  cudaStream_t next = static_cast<cudaStream_t>(stream);
  if (next == ctx->stream) return TSK_OK;
  // The workspace and the status word serve every stream the context is bound to, so work
  // enqueued from now on waits for the work already queued on the previous stream (an event
  // recorded there).  Not while either stream is being captured into a graph: a capture cannot
  // wait on uncaptured work, and the capturing caller orders its streams itself.
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return TSK_ECUDA;
  cudaStreamCaptureStatus cap_next = cudaStreamCaptureStatusNone;
  cudaStreamCaptureStatus cap_prev = cudaStreamCaptureStatusNone;
  bool order = cudaStreamIsCapturing(next, &cap_next) == cudaSuccess &&
               cap_next == cudaStreamCaptureStatusNone;
  if (order)
    order = cudaStreamIsCapturing(ctx->stream, &cap_prev) == cudaSuccess &&
            cap_prev == cudaStreamCaptureStatusNone;
  cudaGetLastError();   // a refused query only means: do not order
  if (order) {
    if (!ctx->ev_switch)
      TSK_CUDA(cudaEventCreateWithFlags(&ctx->ev_switch, cudaEventDisableTiming));
    TSK_CUDA(cudaEventRecord(ctx->ev_switch, ctx->stream));
    TSK_CUDA(cudaStreamWaitEvent(next, ctx->ev_switch, 0));
  }
  ctx->stream = next;
  return TSK_OK;
}

extern "C" int tsk_ctx_status(tsk_ctx* ctx) {
  if (!ctx) return TSK_EINVAL;
  DeviceGuard guard(ctx->device);
  TSK_CUDA(cudaStreamSynchronize(ctx->stream));
  int st = 0;
  TSK_CUDA(cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) TSK_CUDA(cudaMemset(ctx->status, 0, sizeof(int)));
  return st;
}

extern "C" const char* tsk_strerror(int status) {
  switch (status) {
    case TSK_OK: return "ok";
    case TSK_EINVAL: return "invalid argument";
    case TSK_ENOMEM: return "out of device memory";
    case TSK_ECUDA: return "CUDA runtime error";
    case TSK_ETIMEOUT: return "device-side wait timed out";
    case TSK_ENONFINITE: return "zero or non-finite norm in a power update";
    case TSK_EUNSUPPORTED: return "size outside the implemented range";
    default: return "unknown status";
  }
}
