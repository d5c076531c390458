// Shared helpers for the tensor-sketch kernels: complex arithmetic on float2, the padded
// shared-memory layout used by the block FFTs, and the context structure behind tsk.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tsk.h"

#define TSK_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------ complex float helpers
TSK_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
TSK_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
TSK_HD float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
TSK_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
TSK_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * conj(b)
TSK_HD float2 cmulconj(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// Multiply by sqrt(-1)^e, e in {0,1,2,3}.
TSK_HD float2 cmul_ipow(float2 z, int e) {
  switch (e & 3) {
    case 0: return z;
    case 1: return make_float2(-z.y, z.x);
    case 2: return make_float2(-z.x, -z.y);
    default: return make_float2(z.y, -z.x);
  }
}
// Re(sqrt(-1)^e * z)
TSK_HD float re_ipow(float2 z, int e) {
  switch (e & 3) {
    case 0: return z.x;
    case 1: return -z.y;
    case 2: return -z.x;
    default: return z.y;
  }
}

// Padded shared-memory index: one float2 of padding after every 16 elements (128 bytes).  A
// warp's 8-byte accesses are served per half-warp; the first Stockham pass stores element r of
// butterfly j at 16 j + r, and the padding puts those 16 lanes in 16 different bank pairs.
TSK_HD int pad_idx(int i) { return i + (i >> 4); }
TSK_HD constexpr int padded_len(int n) { return n + (n >> 4); }

// ------------------------------------------------------------------ context
constexpr int kCtxAuxStreams = 8;

struct tsk_ctx {
  int device;
  cudaStream_t stream;
  void* ws;            // device workspace
  size_t ws_bytes;
  int* status;         // device status word (first error wins)
  int max_smem_optin;  // cudaDevAttrMaxSharedMemoryPerBlockOptin
  int num_sms;
  // helper streams for independent work inside one call, forked from and joined back into
  // `stream` with events (created on first use)
  int n_aux;
  cudaStream_t aux[kCtxAuxStreams];
  cudaEvent_t ev_fork;
  cudaEvent_t ev_join[kCtxAuxStreams];
  // orders a newly bound stream after the previous one (created on the first re-binding)
  cudaEvent_t ev_switch;
};

// Grow the context workspace to at least `bytes` (synchronising the stream when it grows).
int tsk_ws_reserve(tsk_ctx* ctx, size_t bytes);
// Make sure `count` helper streams and their events exist.
int tsk_ctx_aux_streams(tsk_ctx* ctx, int count);

// Raise KERNEL's dynamic shared-memory limit to `smem` once per device.  The attribute call is
// not a stream operation; doing it once (on the first, uncaptured launch) keeps later launch
// sequences capturable into CUDA graphs.  For kernels whose shared memory does not vary.
template <auto KERNEL>
inline cudaError_t tsk_smem_attr(size_t smem) {
  static unsigned long long done = 0;   // bit d set once device d is configured
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) __atomic_fetch_or(&done, bit, __ATOMIC_RELEASE);
  return e;
}

// Map a CUDA error to a tsk status.
inline int tsk_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TSK_OK;
  if (e == cudaErrorMemoryAllocation) return TSK_ENOMEM;
  return TSK_ECUDA;
}

#define TSK_CHECK_LAUNCH()                                    \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return tsk_from_cuda(e_);          \
  } while (0)

#define TSK_CUDA(...)                                         \
  do {                                                        \
    cudaError_t e_ = (__VA_ARGS__);                           \
    if (e_ != cudaSuccess) return tsk_from_cuda(e_);          \
  } while (0)

// Record a device-side error (first one wins).
__device__ __forceinline__ void tsk_set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Workspace carving helper: 256-byte aligned sub-buffers.
struct WsCarve {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};
inline size_t ws_round(size_t x) { return (x + 255) & ~size_t(255); }
