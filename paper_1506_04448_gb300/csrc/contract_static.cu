// contract_iuu_static: the sketched T^(I,u,u) contraction for callers that cannot allocate.
//
// contract_iuu keeps its per-sketch values, per-sketch eigenvalue estimates and arrival
// counters in a context workspace that grows with cudaMalloc.  Some callers cannot allocate
// device memory at the point where they contract: runtimes whose device memory is owned by
// another allocator and may not be touched by a library, and latency-critical loops that
// forbid allocation after start-up.  This entry point
// runs the same kernel with that scratch in a fixed-size array compiled into the library
// (kStaticScratchBytes per device, held by every GPU that loads the library until the process
// exits) and takes the stream directly, so it creates no context either.
//
// The array's host-side name is only a stand-in for a device address, so the address is looked
// up once per device with cudaGetSymbolAddress, with that device current, the first time the
// entry point runs there.
// All calls share the array and it keeps the last call's contents: the arrival counters are
// cleared on the stream before every launch, and calls whose kernels overlap on the GPU race.
#include <mutex>

#include "contract.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_contract_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_contract_scratch on `device` (current), resolved once per device.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return TSK_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_contract_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TSK_ECUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return TSK_OK;
}

}  // namespace

extern "C" int contract_iuu_static(const float* FS, const float* S, const int32_t* h,
                                   const uint8_t* g, int B, int log2b, const float* U, int L,
                                   int64_t n, float* Vmed, void* stream) {
  if (!FS || !S || !h || !g || !U || !Vmed) return TSK_EINVAL;
  if (B < 1 || L < 1 || n < 1 || log2b < 1 || log2b > 24) return TSK_EINVAL;
  if (log2b < 8 || log2b > 14 || B > tsk::kMaxB || n > 8192 || L > 65535) return TSK_EUNSUPPORTED;
  const size_t vall = ws_round((size_t)L * B * n * sizeof(float));
  const size_t lam = ws_round((size_t)L * B * sizeof(float));
  const size_t cnt = ws_round((size_t)L * sizeof(unsigned));
  if (vall + lam + cnt > kStaticScratchBytes) return TSK_EUNSUPPORTED;   // beyond the static maximum
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return TSK_ECUDA;
  }
  void* base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc != TSK_OK) return rc;
  WsCarve wc{static_cast<char*>(base), 0};
  tsk::ContractArgs a{};
  a.Vall = wc.take<float>((size_t)L * B * n);
  a.lam_all = wc.take<float>((size_t)L * B);
  a.counters = wc.take<unsigned>(L);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TSK_CUDA(cudaMemsetAsync(a.counters, 0, L * sizeof(unsigned), st));
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
  a.status = nullptr;
  return tsk::launch_contract(log2b, 0, tsk::MODE_IUU, a, st);
}
