// noalloc.cu -- bridges_find_noalloc: the whole bridge path with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is owned by someone
// else (a framework's caching allocator, a real-time loop that must not block on the driver,
// an embedded host that maps a fixed memory budget at start-up).  For them this entry point
// keeps every intermediate buffer (union-finds, certificates, Euler tour, ranges, sort keys) in
// one file-scope device array of fixed size, kNoAllocScratchBytes.  The caller still passes
// the edge list and the output buffer.  The paper has no counterpart: it is an interface for
// callers, not part of the method.
#include <algorithm>
#include <mutex>

#include "../../include/bridges.h"
#include "internal.h"

namespace {

using namespace bridges;

// 8 MiB.  A call needs about 1.07 MB plus (132 + 30 M) bytes per vertex, so the largest graph
// that fits has 45,135 vertices at M = 1 (the automatic choice), 38,095 at M = 2, 29,040 at
// M = 4 and 19,679 at M = 8; the edge count does not enter.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr size_t kMiscBytes = 1024;  // status word at 0, the spare output slot at kSpareOut
constexpr size_t kSpareOut = 512;    // output target of a call that writes no pairs (V <= 1)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceSetup {
  bool ready = false;
  void* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  size_t smem_optin = 0;
  int64_t launches = 0;  // kernels launched on this device (calls on one device are serialised)
};

std::mutex g_setup_mu;
DeviceSetup g_setup[64];

// Once per device, with that device current: the device address of the scratch array.  In
// host code the array's name only stands for a host-side shadow, so the address must come from
// cudaGetSymbolAddress.
int64_t setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return BRIDGES_ECUDA;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return BRIDGES_ECUDA;
    }
    s.smem_optin = (size_t)optin;
    s.scratch = ptr;
    s.ready = true;
  }
  *out = &s;
  return BRIDGES_OK;
}

}  // namespace

extern "C" int64_t bridges_find_noalloc(struct CUstream_st* stream, const int32_t* u, const int32_t* v, int64_t E,
                                        int32_t V, int32_t M, int32_t* out, int64_t* out_count_device) {
  if (E < 0 || V < 0 || (E > 0 && (!u || !v)) || (V > 1 && !out)) return BRIDGES_EINVAL;
  if (V > (1 << 30)) return BRIDGES_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return BRIDGES_ECUDA;
  }
  DeviceSetup* S = nullptr;
  int64_t rc = setup_device(dev, &S);
  if (rc) return rc;
  const CertPlan p = make_plan(E, V, M, 0, 0, 0, -1, S->num_sms, S->smem_optin);
  const size_t cert = align_up(cert_bytes(p), 256);
  const size_t need = kMiscBytes + cert + final_bytes(p.V);
  if (need > kNoAllocScratchBytes) return BRIDGES_ENOMEM;  // graph too large for the fixed scratch

  char* base = static_cast<char*>(S->scratch);
  int32_t* status = reinterpret_cast<int32_t*>(base);
  CertBufs cb = carve_cert(base + kMiscBytes, p);
  cb.status = status;
  FinalBufs fb = carve_final(base + kMiscBytes + cert, p.V, status);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Launch L{s, &S->launches, S->num_sms, S->smem_optin};
  // a graph of at most one vertex has no pairs to write; its output pointer may be null, so the
  // stage gets a slot of the scratch array instead (a device address, never a host one)
  int32_t* spare_out = reinterpret_cast<int32_t*>(base + kSpareOut);

  // The array keeps whatever the previous call left: the status word is cleared here, and every
  // other buffer that must start at zero is initialised by the stages themselves.
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) {
    cudaGetLastError();
    return BRIDGES_ECUDA;
  }
  cert_init(L, p, cb);
  cert_leaves(L, p, cb, u, v, nullptr);
  cert_merge(L, p, cb);
  final_stage(L, fb, V, cb.f1u, cb.f1v, cb.cnt + 0, V, cb.f2u, cb.f2v, cb.cnt + 1, V, cb.P1, out ? out : spare_out);
  if (cudaGetLastError() != cudaSuccess) return BRIDGES_ECUDA;
  if (out_count_device) {
    if (cudaMemcpyAsync(out_count_device, fb.count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return BRIDGES_ECUDA;
    }
    return BRIDGES_OK;
  }
  int64_t count = 0;
  if (cudaMemcpyAsync(&count, fb.count, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return BRIDGES_ECUDA;
  }
  return count;
}
