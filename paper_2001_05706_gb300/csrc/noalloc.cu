// lqcd_norm2_noalloc: the deterministic FP64 sum-of-squares reduction with
// its scratch in this file's static device arrays instead of memory the
// library or the caller allocates.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned
// entirely by another allocator (a framework's caching allocator working to
// a fixed budget), and latency-critical loops in which cudaMalloc/cudaFree
// would synchronise the device.  This entry point allocates nothing: the
// per-block partial sums and the completion counter live in the arrays
// below, which every GPU that loads the library holds until the process
// exits.
#include <cuda.h>

#include <mutex>

#include "internal.h"

namespace lqcd {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocMaxRhs = 64;
constexpr int kNoAllocMaxDevices = 64;

// partial sums: at most kNoAllocMaxBlocks per right-hand side (512 KiB)
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kNoAllocMaxRhs];
// completion counter of the last-block reduction
static __device__ __align__(256) unsigned int g_noalloc_counter[64];

struct DeviceScratch {
  bool ready = false;
  CUcontext ctx = nullptr;  // the context the addresses belong to
  double *partials = nullptr;
  unsigned int *counter = nullptr;
};

// the calling thread's current CUDA context (driver entry point looked up
// through the runtime, so the library needs no link against libcuda);
// nullptr if it cannot be found
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext *);
  static Fn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    cudaGetLastError();
    return reinterpret_cast<Fn>(f);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// x must be memory of the current device (device or managed memory)
lqcd_status check_device_pointer(const void *p, int dev, const char *what) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_ARG, "%s: not a CUDA pointer", what);
  }
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
    return set_error(LQCD_ERR_ARG, "%s: must be device or managed memory of the current device %d", what, dev);
  return LQCD_OK;
}
std::mutex g_noalloc_mu;
DeviceScratch g_noalloc_dev[kNoAllocMaxDevices];

__global__ void __launch_bounds__(kNoAllocThreads)
    norm2_noalloc_kernel(const double *__restrict__ x, long n, int nrhs, double *partials, unsigned int *counter,
                         double *result) {
  const int k = blockIdx.y;
  const double *v = x + (long)k * n;
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s = fma(v[i], v[i], s);
  double val[1] = {s};
  grid_reduce<1>(val, partials, counter, result, k, nrhs, 1);
}

}  // namespace
}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_norm2_noalloc(const double *x, long n, int nrhs, double *result, void *cuda_stream) {
  if (!x || !result) return set_error(LQCD_ERR_ARG, "x and result must be device pointers");
  if (n < 1 || n > (1L << 40)) return set_error(LQCD_ERR_ARG, "n = %ld: need 1 <= n <= 2^40", n);
  if (nrhs < 1 || nrhs > kNoAllocMaxRhs)
    return set_error(LQCD_ERR_ARG, "nrhs = %d: the static scratch holds at most %d right-hand sides", nrhs,
                     kNoAllocMaxRhs);
  int dev = 0;
  LQ_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(LQCD_ERR_ARG, "device %d out of range", dev);
  LQ_TRY(check_device_pointer(x, dev, "x"));
  LQ_TRY(check_device_pointer(result, dev, "result"));
  DeviceScratch sc;
  {
    // once per device and context, with that device current: the device
    // addresses of the static arrays (their names in host code are host-side
    // stand-ins); looked up again if the context changed (a cudaDeviceReset,
    // or a caller on another driver-API context of the same device)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    DeviceScratch &d = g_noalloc_dev[dev];
    const CUcontext ctx = current_context();
    if (!d.ready || d.ctx != ctx) {
      void *p = nullptr, *c = nullptr;
      LQ_CU(cudaGetSymbolAddress(&p, g_noalloc_partials));
      LQ_CU(cudaGetSymbolAddress(&c, g_noalloc_counter));
      d.partials = static_cast<double *>(p);
      d.counter = static_cast<unsigned int *>(c);
      d.ctx = ctx;
      d.ready = true;
    }
    sc = d;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  long blocks = (n + kNoAllocThreads * 8L - 1) / (kNoAllocThreads * 8L);
  if (blocks > kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
  // the counter must start at zero even if an earlier launch was abandoned
  LQ_CU(cudaMemsetAsync(sc.counter, 0, sizeof(unsigned int), st));
  norm2_noalloc_kernel<<<dim3((unsigned)blocks, (unsigned)nrhs), kNoAllocThreads, 0, st>>>(x, n, nrhs, sc.partials,
                                                                                           sc.counter, result);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}
