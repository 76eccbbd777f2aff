// sw_jvp_static_scratch: the complex-step JVP with its interface-flux scratch
// in a fixed, file-scope device array instead of context-owned memory.
//
// Who needs it: callers that may not allocate device memory once they are
// running -- e.g. a host application whose memory manager has already claimed
// the device memory it allows and forbids other libraries from calling
// cudaMalloc, a plug-in host that gives libraries no allocation rights, or a
// time-critical loop that cannot afford the implicit device synchronisation
// cudaMalloc/cudaFree may cause.  This entry point allocates nothing: no
// cudaMalloc, cudaFree or allocating library routine.  The read-only grid
// tables it uses were built by sw_init beforehand.
//
// The scratch (kScratchDoubles doubles = 16 MiB) is a static __device__ array:
// every GPU that loads the library holds it until the process exits.  In host
// code the array's name is only a host-side stand-in, so the host learns its
// device address through cudaGetSymbolAddress, done once per device on the
// first call on that device, with that device current; that first call should
// therefore come before any stream capture.  The address is cached per device
// ordinal for the life of the process's primary context: after a
// cudaDeviceReset the module is loaded again and the cached address is stale,
// so this entry point must not be used across a reset.  A call runs on the
// device its context was built on: with another device current it returns
// SW_EINVAL before any launch.  All calls share the array and it keeps the last
// call's contents; every entry a call reads is written earlier in the same
// call, so nothing has to start at zero.  Calls that overlap on the GPU
// (different streams, threads or contexts at once) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "swepi_internal.h"

namespace {

constexpr long long kScratchDoubles = 2LL * 1024 * 1024;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_face_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on device `dev`, which must be the
// current device (set-up on first use).
int scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return SW_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_face_scratch);
    if (e != cudaSuccess || p == nullptr) return SW_ECUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SW_OK;
}

}  // namespace

extern "C" int sw_jvp_static_scratch(sw_ctx_t ctx, const double* q, const double* v, double eps, double* Jv,
                                     void* stream) {
  swepi::Ctx* c = reinterpret_cast<swepi::Ctx*>(ctx);
  if (!c || !q || !v || !Jv || Jv == q || Jv == v || !(eps > 0) || !std::isfinite(eps)) return SW_EINVAL;
  const long long need = c->nelem * 12LL * c->ns;
  if (need > kScratchDoubles) return SW_ESCRATCH;
  // the context's tables live on the device sw_init ran on: refuse to pair
  // them with another device's scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SW_ECUDA;
  if (dev != c->device) return SW_EINVAL;
  double* fb = nullptr;
  int rc = scratch_address(dev, &fb);
  if (rc) return rc;
  return swepi::launch_jvp_fb(*c, q, v, eps, Jv, fb, reinterpret_cast<cudaStream_t>(stream));
}
