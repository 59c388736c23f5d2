// sfd_symeig_noalloc: the symmetric eigensolver of sfd_symeig with its scratch
// in a fixed device array instead of memory allocated per call.
//
// Why: some callers cannot let a library call cudaMalloc. A serving process
// whose caching allocator has already reserved the device's memory budget has
// nothing left for a private allocation, and a latency-critical loop cannot
// absorb the device-wide synchronisation that cudaMalloc / cudaFree may
// perform. This entry point allocates nothing: the caller passes the input and
// the outputs, and the scratch is `g_symeig_scratch`, a file-scope array.
//
// When the array takes device memory: with CUDA's lazy module loading (the
// default), the module that holds it is loaded into a context on the first
// call that needs its device address, so the first call on each device
// reserves the array (~2.1 MB) and the module's code there and may
// synchronise; from then on the device holds it until the context ends.
// Callers that must not see that make one warm-up call per device before they
// hand the memory budget to their allocator and before any stream capture.
#include <cuda.h>

#include <mutex>

#include "sfd_internal.cuh"

namespace sfd {
namespace {

constexpr int kNoAllocMaxN = 256;

// An upper bound of symeig_work_floats(256, 256), the eigensolver's scratch
// for n = nwant = 256 (reflectors, eigenvector blocks, Gram and factor, an
// n x (n|1) matrix when it does not fit in shared memory), ~2.1 MB; every
// call checks the bound.
constexpr size_t kNoAllocFloats = (size_t)kNoAllocMaxN * kNoAllocMaxN + kNoAllocMaxN +
                                  6 * (size_t)kNoAllocMaxN * kNoAllocMaxN +
                                  (size_t)kNoAllocMaxN * (kNoAllocMaxN | 1);

static __device__ __align__(256) float g_symeig_scratch[kNoAllocFloats];

// The array's device address per device, tagged with the id of the context it
// was resolved in. In host code the symbol name is only a host-side stand-in,
// never a device address; and an address is valid only in its own context (a
// cudaDeviceReset ends the primary context, and the module is loaded afresh
// in the next one), so the cache is keyed on the context id, which CUDA never
// reuses within a process.
constexpr int kMaxDevices = 64;
struct Resolved {
  unsigned long long ctx_id = 0;
  float* addr = nullptr;
};
Resolved g_resolved[kMaxDevices];
std::mutex g_mu;

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (0 when there is none).
bool current_ctx_id(unsigned long long* id) {
  static CtxGetCurrent get_current = nullptr;
  static CtxGetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
            cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
      return false;
    get_current = reinterpret_cast<CtxGetCurrent>(a);
    get_id = reinterpret_cast<CtxGetId>(b);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return false;
  *id = 0;
  return !ctx || get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_symeig_scratch in the current context of device `dev`,
// resolved by cudaGetSymbolAddress once per device and context (with that
// device current; the first resolution loads the module).
float* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) return nullptr;
  Resolved& r = g_resolved[dev];
  if (id != 0 && r.addr && r.ctx_id == id) return r.addr;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_symeig_scratch) != cudaSuccess || !p) return nullptr;
  if (!current_ctx_id(&id) || id == 0) return nullptr;  // the lookup made the context current
  r.ctx_id = id;
  r.addr = static_cast<float*>(p);
  return r.addr;
}

}  // namespace
}  // namespace sfd

extern "C" int sfd_symeig_noalloc(int32_t n, const float* S, int32_t nwant, float* evals,
                                  float* evecs) {
  using namespace sfd;
  if (n < 1 || n > kNoAllocMaxN || nwant < 1 || nwant > n || !S || !evals || !evecs)
    return SFD_EINVAL;
  if (symeig_work_floats(n, nwant) > kNoAllocFloats) return SFD_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SFD_ECUDA;
  float* scratch = scratch_address(dev);
  if (!scratch) return SFD_ECUDA;
  try {
    // the eigensolver writes every scratch word before reading it, so nothing
    // needs clearing between calls
    symeig(S, n, nwant, evals, evecs, scratch, 0);
    SFD_CUDA(cudaStreamSynchronize(0));
  } catch (const CudaError&) {
    return SFD_ECUDA;
  }
  return SFD_OK;
}
