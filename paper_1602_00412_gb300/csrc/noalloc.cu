// sfd_symeig_noalloc: the symmetric eigensolver of sfd_symeig with its scratch
// in a fixed device array instead of memory allocated per call.
//
// Why: some callers cannot let a library call cudaMalloc. A serving process
// whose caching allocator has already reserved the device's memory budget has
// nothing left for a private allocation, and a latency-critical loop cannot
// absorb the device-wide synchronisation that cudaMalloc / cudaFree may
// perform. This entry point allocates nothing: the caller passes the input and
// the outputs, and the scratch is `g_symeig_scratch`, a file-scope array that
// every GPU which loads the library holds until the process exits.
#include <atomic>

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

// Device address of g_symeig_scratch, looked up once per device. In host code
// the symbol name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_addr[kMaxDevices];

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
  float* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // first call on this device: resolve the array's device address
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_symeig_scratch) != cudaSuccess || !p) return SFD_ECUDA;
    scratch = static_cast<float*>(p);
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }
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
