// msbem_spd_inverse_noalloc: inversion of one symmetric positive definite
// matrix that allocates no device memory.  The paper has no counterpart; this
// is a service of the library for callers that cannot allocate.
//
// Who cannot allocate: a process that reserves all of its GPU memory for its
// own pool up front (a solve server keeping assembled matrices resident under a
// fixed HBM budget, say) has nothing left for the library's allocator, and a
// latency-critical loop cannot afford cudaMalloc / cudaFree, which synchronize
// the device and may fail under memory pressure.  This entry point therefore
// takes its scratch -- the pivot block and the two panels of the blocked
// Gauss-Jordan recursion, a few index words and the breakdown flag -- from one
// file-scope device array of fixed size.  Every GPU that loads the library holds
// that array until the process exits.
#include <mutex>

#include "msbem_internal.h"

// Bytes the largest admissible matrix needs (see bgj_scratch_bytes in factor.cu):
// 32x32 pivot block + two n x 32 panels of float pairs + 256 bytes of indices.
static constexpr size_t kScratchBytes =
    sizeof(float2) * 32 * 32 + 2 * sizeof(float2) * (size_t)MSBEM_NOALLOC_MAX_N * 32 + 256;

// The scratch.  In host code this name is only a host-side stand-in for the
// device object; the kernels receive its device address obtained below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (the current device), looked
// up once per device.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = (unsigned char*)p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int msbem_spd_inverse_noalloc(const double* A, int64_t n, double* Ainv, void* cuda_stream) {
  if (!A || !Ainv || n < 1 || n > MSBEM_NOALLOC_MAX_N) return MSBEM_INVALID_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return MSBEM_CUDA_ERROR;
  unsigned char* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return MSBEM_CUDA_ERROR;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (A != Ainv &&
      cudaMemcpyAsync(Ainv, A, sizeof(double) * (size_t)n * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return MSBEM_CUDA_ERROR;
  int not_spd = 0;
  if (msbem::bgj_invert_single(Ainv, n, scratch, kScratchBytes, s, &not_spd) != cudaSuccess)
    return MSBEM_CUDA_ERROR;
  return not_spd ? MSBEM_BREAKDOWN : MSBEM_OK;
}
