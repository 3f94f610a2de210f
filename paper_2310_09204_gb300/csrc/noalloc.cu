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
// file-scope device array of fixed size.  The array exists on a GPU once the
// library's device code is loaded there (at the first use of the library on that
// GPU, under lazy module loading) and stays until the process exits.
#include "msbem_internal.h"

// Bytes the largest admissible matrix needs (see bgj_scratch_bytes in factor.cu):
// 32x32 pivot block + two n x 32 panels of float pairs + 256 bytes of indices.
static constexpr size_t kScratchBytes =
    sizeof(float2) * 32 * 32 + 2 * sizeof(float2) * (size_t)MSBEM_NOALLOC_MAX_N * 32 + 256;

// The scratch.  In host code this name is only a host-side stand-in for the
// device object; the kernels receive its device address obtained below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Device address of g_noalloc_scratch on the current device.  It is looked up
// on every call (a cheap query): a cached address would go stale when the
// caller resets the device and the module is loaded again.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = (unsigned char*)p;
  return cudaSuccess;
}

}  // namespace

extern "C" int msbem_spd_inverse_noalloc(const double* A, int64_t n, double* Ainv, void* cuda_stream) {
  if (!A || !Ainv || n < 1 || n > MSBEM_NOALLOC_MAX_N) return MSBEM_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the call copies index words from pageable host memory and waits on the
  // stream for the breakdown flag, neither of which a stream capture allows
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return MSBEM_CUDA_ERROR;
  if (cap != cudaStreamCaptureStatusNone) return MSBEM_INVALID_ARG;
  unsigned char* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return MSBEM_CUDA_ERROR;
  if (A != Ainv &&
      cudaMemcpyAsync(Ainv, A, sizeof(double) * (size_t)n * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return MSBEM_CUDA_ERROR;
  int not_spd = 0;
  if (msbem::bgj_invert_single(Ainv, n, scratch, kScratchBytes, s, &not_spd) != cudaSuccess)
    return MSBEM_CUDA_ERROR;
  return not_spd ? MSBEM_BREAKDOWN : MSBEM_OK;
}
