// Dense Galerkin matrix times k <= 16 vectors, Q = W P (the matrix-vector
// product of the PCG iteration, Sec. 2.1, for one or several right-hand
// sides at once).
//
// W is held as two FP32 planes, hi and lo (W = hi + lo to ~2^-48 relative),
// each N x ldw with ldw a multiple of 32 and zero padding; P is held the same
// way, transposed: planes of k x ldp floats.  A CTA owns 16 rows (two per
// warp) and walks the columns in chunks of 128:
//
//   * one thread issues two TMA tensor copies per chunk (a 16 x 128 x planes
//     box of W and a k x 128 x planes box of P) into a 3-stage shared-memory
//     ring, completed through one mbarrier per stage;
//   * lane l handles columns 4l .. 4l+3 of the chunk (float4 reads of both
//     tiles, free of bank conflicts) and keeps, per row and right-hand side,
//     a running sum;
//   * at the end each warp reduces its rows across lanes, writes Q and the
//     block's partial sums of p_c . q_c.
//
// MODE 0 (double-float): products are formed exactly with FMA and summed as
// unevaluated float pairs (13 FP32 operations per entry and right-hand side);
// the FP32 pipe bounds it once k >= 2, HBM (8 bytes per entry) below that.
// MODE 1 (FP32): the hi plane only, plain FMA accumulation (4 bytes per entry,
// HBM-bound for every k <= 16); used by the inner solves of iterative
// refinement.
//
// Every wait on an mbarrier is bounded (time and iteration count); a CTA that
// gives up records the failure in *err, waits (bounded again) for its copies
// still in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define MV_ROWS 16
#define MV_KC 128
#define MV_STAGES 3
#define MV_MAXK 16

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the given phase parity; false after ~2 s or 2^24 polls
__device__ __noinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int MODE>
struct MvLayout {
  static constexpr int NPL = MODE == 0 ? 2 : 1;
  static constexpr int W_FLOATS = NPL * MV_ROWS * MV_KC;   // per stage
  static constexpr int P_FLOATS = NPL * MV_MAXK * MV_KC;   // per stage
  static constexpr size_t BYTES = 128 + sizeof(float) * MV_STAGES * (W_FLOATS + P_FLOATS) +
                                  sizeof(uint64_t) * MV_STAGES + sizeof(double) * 8 * MV_MAXK;
};

template <int MODE>
__global__ void __launch_bounds__(256, 2) matvec_kernel(const __grid_constant__ CUtensorMap tmW,
                                                        const __grid_constant__ CUtensorMap tmP,
                                                        int N, int nchunks, int kb,
                                                        const double* __restrict__ P,
                                                        double* __restrict__ Q,
                                                        double* __restrict__ part,
                                                        const int* __restrict__ stop,
                                                        int* __restrict__ err) {
  if (*stop) return;
  using L = MvLayout<MODE>;
  extern __shared__ unsigned char mv_raw[];
  float* sw = (float*)(((uintptr_t)mv_raw + 127) & ~(uintptr_t)127);
  float* sp = sw + MV_STAGES * L::W_FLOATS;
  uint64_t* bar = (uint64_t*)(sp + MV_STAGES * L::P_FLOATS);
  double* spart = (double*)(bar + MV_STAGES);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int row0 = blockIdx.x * MV_ROWS;
  const uint32_t tx_bytes = (uint32_t)(sizeof(float) * L::NPL * MV_KC * (MV_ROWS + kb));
  if (tid == 0) {
    for (int s = 0; s < MV_STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int stage, int chunk) {
    mbar_expect_tx(&bar[stage], tx_bytes);
    tma_load_3d(sw + stage * L::W_FLOATS, &tmW, chunk * MV_KC, row0, 0, &bar[stage]);
    tma_load_3d(sp + stage * L::P_FLOATS, &tmP, chunk * MV_KC, 0, 0, &bar[stage]);
  };
  if (tid == 0)
    for (int s = 0; s < MV_STAGES && s < nchunks; ++s) issue(s, s);

  float h[2][MV_MAXK], l[2][MV_MAXK];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < MV_MAXK; ++c) { h[r][c] = 0.f; l[r][c] = 0.f; }

  int failed_at = -1;
  for (int t = 0; t < nchunks; ++t) {
    const int s = t % MV_STAGES;
    const bool got = mbar_wait_bounded(&bar[s], (uint32_t)((t / MV_STAGES) & 1));
    // every thread has finished chunk t-1 once past this barrier
    if (__syncthreads_or(!got)) { failed_at = t; break; }
    if (tid == 0 && t >= 1 && t - 1 + MV_STAGES < nchunks)
      issue((t - 1) % MV_STAGES, t - 1 + MV_STAGES);
    const float* ws = sw + s * L::W_FLOATS;
    const float* ps = sp + s * L::P_FLOATS;
    const float4 wh0 = *(const float4*)(ws + (2 * wid) * MV_KC + 4 * lane);
    const float4 wh1 = *(const float4*)(ws + (2 * wid + 1) * MV_KC + 4 * lane);
    if (MODE == 0) {
      const float4 wl0 = *(const float4*)(ws + (MV_ROWS + 2 * wid) * MV_KC + 4 * lane);
      const float4 wl1 = *(const float4*)(ws + (MV_ROWS + 2 * wid + 1) * MV_KC + 4 * lane);
#pragma unroll
      for (int c = 0; c < MV_MAXK; ++c) {
        if (c < kb) {
          const float4 ph = *(const float4*)(ps + c * MV_KC + 4 * lane);
          const float4 pl = *(const float4*)(ps + (kb + c) * MV_KC + 4 * lane);
          df_fma_acc(wh0.x, wl0.x, ph.x, pl.x, h[0][c], l[0][c]);
          df_fma_acc(wh1.x, wl1.x, ph.x, pl.x, h[1][c], l[1][c]);
          df_fma_acc(wh0.y, wl0.y, ph.y, pl.y, h[0][c], l[0][c]);
          df_fma_acc(wh1.y, wl1.y, ph.y, pl.y, h[1][c], l[1][c]);
          df_fma_acc(wh0.z, wl0.z, ph.z, pl.z, h[0][c], l[0][c]);
          df_fma_acc(wh1.z, wl1.z, ph.z, pl.z, h[1][c], l[1][c]);
          df_fma_acc(wh0.w, wl0.w, ph.w, pl.w, h[0][c], l[0][c]);
          df_fma_acc(wh1.w, wl1.w, ph.w, pl.w, h[1][c], l[1][c]);
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < MV_MAXK; ++c) {
        if (c < kb) {
          const float4 ph = *(const float4*)(ps + c * MV_KC + 4 * lane);
          h[0][c] = fmaf(wh0.x, ph.x, h[0][c]);
          h[1][c] = fmaf(wh1.x, ph.x, h[1][c]);
          l[0][c] = fmaf(wh0.y, ph.y, l[0][c]);
          l[1][c] = fmaf(wh1.y, ph.y, l[1][c]);
          h[0][c] = fmaf(wh0.z, ph.z, h[0][c]);
          h[1][c] = fmaf(wh1.z, ph.z, h[1][c]);
          l[0][c] = fmaf(wh0.w, ph.w, l[0][c]);
          l[1][c] = fmaf(wh1.w, ph.w, l[1][c]);
        }
      }
    }
  }
  if (failed_at >= 0) {
    // drain the copies still in flight (chunks failed_at .. failed_at+STAGES-2)
    if (tid == 0) {
      for (int u = failed_at; u < nchunks && u <= failed_at + MV_STAGES - 2; ++u)
        mbar_wait_bounded(&bar[u % MV_STAGES], (uint32_t)((u / MV_STAGES) & 1));
      atomicExch(err, 1);
    }
    return;
  }

  double pq[MV_MAXK];
#pragma unroll
  for (int c = 0; c < MV_MAXK; ++c) pq[c] = 0.0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int row = row0 + 2 * wid + r;
#pragma unroll
    for (int c = 0; c < MV_MAXK; ++c) {
      if (c >= kb) break;
      double q;
      if (MODE == 0) {
        float acch = h[r][c], accl = l[r][c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float oh = __shfl_xor_sync(0xffffffffu, acch, off);
          const float ol = __shfl_xor_sync(0xffffffffu, accl, off);
          float sh, se;
          two_sum(acch, oh, sh, se);
          acch = sh;
          accl = accl + ol + se;
        }
        q = df_to_double(acch, accl);
      } else {
        float acc = h[r][c] + l[r][c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        q = (double)acc;
      }
      if (row < N) {
        if (lane == 0) Q[(int64_t)row * kb + c] = q;
        pq[c] = fma(q, P[(int64_t)row * kb + c], pq[c]);
      }
    }
  }
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < MV_MAXK; ++c)
      if (c < kb) spart[wid * MV_MAXK + c] = pq[c];
  __syncthreads();
  if (tid < kb) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += spart[w * MV_MAXK + tid];
    part[(int64_t)tid * gridDim.x + blockIdx.x] = sum;
  }
}

// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

cudaError_t encode_planes(CUtensorMap* map, const float* base, int64_t ld, int64_t rows,
                          int64_t plane_stride, int nplanes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (ld % 4 || plane_stride % 4 || ((uintptr_t)base & 15) || box_rows < 1 || box_rows > 256 ||
      rows < 1)
    return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)plane_stride * 4};
  cuuint32_t box[3] = {MV_KC, (cuuint32_t)box_rows, (cuuint32_t)nplanes};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

unsigned matvec_blocks(int64_t N) { return (unsigned)((N + MV_ROWS - 1) / MV_ROWS); }

// opt in to the dynamic shared memory of both modes (once per process and
// device; called outside any stream capture)
cudaError_t matvec_init() {
  static std::mutex mu;
  static std::vector<int> ready;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int d : ready)
    if (d == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(matvec_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)MvLayout<0>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(matvec_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MvLayout<1>::BYTES);
  if (e == cudaSuccess) ready.push_back(dev);
  return e;
}

template <int MODE>
static cudaError_t launch_mode(const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb,
                               const double* P, double* Q, double* part, const int* stop, int* err,
                               cudaStream_t s) {
  const int nchunks = (int)((N + MV_KC - 1) / MV_KC);
  matvec_kernel<MODE><<<matvec_blocks(N), 256, MvLayout<MODE>::BYTES, s>>>(tmW, tmP, (int)N, nchunks, kb,
                                                                           P, Q, part, stop, err);
  return cudaGetLastError();
}

cudaError_t launch_matvec(int mode, const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb,
                          const double* P, double* Q, double* part, const int* stop, int* err,
                          cudaStream_t s) {
  if (N <= 0 || N > 0x7fffffff || kb < 1 || kb > MV_MAXK) return cudaErrorInvalidValue;
  return mode == 0 ? launch_mode<0>(tmW, tmP, N, kb, P, Q, part, stop, err, s)
                   : launch_mode<1>(tmW, tmP, N, kb, P, Q, part, stop, err, s);
}

}  // namespace msbem
