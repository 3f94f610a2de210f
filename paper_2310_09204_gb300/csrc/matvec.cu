// Dense Galerkin matrix times k <= 16 vectors, Q = W P (the matrix-vector
// product of the PCG iteration, Sec. 2.1, for one or several right-hand
// sides at once).
//
// W is held as two FP32 planes, hi and lo (W = hi + lo to ~2^-48 relative),
// each N x ldw with ldw a multiple of 32 and zero padding; P is held the same
// way, transposed: planes of k x ldp floats.  A CTA owns 16 rows (two per
// warp; 32 rows, four per warp, in FP32) and walks the columns in chunks of
// 128:
//
//   * one thread issues two TMA tensor copies per chunk (a rows x 128 x planes
//     box of W and a KB x 128 x planes box of P, KB = k rounded up to a power
//     of two, the extra rows zero-filled by the copy) into a shared-memory
//     ring of 2-6 stages, completed through one mbarrier per stage;
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

#include <algorithm>
#include <array>
#include <mutex>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define MV_ROWS 16
#define MV_KC 128
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

// Test hook of the error path (msbem_test_expire_waits): when non-zero, every
// product CTA first waits up to this many nanoseconds for g_mv_never, a flag
// that nothing sets, and on expiry takes the path of a copy that never
// completed.  Zero in normal use: one global load per CTA.
__device__ long long g_mv_expire_ns = 0;
__device__ int g_mv_never = 0;

__device__ __noinline__ bool mv_wait_never(long long limit_ns) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (*(volatile int*)&g_mv_never) return true;
    if (global_ns() - t0 > (uint64_t)limit_ns) return false;
  }
  return false;
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

// Compile-time shape of one instantiation: MODE, KB (columns of P, the
// caller's k rounded up to 1, 2, 4, 8 or 16; the TMA fills the extra rows with
// zeros), rows per warp (2 in double-float, 4 in FP32, where the accumulators
// are single floats), and as many pipeline stages as fit in ~100 KB so that
// two CTAs share an SM.
template <int MODE, int KB>
struct MvCfg {
  static constexpr int NPL = MODE == 0 ? 2 : 1;
  static constexpr int RPW = MODE == 0 ? 2 : 4;
  static constexpr int ROWS = 8 * RPW;
  static constexpr int V = RPW * KB;                        // sums per lane
  static constexpr int W_FLOATS = NPL * ROWS * MV_KC;      // per stage
  static constexpr int P_FLOATS = NPL * KB * MV_KC;        // per stage
  static constexpr int STAGE_BYTES = 4 * (W_FLOATS + P_FLOATS);
  static constexpr int S0 = (100 * 1024) / STAGE_BYTES;
  static constexpr int STAGES = S0 > 6 ? 6 : (S0 < 2 ? 2 : S0);
  static constexpr size_t BYTES = 128 + (size_t)STAGES * STAGE_BYTES + sizeof(uint64_t) * STAGES +
                                  sizeof(double) * 8 * V;
};

template <int MODE, int KB>
__global__ void __launch_bounds__(256, 2) matvec_kernel(const __grid_constant__ CUtensorMap tmW,
                                                        const __grid_constant__ CUtensorMap tmP,
                                                        int N, int nchunks_all, int cps, int kb,
                                                        const double* __restrict__ P,
                                                        double* __restrict__ Q,
                                                        double* __restrict__ part,
                                                        float2* __restrict__ split_part,
                                                        const int* __restrict__ stop,
                                                        int* __restrict__ err) {
  if (*stop) return;
  using C = MvCfg<MODE, KB>;
  constexpr int ST = C::STAGES, RPW = C::RPW, V = C::V;
  // column split blockIdx.y covers chunks [chunk0, chunk0 + nchunks)
  const int chunk0 = blockIdx.y * cps;
  const int nchunks = min(nchunks_all - chunk0, cps);
  extern __shared__ unsigned char mv_raw[];
  float* sw = (float*)(((uintptr_t)mv_raw + 127) & ~(uintptr_t)127);
  float* sp = sw + ST * C::W_FLOATS;
  uint64_t* bar = (uint64_t*)(sp + ST * C::P_FLOATS);
  double* spq = (double*)(bar + ST);                        // [8 warps][V]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int row0 = blockIdx.x * C::ROWS;
  const uint32_t tx_bytes = (uint32_t)C::STAGE_BYTES;
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int stage, int chunk) {
    mbar_expect_tx(&bar[stage], tx_bytes);
    tma_load_3d(sw + stage * C::W_FLOATS, &tmW, (chunk0 + chunk) * MV_KC, row0, 0, &bar[stage]);
    tma_load_3d(sp + stage * C::P_FLOATS, &tmP, (chunk0 + chunk) * MV_KC, 0, 0, &bar[stage]);
  };
  if (tid == 0)
    for (int s = 0; s < ST && s < nchunks; ++s) issue(s, s);

  // running sums, index r * KB + c (row r of this warp, column c)
  float h[V], l[MODE == 0 ? V : 1];
#pragma unroll
  for (int i = 0; i < V; ++i) h[i] = 0.f;
#pragma unroll
  for (int i = 0; i < (MODE == 0 ? V : 1); ++i) l[i] = 0.f;

  int failed_at = -1;
  const long long expire = g_mv_expire_ns;
  if (expire > 0) {
    bool got = true;
    if (tid == 0) got = mv_wait_never(expire);
    if (__syncthreads_or(!got)) failed_at = 0;
  }
  for (int t = 0; failed_at < 0 && t < nchunks; ++t) {
    const int s = t % ST;
    const bool got = mbar_wait_bounded(&bar[s], (uint32_t)((t / ST) & 1));
    // every thread has finished chunk t-1 once past this barrier
    if (__syncthreads_or(!got)) { failed_at = t; break; }
    if (tid == 0 && t >= 1 && t - 1 + ST < nchunks) issue((t - 1) % ST, t - 1 + ST);
    const float* ws = sw + s * C::W_FLOATS;
    const float* ps = sp + s * C::P_FLOATS;
    float4 wh[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) wh[r] = *(const float4*)(ws + (RPW * wid + r) * MV_KC + 4 * lane);
    if constexpr (MODE == 0) {
      float4 wl[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        wl[r] = *(const float4*)(ws + (C::ROWS + RPW * wid + r) * MV_KC + 4 * lane);
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        const float4 ph = *(const float4*)(ps + c * MV_KC + 4 * lane);
        const float4 pl = *(const float4*)(ps + (KB + c) * MV_KC + 4 * lane);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          float& ah = h[r * KB + c];
          float& al = l[r * KB + c];
          df_fma_acc(wh[r].x, wl[r].x, ph.x, pl.x, ah, al);
          df_fma_acc(wh[r].y, wl[r].y, ph.y, pl.y, ah, al);
          df_fma_acc(wh[r].z, wl[r].z, ph.z, pl.z, ah, al);
          df_fma_acc(wh[r].w, wl[r].w, ph.w, pl.w, ah, al);
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < KB; ++c) {
        const float4 ph = *(const float4*)(ps + c * MV_KC + 4 * lane);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          float a = h[r * KB + c];
          a = fmaf(wh[r].x, ph.x, a);
          a = fmaf(wh[r].y, ph.y, a);
          a = fmaf(wh[r].z, ph.z, a);
          a = fmaf(wh[r].w, ph.w, a);
          h[r * KB + c] = a;
        }
      }
    }
  }
  if (failed_at >= 0) {
    // drain the copies still in flight: chunks 0 .. ST-1 when nothing was
    // consumed yet, else failed_at .. failed_at+ST-2 (chunk failed_at-1+ST is
    // issued only after chunk failed_at has landed)
    if (tid == 0) {
      const int last = failed_at == 0 ? ST - 1 : failed_at + ST - 2;
      for (int u = failed_at; u < nchunks && u <= last; ++u)
        mbar_wait_bounded(&bar[u % ST], (uint32_t)((u / ST) & 1));
      atomicExch(err, 1);
    }
    return;
  }

  warp_xreduce<V, 16, MODE == 0>(h, l, lane);
  constexpr int F = V >= 32 ? V / 32 : 1;          // sums held per lane
  constexpr int SH = V >= 32 ? 0 : (V == 16 ? 1 : V == 8 ? 2 : V == 4 ? 3 : V == 2 ? 4 : 5);
  const bool writer = (lane & ((1 << SH) - 1)) == 0;
  const bool split = gridDim.y > 1;
#pragma unroll
  for (int j = 0; j < F; ++j) {
    const int idx = V >= 32 ? lane * F + j : (lane >> SH);
    const int r = idx / KB, c = idx - (idx / KB) * KB;
    const int row = row0 + RPW * wid + r;
    const float sh = h[j];
    float sl = 0.f;
    if constexpr (MODE == 0) sl = l[j];
    const bool valid = writer && row < N && c < kb;
    if (split) {
      // this split's partial sum; matvec_combine_kernel adds the splits
      if (valid) split_part[((int64_t)blockIdx.y * N + row) * kb + c] = make_float2(sh, sl);
    } else {
      double pqv = 0.0;
      if (valid) {
        const double q = MODE == 0 ? df_to_double(sh, sl) : (double)sh;
        Q[(int64_t)row * kb + c] = q;
        pqv = q * P[(int64_t)row * kb + c];
      }
      if (writer) spq[wid * V + idx] = pqv;
    }
  }
  if (split) return;
  __syncthreads();
  if (tid < kb) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w)
      for (int r = 0; r < RPW; ++r) sum += spq[w * V + r * KB + tid];
    part[(int64_t)tid * gridDim.x + blockIdx.x] = sum;
  }
}

// Sum of the column splits' partials in split order (double-float), Q and the
// per-block partial sums of p_c . q_c with the same block layout as the
// unsplit kernel (rows blocks of `rows`).
__global__ void __launch_bounds__(256) matvec_combine_kernel(const float2* __restrict__ split_part, int S, int N,
                                                             int kb, int rows, const double* __restrict__ P,
                                                             double* __restrict__ Q, double* __restrict__ part,
                                                             const int* __restrict__ stop) {
  if (*stop) return;
  __shared__ double sq[32 * MV_MAXK];
  const int64_t row0 = (int64_t)blockIdx.x * rows;
  for (int e = threadIdx.x; e < rows * kb; e += 256) {
    const int r = e / kb, c = e - r * kb;
    const int64_t row = row0 + r;
    double pq = 0.0;
    if (row < N) {
      float h = 0.f, l = 0.f;
      for (int sp = 0; sp < S; ++sp) {
        const float2 v = split_part[((int64_t)sp * N + row) * kb + c];
        float sh, se;
        two_sum(h, v.x, sh, se);
        h = sh;
        l = l + v.y + se;
      }
      const double q = df_to_double(h, l);
      Q[row * kb + c] = q;
      pq = q * P[row * kb + c];
    }
    sq[e] = pq;
  }
  __syncthreads();
  if (threadIdx.x < kb) {
    double sum = 0.0;
    for (int r = 0; r < rows; ++r) sum += sq[r * kb + threadIdx.x];
    part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = sum;
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

int matvec_pad(int kb) { return kb <= 1 ? 1 : kb <= 2 ? 2 : kb <= 4 ? 4 : kb <= 8 ? 8 : 16; }
int matvec_rows(int mode) { return mode == 0 ? MvCfg<0, 1>::ROWS : MvCfg<1, 1>::ROWS; }
unsigned matvec_blocks(int64_t N, int mode) {
  const int rows = matvec_rows(mode);
  return (unsigned)((N + rows - 1) / rows);
}

template <int MODE, int KB>
static cudaError_t set_attr() {
  return cudaFuncSetAttribute(matvec_kernel<MODE, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)MvCfg<MODE, KB>::BYTES);
}

// opt in to the dynamic shared memory of every instantiation (once per
// process and device; called outside any stream capture)
cudaError_t matvec_init() {
  static std::mutex mu;
  static std::vector<int> ready;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int d : ready)
    if (d == dev) return cudaSuccess;
  cudaError_t r[10] = {set_attr<0, 1>(), set_attr<0, 2>(), set_attr<0, 4>(), set_attr<0, 8>(), set_attr<0, 16>(),
                       set_attr<1, 1>(), set_attr<1, 2>(), set_attr<1, 4>(), set_attr<1, 8>(), set_attr<1, 16>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  ready.push_back(dev);
  return cudaSuccess;
}

// Column splits for a matrix of order N: enough (row block x split) work
// items for about four waves of two CTAs on each of the 152 SMs, at most 8,
// and none for small matrices.  A function of N and the mode only, so a
// vector's product never depends on how many vectors share the launch.
int matvec_split(int64_t N, int mode) {
  const int64_t nchunks = (N + MV_KC - 1) / MV_KC;
  const int64_t blocks = matvec_blocks(N, mode);
  if (nchunks < 16 || blocks >= 4 * 2 * 152) return 1;
  int64_t S = (4 * 2 * 152 + blocks - 1) / blocks;
  S = std::min<int64_t>(S, 8);
  S = std::min<int64_t>(S, nchunks / 8);
  // every split must own at least one chunk
  while (S > 1 && (S - 1) * ((nchunks + S - 1) / S) >= nchunks) --S;
  return (int)std::max<int64_t>(S, 1);
}

size_t matvec_scratch_bytes(int64_t N, int kb, int split) {
  return split > 1 ? sizeof(float2) * (size_t)split * N * kb : 0;
}

int matvec_split_of(const DevGeom& g, int mode) {
  const int m = mode == 1 ? 1 : 0;
  return g.mv_split[m] > 0 ? g.mv_split[m] : matvec_split(g.ndof, mode);
}

// Candidate column splits (each must own at least one chunk), and the
// process-wide record of the picks
static const int kSplitCandidates[] = {1, 2, 3, 4, 6, 8};
static std::mutex g_tune_mu;
static std::vector<std::array<int64_t, 4>> g_tuned;   // (device, N, mode, split)

cudaError_t matvec_autotune(DevGeom& g, cudaStream_t s) {
  const int64_t N = g.ndof;
  g.mv_split[0] = g.mv_split[1] = 0;
  if (N <= 0) return cudaSuccess;
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t nchunks = (N + MV_KC - 1) / MV_KC;
  bool todo[2] = {true, true};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& t : g_tuned)
      if (t[0] == dev && t[1] == N) {
        g.mv_split[t[2]] = (int)t[3];
        todo[t[2]] = false;
      }
  }
  for (int m = 0; m < 2; ++m)
    if (todo[m] && (nchunks < 16 || matvec_blocks(N, m) >= 4 * 2 * 152)) {
      // small matrices, and large ones whose row blocks alone fill four
      // waves: one CTA per row block, no timing (it would cost a second of
      // products at the cube's size)
      g.mv_split[m] = 1;
      todo[m] = false;
    }
  if (!todo[0] && !todo[1]) return cudaSuccess;
  // scratch: 16 zero vectors, their planes, products, partial sums, the
  // widest split's partials, flags
  const int KBT = 16;
  const size_t nvec = (size_t)N * KBT;
  const size_t nparts = (size_t)KBT * matvec_blocks(N, 0) + (size_t)KBT * matvec_blocks(N, 1);
  const size_t bytes = sizeof(double) * (2 * nvec + nparts) + sizeof(float) * 2 * KBT * g.ldw +
                       matvec_scratch_bytes(N, KBT, 8) + 2 * sizeof(int) + 2048;
  char* base = nullptr;
  cudaError_t e = pool_alloc((void**)&base, bytes, g.pool, s);
  if (e != cudaSuccess) return e;
  auto take = [&](size_t b) { char* p = base; base += (b + 255) / 256 * 256; return p; };
  char* const mem = base;
  double* P = (double*)take(sizeof(double) * nvec);
  double* Q = (double*)take(sizeof(double) * nvec);
  double* part = (double*)take(sizeof(double) * nparts);
  float* Pf = (float*)take(sizeof(float) * 2 * KBT * g.ldw);
  void* scr = take(matvec_scratch_bytes(N, KBT, 8));
  int* flags = (int*)take(2 * sizeof(int));
  cudaMemsetAsync(mem, 0, bytes, s);
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  for (int m = 0; m < 2 && e == cudaSuccess; ++m) {
    if (!todo[m]) continue;
    float best = 3.4e38f;
    int pick = matvec_split(N, m);
    for (int S : kSplitCandidates) {
      if (S > 1 && ((S - 1) * ((nchunks + S - 1) / S) >= nchunks || nchunks / S < 2)) continue;
      float total = 0.f;
      for (int kb : {1, KBT}) {
        CUtensorMap tmP;
        if ((e = encode_planes(&tmP, Pf, g.ldw, kb, kb * g.ldw, m == 0 ? 2 : 1, matvec_pad(kb))) != cudaSuccess)
          break;
        const CUtensorMap& tmW = m == 0 ? g.tm_W : g.tm_Whi;
        float t = 3.4e38f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
          cudaEventRecord(ev[0], s);
          e = launch_matvec(m, tmW, tmP, N, kb, P, Q, part, flags, flags + 1, s, S, scr);
          cudaEventRecord(ev[1], s);
          if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
          float ms = 0.f;
          if (e == cudaSuccess && rep > 0) {   // the first launch warms up
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            t = std::min(t, ms);
          }
        }
        total += t;
      }
      if (e != cudaSuccess) break;
      if (total < best) {
        best = total;
        pick = S;
      }
    }
    g.launches += 36;
    if (e == cudaSuccess) {
      g.mv_split[m] = pick;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned.push_back({dev, N, m, pick});
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  int err = 0;
  cudaMemcpyAsync(&err, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(mem, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess && err) e = cudaErrorTimeout;
  return e != cudaSuccess ? e : e2;
}

template <int MODE, int KB>
static cudaError_t launch_cfg(const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb, int split,
                              const double* P, double* Q, double* part, float2* scratch, const int* stop,
                              int* err, cudaStream_t s) {
  const int nchunks = (int)((N + MV_KC - 1) / MV_KC);
  const int cps = (nchunks + split - 1) / split;
  const dim3 grid(matvec_blocks(N, MODE), split);
  matvec_kernel<MODE, KB><<<grid, 256, MvCfg<MODE, KB>::BYTES, s>>>(tmW, tmP, (int)N, nchunks, cps, kb, P, Q,
                                                                    part, scratch, stop, err);
  if (split > 1)
    matvec_combine_kernel<<<matvec_blocks(N, MODE), 256, 0, s>>>(scratch, split, (int)N, kb, MvCfg<MODE, KB>::ROWS,
                                                                 P, Q, part, stop);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb, int split,
                               const double* P, double* Q, double* part, float2* scr, const int* stop, int* err,
                               cudaStream_t s) {
  switch (matvec_pad(kb)) {
    case 1: return launch_cfg<MODE, 1>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
    case 2: return launch_cfg<MODE, 2>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
    case 4: return launch_cfg<MODE, 4>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
    case 8: return launch_cfg<MODE, 8>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
    default: return launch_cfg<MODE, 16>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
  }
}

cudaError_t set_matvec_expire_ns(long long ns) {
  return cudaMemcpyToSymbol(g_mv_expire_ns, &ns, sizeof(ns));
}

cudaError_t launch_matvec(int mode, const CUtensorMap& tmW, const CUtensorMap& tmP, int64_t N, int kb,
                          const double* P, double* Q, double* part, const int* stop, int* err,
                          cudaStream_t s, int split, void* scratch) {
  if (N <= 0 || N > 0x7fffffff || kb < 1 || kb > MV_MAXK || split < 1 || (split > 1 && !scratch))
    return cudaErrorInvalidValue;
  float2* scr = (float2*)scratch;
  return mode == 0 ? launch_mode<0>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s)
                   : launch_mode<1>(tmW, tmP, N, kb, split, P, Q, part, scr, stop, err, s);
}

}  // namespace msbem
