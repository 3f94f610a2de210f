// The rank-32 update of the blocked Gauss-Jordan set-up (Sec. 5, eq.
// jumpSplit: the face, wire-basket and coarse blocks of M(H;h) inverted
// explicitly) on the tcgen05 tensor cores, with the accuracy of the
// double-float path.
//
// One step updates every entry of an active matrix from the left operand L
// (row r: the scaled pivot row P[r - k0] for the 32 pivot rows K, else the
// panel row C'_r) and the right operand R (the old pivot rows A[K][c]):
//   A[r][c] = L(r)[c - k0]                          for c in K,
//   A[r][c] = [r not in K] A[r][c] + L(r) . R[:, c]   otherwise.
// The product L R is formed exactly in integers: each row of L is scaled by a
// power of two 2^-e_r into (-1/2, 1/2), rounded to 48 bits and cut into six
// balanced base-256 digits (each exact in bf16); each column of R likewise
// with 2^-f_c.  Then (L R)[r][c] = 2^(e_r + f_c) sum_l 2^(-8l) Q_l[r][c] with
// Q_l = sum_{s+t=l} a_s b_t, a product of integer matrices that a kind::f16
// MMA (bf16 operands, FP32 accumulators in tensor memory) forms exactly (K =
// 32 terms of at most 2^14, at most 7 slice pairs per level: below 2^22).
// Levels up to 8 are kept (26 slice pairs); the rest lie below 2^-51 of the
// operands' scales.  The levels are folded into double-float sums and the
// entries of A (FP64) updated.
//
// Work per step: two slicing kernels (left rows, right columns) write the
// digits in the tensor cores' shared-memory order (128-byte rows, 128-byte
// swizzle), so one CTA per 128 x 64 output tile brings its twelve digit tiles
// in by bulk asynchronous copies, issues 52 MMAs from one thread, folds the
// seven level accumulators and rewrites its tile of A.  Every wait is bounded
// (an error flag, the copies in flight drained, the tensor memory freed).
#include <cuda_bf16.h>

#include <mutex>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

namespace {

constexpr int KG = 32;            // pivot panel width of the recursion
constexpr int TR = 128;           // rows of an output tile (TMEM lanes)
constexpr int TCC = 64;           // columns of an output tile
constexpr int ND = 6;             // digits per operand entry
constexpr int LEVELS = 7;         // levels 2 .. 8
constexpr int LBLK = TR * 128;    // bytes of one left digit tile (128 rows x 64 K bf16)
constexpr int RBLK = TCC * 128;   // bytes of one right digit tile (64 columns x 64 K bf16)
constexpr int SMEM_OPS = ND * LBLK + ND * RBLK;
constexpr int SMEM = 1024 + SMEM_OPS + 128;

using TcuArgs = TcuDev;

__device__ __forceinline__ int tcu_find(const int64_t* pre, int active, int64_t t) {
  int lo = 0, hi = active - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// e with |x| < 2^(e-1) for every x of the float pairs whose largest |hi| is m
// (0 for a zero row, whose digits are all zero)
__device__ __forceinline__ int tcu_exp(float m) {
  if (!(m > 0.f)) return 0;
  int k = 0;
  frexpf(m, &k);   // m in [2^(k-1), 2^k)
  return k + 1;
}

// the six balanced base-256 digits of x (|x| < 1/2): x = sum_i d[i] 2^(-8(i+1)),
// d[0] the most significant
__device__ __forceinline__ void tcu_digits(double x, int* d) {
  long long v = llrint(x * 281474976710656.0);   // x 2^48, |v| < 2^47
#pragma unroll
  for (int i = ND - 1; i >= 1; --i) {
    const long long r = ((v + 128) & 255) - 128;   // in [-128, 127]
    d[i] = (int)r;
    v = (v - r) >> 8;                               // exact: v - r is a multiple of 256
  }
  d[0] = (int)v;                                    // |d[0]| <= 128
}

// One row (left) or column (right) of an operand: its K = 32 float pairs
// (kb of them used), the exponent, and the 64 K positions of the six digit
// tiles (K >= kb and 32 .. 63 zero), written as 16-byte chunks in the
// swizzled order of row `row` of tiles digit_stride bytes apart.
__device__ __forceinline__ int tcu_slice_row(const float2* v, int64_t vstride, int kb, unsigned char* base,
                                             size_t digit_stride, int row) {
  float m = 0.f;
  for (int k = 0; k < kb; ++k) m = fmaxf(m, fabsf(v[k * vstride].x));
  const int e = tcu_exp(m);
  const double sc = ldexp(1.0, -e);
#pragma unroll 1
  for (int j = 0; j < 8; ++j) {              // 16-byte chunk j: K positions 8j .. 8j+7
    unsigned short h[ND][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = 8 * j + q;
      int d[ND] = {0, 0, 0, 0, 0, 0};
      if (k < kb && m > 0.f) {   // (e = 0 is also the exponent of a row whose largest |hi| is in [1/4, 1/2))
        const float2 x = v[k * vstride];
        tcu_digits((widen(x.x) + widen(x.y)) * sc, d);
      }
#pragma unroll
      for (int i = 0; i < ND; ++i) h[i][q] = __bfloat16_as_ushort(__float2bfloat16((float)d[i]));
    }
    const uint32_t o = (uint32_t)(row * 128 + ((j ^ (row & 7)) << 4));
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      uint4 w;
      w.x = h[i][0] | ((uint32_t)h[i][1] << 16);
      w.y = h[i][2] | ((uint32_t)h[i][3] << 16);
      w.z = h[i][4] | ((uint32_t)h[i][5] << 16);
      w.w = h[i][6] | ((uint32_t)h[i][7] << 16);
      *(uint4*)(base + (size_t)i * digit_stride + o) = w;
    }
  }
  return e;
}

// left operand: one thread per row of the active matrices (rows padded to 128)
__global__ void __launch_bounds__(128) tcu_left_kernel(TcuArgs g, int active, int64_t k0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.pl[active]) return;
  const int a = tcu_find(g.pl, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int64_t r = t - g.pl[a];
  const int kb = (int)(n - k0 < KG ? n - k0 : KG);
  unsigned char* base = g.Lsl + (size_t)(t / TR) * ND * LBLK;
  const float2 zero[1] = {make_float2(0.f, 0.f)};
  const float2* v = zero;
  int64_t vs = 0;
  int kk = 0;
  if (r < n) {
    kk = kb;
    vs = 1;
    v = (r >= k0 && r < k0 + kb) ? g.Pf + (int64_t)a * KG * KG + (r - k0) * KG : g.Cf + g.soff[a] + r * KG;
  }
  g.exL[t] = tcu_slice_row(v, vs, kk, base, LBLK, (int)(t % TR));
}

// right operand: one thread per column of the active matrices (padded to 64)
__global__ void __launch_bounds__(128) tcu_right_kernel(TcuArgs g, int active, int64_t k0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.pr[active]) return;
  const int a = tcu_find(g.pr, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int64_t c = t - g.pr[a];
  const int kb = (int)(n - k0 < KG ? n - k0 : KG);
  unsigned char* base = g.Rsl + (size_t)(t / TCC) * ND * RBLK;
  const float2 zero[1] = {make_float2(0.f, 0.f)};
  const float2* v = zero;
  int64_t vs = 0;
  int kk = 0;
  if (c < n) {
    kk = kb;
    vs = n;
    v = g.Rf + g.soff[a] + c;
  }
  g.exR[t] = tcu_slice_row(v, vs, kk, base, RBLK, (int)(t % TCC));
}

__device__ __forceinline__ uint32_t tcu_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// wait for phase 0 of the barrier; false after ~2 s or 2^24 polls
__device__ __noinline__ bool tcu_wait(uint64_t* bar) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0,1,0,p;\n}\n"
        : "=r"(ok) : "r"(tcu_smem(bar)) : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 2000000000ull) return false;
  }
  return false;
}

// shared-memory matrix descriptor: K-major, 128-byte rows under the 128-byte
// swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t tcu_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tcu_ld16(uint32_t addr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(addr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :: "memory");
}

// One 128 x 64 tile of one active matrix per CTA (four warps = the 128 TMEM
// lanes).  Thread 0 brings in the twelve digit tiles and issues the MMAs;
// every warp folds its 32 rows; the tile of A is rewritten row by row.
__global__ void __launch_bounds__(128, 1) tcu_update_kernel(TcuArgs g, int active, int64_t k0) {
  extern __shared__ unsigned char tcu_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcu_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB = base + ND * LBLK;
  uint64_t* bars = (uint64_t*)(base + SMEM_OPS);   // [0] copies landed, [1] MMAs done
  uint32_t* tbase = (uint32_t*)(bars + 2);
  float2* stage = (float2*)base;                   // the tile's sums, once the MMAs are done
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t t = blockIdx.x;
  const int a = tcu_find(g.pt, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int64_t ntc = (n + TCC - 1) / TCC;
  const int64_t loc = t - g.pt[a];
  const int64_t r0 = (loc / ntc) * TR, c0 = (loc % ntc) * TCC;
  const int kb = (int)(n - k0 < KG ? n - k0 : KG);
  const int64_t Lt = (g.pl[a] + r0) / TR, Rt = (g.pr[a] + c0) / TCC;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcu_smem(tbase)),
                 "r"(512) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcu_smem(&bars[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tcu_smem(&bars[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tbase;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tcu_smem(&bars[0])),
                 "r"(SMEM_OPS) : "memory");
    for (int i = 0; i < ND; ++i) {
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(tcu_smem(sA + i * LBLK)), "l"(g.Lsl + ((size_t)Lt * ND + i) * LBLK), "r"(LBLK),
                   "r"(tcu_smem(&bars[0])) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(tcu_smem(sB + i * RBLK)), "l"(g.Rsl + ((size_t)Rt * ND + i) * RBLK), "r"(RBLK),
                   "r"(tcu_smem(&bars[0])) : "memory");
    }
  }
  const bool landed = __syncthreads_and(tcu_wait(&bars[0]));
  if (landed && tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // bf16 A and B, FP32 accumulators, M = 128, N = 64
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TCC >> 3) << 17) |
                           ((uint32_t)(TR >> 4) << 24);
    for (int l = 0; l < LEVELS; ++l) {        // level l + 2: digit pairs i + j = l
      uint32_t en = 0;                        // the level's first MMA overwrites its accumulator
      for (int i = 0; i < ND && i <= l; ++i) {
        const int j = l - i;
        if (j >= ND) continue;
        for (int kk = 0; kk < KG / 16; ++kk) {
          const uint64_t ad = tcu_desc(tcu_smem(sA + i * LBLK) + 32u * kk);
          const uint64_t bd = tcu_desc(tcu_smem(sB + j * RBLK) + 32u * kk);
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(taddr + (uint32_t)(l * TCC)), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
          en = 1;
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(tcu_smem(&bars[1])) : "memory");
  }
  const bool done = __syncthreads_and(landed && tcu_wait(&bars[1]));
  if (!done) {
    // give up: let the copies (or the MMAs) in flight finish, bounded, before
    // the shared memory and the accumulators are given back
    if (tid == 0) {
      tcu_wait(landed ? &bars[1] : &bars[0]);
      atomicExch(g.err, 1);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = 32 * warp + lane;
    const int eL = g.exL[Lt * TR + row];
    for (int cc = 0; cc < TCC / 16; ++cc) {
      uint32_t q[LEVELS][16];
#pragma unroll
      for (int l = 0; l < LEVELS; ++l)
        tcu_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(l * TCC + 16 * cc), q[l]);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        // sum_l Q_l 2^(-8(l+2)) in double-float, smallest level first (each
        // term exact: Q_l is an integer below 2^22)
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int l = LEVELS - 1; l >= 0; --l) {
          float s2, e2;
          two_sum(sh, ldexpf(__uint_as_float(q[l][j]), -8 * (l + 2)), s2, e2);
          sh = s2;
          sl += e2;
        }
        const int sc = eL + g.exR[Rt * TCC + 16 * cc + j];
        stage[row * TCC + 16 * cc + j] = make_float2(ldexpf(sh, sc), ldexpf(sl, sc));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (done) {
    double* A = g.Ap[b];
    for (int rr = warp; rr < TR; rr += 4) {
      const int64_t R = r0 + rr;
      if (R >= n) break;
      const bool rK = R >= k0 && R < k0 + kb;
      for (int jj = lane; jj < TCC; jj += 32) {
        const int64_t C = c0 + jj;
        if (C >= n) continue;
        double* dst = A + R * n + C;
        if (C >= k0 && C < k0 + kb) {
          const float2 L = rK ? g.Pf[(int64_t)a * KG * KG + (R - k0) * KG + (C - k0)]
                              : g.Cf[g.soff[a] + R * KG + (C - k0)];
          *dst = df_to_double(L.x, L.y);
        } else {
          const float2 u = stage[rr * TCC + jj];
          *dst = (rK ? 0.0 : *dst) + df_to_double(u.x, u.y);
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(512) : "memory");
}

}  // namespace

size_t tc_update_bytes(int64_t rows, int64_t cols) {
  return (size_t)rows * ND * 128 + (size_t)cols * ND * 128;
}

cudaError_t tc_update_init() {
  static std::mutex mu;
  static std::vector<int> ready;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int d : ready)
    if (d == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(tcu_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e == cudaSuccess) ready.push_back(dev);
  return e;
}

cudaError_t launch_tc_update(const TcuDev& d, int active, int64_t k0, int64_t rows, int64_t cols, int64_t tiles,
                             cudaStream_t s) {
  if (rows <= 0 || tiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffff || rows / 128 > 0x7fffffff || cols / 128 > 0x7fffffff) return cudaErrorInvalidValue;
  tcu_left_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(d, active, k0);
  tcu_right_kernel<<<(unsigned)((cols + 127) / 128), 128, 0, s>>>(d, active, k0);
  tcu_update_kernel<<<(unsigned)tiles, 128, SMEM, s>>>(d, active, k0);
  return cudaGetLastError();
}

}  // namespace msbem
