// Q = W P in double-float accuracy on the tensor cores (tcgen05), for up to
// 16 vectors: exact integer slicing of both operands.
//
// Every row i of W is scaled by 2^-e_i so that its entries lie in (-1/2, 1/2)
// and written as six signed 8-bit digits, W_ij = 2^e_i sum_s a_s[i,j] 2^-8s
// (+ a remainder below 2^-49 of 2^e_i), each digit rounded to nearest so that
// |a_s| <= 128: an integer that bf16 holds exactly.  The vectors P are sliced
// the same way per column (exponent f_c, digits b_t).  Then
//
//   (W P)_ic = 2^(e_i + f_c) sum_l 2^-8l sum_{s+t=l} sum_j a_s[i,j] b_t[j,c],
//
// and every inner sum over j is a product of bf16 integer matrices: the tensor
// core forms it with FP32 accumulation, exactly, as long as the partial sums
// stay below 2^24.  Every slice pair (s, t) has its own accumulator; products
// are below 2^14, so a window of 512 columns (sums below 2^23) is folded from
// TMEM into double-float registers before the next one starts.  Levels above
// 8 are left out: they add less than 2^-46 of the row and column scales.
//
// One CTA: 128 rows (M = 128), all vectors padded to 16, a range of 32-column
// chunks; TMA brings the six W slices (128 x 32 x 6 bf16, 64-byte swizzle)
// and the six P slices (16 x 32 x 6) of a chunk into a four-stage ring.  The P
// slices lie side by side in shared memory, so one MMA per W slice s and K
// step (N = 16 x the slices u with s + u <= 8) forms all its pair sums at once
// into TMEM (416 columns); all four warps fold them every 512 columns.  Warp 5
// issues the copies, warp 4 the MMAs, warps 0-3 fold.  Waits are bounded;
// TMEM is always freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define TC_NSL 6          // slices per operand
#define TC_LMAX 8         // highest level kept (s + t)
#ifndef TC_ROWB
#define TC_ROWB 128       // bytes of a chunk row: the swizzle span (32, 64 or 128)
#endif
#define TC_KC (TC_ROWB / 2)   // columns per chunk
#define TC_WIN (512 / TC_KC)  // chunks per fold window (512 columns: pair sums below 2^23)
#define TC_ROWS 128
#define TC_NV 16          // vectors (MMA N)
#ifndef TC_STAGES
#define TC_STAGES (256 / TC_ROWB)
#endif
#ifndef TC_PROMO
#define TC_PROMO CU_TENSOR_MAP_L2_PROMOTION_L2_256B
#endif
#define TC_W_BYTES (TC_NSL * TC_ROWS * TC_KC * 2)   // 48 KB
#define TC_P_BYTES (TC_NSL * TC_NV * TC_KC * 2)     // 6 KB
#define TC_STAGE_BYTES (TC_W_BYTES + TC_P_BYTES)
#define TC_SMEM (1024 + TC_STAGES * TC_STAGE_BYTES + 256)   // + barriers and flags (< 256 B)

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t tc_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of `parity`: false after 2 s, or at once when
// another role of the CTA has given up (*fail set; fail may be null).
__device__ __noinline__ bool tc_wait(uint64_t* bar, uint32_t parity, const volatile int* fail) {
  const uint64_t t0 = tc_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0,1,0,p;\n}\n"
        : "=r"(ok) : "r"(tc_smem(bar)), "r"(parity) : "memory");
    if (ok) return true;
    if ((fail && *fail) || tc_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}
// shared-memory matrix descriptor: K-major, rows of TC_ROWB bytes under the
// swizzle of that span (layout 2: 128 B, 4: 64 B, 6: 32 B), 8-row groups
// group_stride bytes apart
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t group_stride = 8 * TC_ROWB) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(group_stride >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)(TC_ROWB == 128 ? 2 : TC_ROWB == 64 ? 4 : 6) << 61);
}

// ---- slicing ---------------------------------------------------------------
// e_i: 2^e_i in (2 max_j |W_ij|, 4 max_j |W_ij|] (0 for a zero row)
__global__ void tc_row_exp_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl, int64_t ldw,
                                  int64_t N, int* __restrict__ ex) {
  __shared__ double sm[256];
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < N; j += 256) m = fmax(m, fabs(df_to_double(Wh[i * ldw + j], Wl[i * ldw + j])));
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int e = 0;
    if (sm[0] > 0.0) frexp(sm[0], &e);   // max in [2^(e-1), 2^e)
    ex[i] = sm[0] > 0.0 ? e + 1 : 0;
  }
}

// six signed 8-bit digits of x in (-1/2, 1/2): x = sum_s d_s 256^-s + r
__device__ __forceinline__ void tc_digits(double x, __nv_bfloat16* d, int64_t stride) {
#pragma unroll
  for (int s = 0; s < TC_NSL; ++s) {
    x *= 256.0;
    const double a = rint(x);
    x -= a;
    d[s * stride] = __float2bfloat16((float)a);
  }
}

// Blocked layout of the W slices: tiles of 8 rows x TC_KC columns, the six
// slices of a tile side by side, tiles by chunk within a row group:
//   element (s, i, j) at (((i / 8) * nch + j / TC_KC) * 6 + s) * 8 * TC_KC + (i % 8) * TC_KC + j % TC_KC,
// so that the copy of 128 rows x one chunk reads 16 runs of 6 tiles; rows
// and columns past N hold zeros.
__host__ __device__ inline int64_t tc_wsl_index(int s, int64_t i, int64_t j, int64_t nch) {
  return (((i >> 3) * nch + j / TC_KC) * TC_NSL + s) * (8 * TC_KC) + (i & 7) * TC_KC + j % TC_KC;
}
__global__ void tc_slice_w_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl, int64_t ldw, int64_t N,
                                  int64_t nch, int64_t ngroups, const int* __restrict__ ex,
                                  __nv_bfloat16* __restrict__ S) {
  const int64_t cols = nch * TC_KC;
  const int64_t n = ngroups * 8 * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    const double w = (i < N && j < N) ? ldexp(df_to_double(Wh[i * ldw + j], Wl[i * ldw + j]), -ex[i]) : 0.0;
    __nv_bfloat16* d = S + tc_wsl_index(0, i, j, nch);
    tc_digits(w, d, 8 * TC_KC);
  }
}

// column exponents of P (N x kb row-major): f_c as for the rows of W
__global__ void tc_col_exp_kernel(const double* __restrict__ P, int64_t N, int kb, int* __restrict__ fx) {
  __shared__ double sm[256];
  const int c = blockIdx.x;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += 256) m = fmax(m, fabs(P[i * kb + c]));
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int e = 0;
    if (sm[0] > 0.0) frexp(sm[0], &e);
    fx[c] = sm[0] > 0.0 ? e + 1 : 0;
  }
}

// P slices by chunk: element (u, c, j) at ((j / TC_KC * 6 + u) * 16 + c) * TC_KC + j % TC_KC
// (vectors c >= kb and entries j >= N stay zero)
__global__ void tc_slice_p_kernel(const double* __restrict__ P, int64_t N, int kb, const int* __restrict__ fx,
                                  __nv_bfloat16* __restrict__ S) {
  const int64_t n = N * kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / kb;
    const int c = (int)(e - j * kb);
    tc_digits(ldexp(P[e], -fx[c]), S + ((j / TC_KC) * TC_NSL * TC_NV + c) * TC_KC + j % TC_KC, TC_NV * TC_KC);
  }
}

// ---- the product -------------------------------------------------------------
// P slices paired with W slice s (levels s + u <= 8) and the TMEM column where
// its accumulators start: 96 + 96 + 80 + 64 + 48 + 32 = 416 columns
__host__ __device__ constexpr int tc_nu(int s) { return TC_LMAX - s < TC_NSL ? TC_LMAX - s : TC_NSL; }
__host__ __device__ constexpr int tc_off(int s) { return s <= 1 ? 0 : tc_off(s - 1) + TC_NV * tc_nu(s - 1); }
static_assert(tc_off(TC_NSL + 1) <= 512, "accumulators exceed TMEM");
#define TC_TMEM_COLS 512

// 16 consecutive accumulator columns of this warp's 32 lanes; the wait names
// the registers so that no use is scheduled before the data has arrived
__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(addr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :: "memory");
}
__global__ void __launch_bounds__(192, 1) tc_matvec_kernel(const __grid_constant__ CUtensorMap tmW,
                                                           const __grid_constant__ CUtensorMap tmP, int N,
                                                           int nchunks_all, int cps, int kb,
                                                           const int* __restrict__ ex, const int* __restrict__ fx,
                                                           double* __restrict__ split_part,
                                                           const int* __restrict__ stop, int* __restrict__ err) {
  if (*stop) return;
  extern __shared__ unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(base + TC_STAGES * TC_STAGE_BYTES);   // copy landed
  uint64_t* empty = full + TC_STAGES;                                  // its MMAs done
  uint64_t* accfull = empty + TC_STAGES;                               // a window's sums final
  uint64_t* accempty = accfull + 1;                                    // a window's sums read
  uint32_t* tbase = (uint32_t*)(accempty + 1);
  volatile int* s_fail = (volatile int*)(tbase + 1);
  volatile int* s_issued = s_fail + 1;   // chunks whose copy was issued
  volatile int* s_taken = s_fail + 2;    // chunks whose MMAs were issued
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * TC_ROWS;
  const int chunk0 = blockIdx.y * cps;
  const int nchunks = min(nchunks_all - chunk0, cps);
  const int nwin = (nchunks + TC_WIN - 1) / TC_WIN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(tbase)),
                 "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int st = 0; st < TC_STAGES; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&full[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&empty[st])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(accfull)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(tc_smem(accempty)) : "memory");
    *s_fail = 0;
    *s_issued = 0;
    *s_taken = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tbase;

  float acch[TC_NV], accl[TC_NV];
#pragma unroll
  for (int c = 0; c < TC_NV; ++c) { acch[c] = 0.f; accl[c] = 0.f; }

  if (warp == 5) {
    // ---- producer: the copies of chunk t once the MMAs of chunk t - STAGES are done
    if (lane == 0) {
      for (int t = 0; t < nchunks; ++t) {
        const int st = t % TC_STAGES;
        if (t >= TC_STAGES && !tc_wait(&empty[st], (uint32_t)((t / TC_STAGES - 1) & 1), s_fail)) {
          *s_fail = 1;
          break;
        }
        unsigned char* sw = base + st * TC_STAGE_BYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(&full[st])),
                     "r"(TC_STAGE_BYTES) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
            ::"r"(tc_smem(sw)), "l"((uint64_t)&tmW), "r"(0), "r"(0), "r"(0), "r"(chunk0 + t), "r"(row0 >> 3),
            "r"(tc_smem(&full[st])) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            ::"r"(tc_smem(sw + TC_W_BYTES)), "l"((uint64_t)&tmP), "r"(0), "r"(0), "r"(0), "r"(chunk0 + t),
            "r"(tc_smem(&full[st])) : "memory");
        *s_issued = t + 1;
      }
    }
  } else if (warp == 4) {
    // ---- MMA issuer: one MMA per W slice and K step, B = the P slices paired with it
    if (lane == 0) {
      for (int t = 0; t < nchunks; ++t) {
        const int st = t % TC_STAGES;
        const int w = t / TC_WIN;
        const bool first = t % TC_WIN == 0;
        if (!tc_wait(&full[st], (uint32_t)((t / TC_STAGES) & 1), s_fail) ||
            (first && w > 0 && !tc_wait(accempty, (uint32_t)((w - 1) & 1), s_fail))) {
          *s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sw = tc_smem(base + st * TC_STAGE_BYTES);
        const uint32_t sp = sw + TC_W_BYTES;
        for (int k = 0; k < TC_KC / 16; ++k)
#pragma unroll
          for (int sl = 1; sl <= TC_NSL; ++sl) {
            // slice s of the copied tiles: one 8-row group every six tiles
            const uint64_t ad = tc_desc(sw + (uint32_t)((sl - 1) * 8 * TC_ROWB) + 32u * k, TC_NSL * 8 * TC_ROWB);
            const uint64_t bd = tc_desc(sp + 32u * k);
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                   ((uint32_t)(TC_NV * tc_nu(sl) >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
            const uint32_t en = (first && k == 0) ? 0u : 1u;
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(taddr + (uint32_t)tc_off(sl)), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tc_smem(&empty[st])) : "memory");
        if (t % TC_WIN == TC_WIN - 1 || t + 1 == nchunks)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(tc_smem(accfull)) : "memory");
        *s_taken = t + 1;
      }
    }
  } else {
    // ---- warps 0-3 (TMEM lanes 32 warp ..): fold each window into double-float sums
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    for (int w = 0; w < nwin; ++w) {
      if (!tc_wait(accfull, (uint32_t)(w & 1), s_fail)) {
        *s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // level by level: the pair sums (exact integers below 2^23) add exactly
      // in 32-bit integers; the sum v (below 2^26) enters the double-float
      // accumulator as its FP32 rounding plus the (at most 2) that it missed
#pragma unroll
      for (int l = 2; l <= TC_LMAX; ++l) {
        int lv[TC_NV];
#pragma unroll
        for (int c = 0; c < TC_NV; ++c) lv[c] = 0;
#pragma unroll
        for (int sl = 1; sl <= TC_NSL; ++sl) {
          const int u = l - sl;
          if (u < 1 || u > tc_nu(sl)) continue;
          uint32_t r[16];
          tc_ld16(taddr + lanes + (uint32_t)(tc_off(sl) + TC_NV * (u - 1)), r);
#pragma unroll
          for (int c = 0; c < TC_NV; ++c) lv[c] += __float2int_rn(__uint_as_float(r[c]));
        }
        const float sc = ldexpf(1.0f, -8 * l);
#pragma unroll
        for (int c = 0; c < TC_NV; ++c) {
          const float hi = __int2float_rn(lv[c]);
          const int lo = lv[c] - __float2int_rn(hi);   // |lo| <= 2: v is below 2^26
          float sh, e;
          two_sum(acch[c], hi * sc, sh, e);
          acch[c] = sh;
          accl[c] += e + (float)lo * sc;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(accempty)) : "memory");
    }
  }
  __syncthreads();
  const bool ok = *s_fail == 0;
  if (ok) {
    if (warp < 4) {
      const int row = row0 + 32 * warp + lane;
      if (row < N) {
        const int e = ex[row];
#pragma unroll
        for (int c = 0; c < TC_NV; ++c) {
          if (c >= kb) break;
          // scaled in FP64, so that no vector's range is limited by FP32's
          split_part[((int64_t)blockIdx.y * N + row) * kb + c] =
              ldexp((double)acch[c] + (double)accl[c], e + fx[c]);
        }
      }
    }
  } else if (tid == 0) {
    // let the copies and the MMAs still in flight finish (bounded) before the
    // shared memory and the accumulators are given back
    const int taken = *s_taken, issued = *s_issued;
    for (int u = taken; u < issued; ++u)
      tc_wait(&full[u % TC_STAGES], (uint32_t)((u / TC_STAGES) & 1), nullptr);
    if (taken > 0) tc_wait(&empty[(taken - 1) % TC_STAGES], (uint32_t)(((taken - 1) / TC_STAGES) & 1), nullptr);
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS) : "memory");
}

// Q = the sum of the S splits' partials (in split order, FP64) and the
// per-block partial sums of p_c . q_c over blocks of TC_PART_ROWS rows (the
// layout of the double-float product's reduction)
#define TC_PART_ROWS 16
__global__ void __launch_bounds__(256) tc_combine_kernel(const double* __restrict__ split_part, int S, int N, int kb,
                                                         const double* __restrict__ P, double* __restrict__ Q,
                                                         double* __restrict__ part, const int* __restrict__ stop) {
  if (*stop) return;
  __shared__ double sq[TC_PART_ROWS * TC_NV];
  const int64_t row0 = (int64_t)blockIdx.x * TC_PART_ROWS;
  for (int e = threadIdx.x; e < TC_PART_ROWS * kb; e += 256) {
    const int r = e / kb, c = e - r * kb;
    const int64_t row = row0 + r;
    double pq = 0.0;
    if (row < N) {
      double q = 0.0;
      for (int sp = 0; sp < S; ++sp) q += split_part[((int64_t)sp * N + row) * kb + c];
      Q[row * kb + c] = q;
      pq = q * P[row * kb + c];
    }
    sq[e] = pq;
  }
  __syncthreads();
  if (threadIdx.x < kb) {
    double sum = 0.0;
    for (int r = 0; r < TC_PART_ROWS; ++r) sum += sq[r * kb + threadIdx.x];
    part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = sum;
  }
}

// ---- host side ------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// bf16 tensor of `rank` dims (dims[0] innermost), byte strides of dims 1.., one box
static cudaError_t encode_bf16(CUtensorMap* map, const void* base, int rank, const cuuint64_t* dims,
                               const cuuint64_t* strides, const cuuint32_t* box) {
  auto fn = tc_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  TC_ROWB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : TC_ROWB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                  TC_PROMO, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int64_t tc_nch(int64_t N) { return (N + TC_KC - 1) / TC_KC; }
static int64_t tc_ngroups(int64_t N) { return (N + 7) / 8; }
static size_t tc_wsl_elems(int64_t N) { return (size_t)tc_ngroups(N) * 8 * tc_nch(N) * TC_KC * TC_NSL; }
static size_t tc_psl_elems(int64_t N) { return (size_t)tc_nch(N) * TC_NSL * TC_NV * TC_KC; }

size_t tc_slices_bytes(const DevGeom& g) { return tc_wsl_elems(g.ndof) * 2 + sizeof(int) * g.ndof; }

cudaError_t ensure_w_slices(DevGeom& g, cudaStream_t s) {
  if (g.d_wsl || g.ndof == 0) return cudaSuccess;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    static std::vector<int> ready;
    int dev = 0;
    cudaGetDevice(&dev);
    if (std::find(ready.begin(), ready.end(), dev) == ready.end()) {
      cudaError_t e = cudaFuncSetAttribute(tc_matvec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
      if (e != cudaSuccess) return e;
      ready.push_back(dev);
    }
  }
  cudaError_t e = pool_alloc((void**)&g.d_wsl, tc_slices_bytes(g), g.pool, s);
  if (e != cudaSuccess) return e;
  const int64_t N = g.ndof, nch = tc_nch(N), ngr = tc_ngroups(N);
  g.d_wexp = (int*)((char*)g.d_wsl + tc_wsl_elems(N) * 2);
  tc_row_exp_kernel<<<(unsigned)N, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, N, g.d_wexp);
  const int64_t n = ngr * 8 * nch * TC_KC;
  tc_slice_w_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 64), 256, 0, s>>>(
      g.d_Wh, g.wlo(), g.ldw, N, nch, ngr, g.d_wexp, (__nv_bfloat16*)g.d_wsl);
  g.launches += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // (column in chunk, row in group, slice, chunk, row group); boxes of 16 row groups
  const cuuint64_t dims[5] = {TC_KC, 8, TC_NSL, (cuuint64_t)nch, (cuuint64_t)ngr};
  const cuuint64_t strides[4] = {TC_KC * 2, 8 * TC_KC * 2, TC_NSL * 8 * TC_KC * 2,
                                 (cuuint64_t)nch * TC_NSL * 8 * TC_KC * 2};
  const cuuint32_t box[5] = {TC_KC, 8, TC_NSL, 1, TC_ROWS / 8};
  return encode_bf16(&g.tm_wsl, g.d_wsl, 5, dims, strides, box);
}

// Column splits for order N (a function of N only, so that a vector's product
// never depends on the batch): the count that fills the last wave of
// (row block x split) CTAs best, one CTA per SM on 152 SMs, with a slight
// preference for fewer splits; every split keeps at least two fold windows.
static int tc_split(int64_t N) {
  const int64_t nchunks = (N + TC_KC - 1) / TC_KC;
  const int64_t blocks = (N + TC_ROWS - 1) / TC_ROWS;
  const int64_t smax = std::min<int64_t>(64, std::max<int64_t>(1, nchunks / (2 * TC_WIN)));
  int best = 1;
  double bestv = -1.0;
  for (int64_t S = 1; S <= smax; ++S) {
    const int64_t per = (nchunks + S - 1) / S;
    if ((S - 1) * per >= nchunks) continue;   // a split without columns
    const int64_t items = blocks * S;
    const double eff = (double)items / (double)(((items + 151) / 152) * 152);
    const double v = eff - 0.004 * (double)S;
    if (v > bestv + 1e-12) {
      bestv = v;
      best = (int)S;
    }
  }
  return best;
}

size_t tc_work_bytes(const DevGeom& g) {
  return tc_psl_elems(g.ndof) * 2 + sizeof(double) * (size_t)tc_split(g.ndof) * g.ndof * TC_NV + 1024;
}

void drop_w_slices(DevGeom& g, cudaStream_t s) {
  if (g.d_wsl) cudaFreeAsync(g.d_wsl, s);
  g.d_wsl = nullptr;
  g.d_wexp = nullptr;
}

// Q (N x kb) and the partial sums of p.q (layout of launch_matvec) from P
// (N x kb, row-major double); work: tc_work_bytes(g) of scratch.
cudaError_t launch_matvec_tc(DevGeom& g, int kb, const double* P, double* Q, double* part, const int* stop, int* err,
                             void* work, cudaStream_t s) {
  const int64_t N = g.ndof;
  if (N <= 0 || kb < 1 || kb > TC_NV || !g.d_wsl) return cudaErrorInvalidValue;
  const int split = tc_split(N);
  char* cur = (char*)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  __nv_bfloat16* ps = (__nv_bfloat16*)cur;
  const size_t pbytes = tc_psl_elems(N) * 2;
  cur += (pbytes + 255) / 256 * 256;
  int* fx = (int*)cur;
  cur += 256;
  double* sp = (double*)cur;
  CUtensorMap tmP;
  // (column in chunk, vector, slice, chunk); one chunk per box
  const cuuint64_t dims[4] = {TC_KC, TC_NV, TC_NSL, (cuuint64_t)tc_nch(N)};
  const cuuint64_t strides[3] = {TC_KC * 2, TC_NV * TC_KC * 2, TC_NSL * TC_NV * TC_KC * 2};
  const cuuint32_t box[4] = {TC_KC, TC_NV, TC_NSL, 1};
  cudaError_t e = encode_bf16(&tmP, ps, 4, dims, strides, box);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(ps, 0, pbytes, s);
  cudaMemsetAsync(fx, 0, sizeof(int) * TC_NV, s);
  tc_col_exp_kernel<<<kb, 256, 0, s>>>(P, N, kb, fx);
  tc_slice_p_kernel<<<(unsigned)std::min<int64_t>((N * kb + 255) / 256, 152 * 16), 256, 0, s>>>(P, N, kb, fx, ps);
  const int nchunks = (int)((N + TC_KC - 1) / TC_KC);
  const int cps = (nchunks + split - 1) / split;
  const int nsplit = (nchunks + cps - 1) / cps;
  const dim3 grid((unsigned)((N + TC_ROWS - 1) / TC_ROWS), (unsigned)nsplit);
  tc_matvec_kernel<<<grid, 192, TC_SMEM, s>>>(g.tm_wsl, tmP, (int)N, nchunks, cps, kb, g.d_wexp, fx, sp, stop, err);
  g.launches += 4;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the reduction blocks must match those of the double-float product
  static_assert(TC_PART_ROWS == 16, "blocks of the p.q partial sums");
  tc_combine_kernel<<<(unsigned)((N + TC_PART_ROWS - 1) / TC_PART_ROWS), 256, 0, s>>>(sp, nsplit, (int)N, kb, P, Q,
                                                                                      part, stop);
  return cudaGetLastError();
}

}  // namespace msbem
