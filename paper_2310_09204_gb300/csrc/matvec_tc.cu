// Q = W P on the tensor cores (tcgen05) for up to 16 vectors, from integer
// slices of both operands: double-float accuracy, or a scaled-FP16 product
// for the inner solves of the iterative refinement.
//
// Every row i of W is scaled by 2^-e_i so that its entries lie in (-1/2, 1/2)
// and written in base 2^B as W_ij = 2^e_i sum_s a_s[i,j] 2^-Bs (+ remainder),
// each digit rounded to nearest so that |a_s| <= 2^(B-1): an integer that the
// MMA's 16-bit type holds exactly.  The vectors P are sliced the same way per
// column (exponent f_c, digits b_t).  Then
//
//   (W P)_ic = 2^(e_i + f_c) sum_l 2^-Bl sum_{s+t=l} sum_j a_s[i,j] b_t[j,c],
//
// and every inner sum over j is a product of integer matrices that the tensor
// core forms with FP32 accumulation.
//
// * Double-float (TcDF): B = 8, six slices of W and of P in bf16, the slice
//   pairs with s + t <= 8.  Products are below 2^14, so the pair sums of a
//   window of 512 columns stay below 2^23 and are exact; they are folded from
//   TMEM into double-float registers before the next window starts.  The
//   levels left out and the remainders (2^-49 of the scales) keep the error
//   below 2^-44 max_j |W_ij| sum_j |P_jc|.
// * Scaled FP16 (TcF16): no digits but floating-point fp16 values: W_ij 2^(14-e_i)
//   rounded to fp16 (2 bytes an entry; each entry to 2^-11 of itself, its
//   own exponent within fp16's range below the row's largest entry), and the
//   vectors as P_jc 2^(14-f_c) = hi + lo, two fp16 values; the two products
//   accumulate in FP32 and (W P)_ic = 2^(e_i + f_c - 28) (W P_hi + W P_lo)_ic.
//
// The slices of W are kept in a blocked layout: tiles of 8 rows x 64 columns
// (128-byte rows), the slices of a tile side by side, tiles by column chunk
// within a row group, so that one copy of 128 rows x 64 columns reads 16
// contiguous runs.  One CTA: 128 rows (M = 128), the vectors padded to 16, a
// range of 64-column chunks.  Warp 5 issues the TMA copies (W slices with a
// 128-byte swizzle, P slices side by side) into a ring of stages, warp 4
// issues one MMA per W slice and K step with B = all the P slices paired with
// it (N = 16 x their count), and warps 0-3 fold the accumulators every 512
// columns.  Waits are bounded; TMEM is always freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define TC_ROWB 128           // bytes of a chunk row (the 128-byte swizzle span)
#define TC_KC 64              // columns per chunk
#define TC_WIN (512 / TC_KC)  // chunks per fold window (512 columns)
#define TC_ROWS 128
#define TC_NV 16              // vectors (16 columns per slice in the MMA's N)
#define TC_NSTORE 6           // bf16 slices stored per entry of W
#define TC_SMEM_RING (216 * 1024)

// a slicing of the product: W slices read, P slices, highest level kept,
// digit bits (0: floating-point fp16 values scaled by 2^14 instead of
// integer digits), fp16 (else bf16) operands
template <int NW_, int NP_, int LMAX_, int BITS_, bool F16_>
struct TcCfg {
  static constexpr int NW = NW_, NP = NP_, LMAX = LMAX_, BITS = BITS_;
  static constexpr bool F16 = F16_;
  static constexpr bool FLOATING = BITS_ == 0;
  static constexpr int FSHIFT = 14;   // the floating values' scale 2^14 (per operand)
  static constexpr int STAGE_W = NW * TC_ROWS * TC_ROWB;
  static constexpr int STAGE_P = NP * TC_NV * TC_ROWB;
  static constexpr int STAGE = STAGE_W + STAGE_P;
  static constexpr int STAGES = TC_SMEM_RING / STAGE < 8 ? TC_SMEM_RING / STAGE : 8;
  static constexpr int SMEM = 1024 + STAGES * STAGE + 256;   // + barriers and flags (< 256 B)
  // P slices paired with W slice s, and the TMEM column where its pair sums start
  __host__ __device__ static constexpr int nu(int s) { return LMAX - s < NP ? LMAX - s : NP; }
  __host__ __device__ static constexpr int off(int s) { return s <= 1 ? 0 : off(s - 1) + TC_NV * nu(s - 1); }
  static constexpr int COLS = off(NW + 1);
  static constexpr int TMEM = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static_assert(COLS <= 512, "accumulators exceed TMEM");
  static_assert(STAGES >= 2, "ring too shallow");
};
using TcDF = TcCfg<6, 6, 8, 8, false>;     // 96 + 96 + 80 + 64 + 48 + 32 = 416 columns
using TcF16 = TcCfg<1, 2, 3, 0, true>;     // 32 columns: W P_hi, W P_lo

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
// Test hook of the error path (msbem_test_expire_waits): when non-zero, the
// producer of every CTA first waits up to this many nanoseconds for
// g_tc_never, a flag that nothing sets, and on expiry gives up before its first
// copy, as if a copy had never completed.  Zero in normal use.
__device__ long long g_tc_expire_ns = 0;
__device__ int g_tc_never = 0;

__device__ __noinline__ bool tc_wait_never(long long limit_ns) {
  const uint64_t t0 = tc_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (*(volatile int*)&g_tc_never) return true;
    if (tc_ns() - t0 > (uint64_t)limit_ns) return false;
  }
  return false;
}

// shared-memory matrix descriptor: K-major, 128-byte rows under the 128-byte
// swizzle (layout 2), 8-row groups group_stride bytes apart
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t group_stride) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(group_stride >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// ---- slicing ---------------------------------------------------------------
// e_i with |W_ij| < 2^(e_i - 1) for every j (0 for a zero row), from the hi
// plane: max |hi| in [2^(k-1), 2^k) gives e_i = k + 1, and |hi + lo| <=
// |hi| (1 + 2^-24) stays below 2^k
__global__ void tc_row_exp_kernel(const float* __restrict__ Wh, int64_t ldw, int64_t N, int* __restrict__ ex) {
  __shared__ float sm[256];
  const int64_t i = blockIdx.x;
  float m = 0.f;
  for (int64_t j = threadIdx.x; j < N; j += 256) m = fmaxf(m, fabsf(Wh[i * ldw + j]));
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int k = 0;
    if (sm[0] > 0.f) frexpf(sm[0], &k);   // max in [2^(k-1), 2^k)
    ex[i] = sm[0] > 0.f ? k + 1 : 0;
  }
}

// n balanced digits of x in (-1/2, 1/2) in base 2^bits (n * bits <= 56):
// X = x 2^(n bits) rounded to the nearest integer (exact in 64 bits), then
// X = sum_s d_s 2^(bits (n - s)), d_s in [-2^(bits-1), 2^(bits-1)) taken
// from the least significant end (|d_1| <= 2^(bits-1) as |x| < 1/2); so
// x = sum_s d_s 2^-(bits s) + r, |r| <= 2^-(n bits + 1)
__device__ __forceinline__ void tc_digits(double x, int n, int bits, __nv_bfloat16* d, int64_t stride) {
  long long X = __double2ll_rn(ldexp(x, n * bits));
  const long long half = 1ll << (bits - 1), mask = (1ll << bits) - 1;
  for (int s = n - 1; s >= 0; --s) {
    const long long dig = s == 0 ? X : ((X + half) & mask) - half;
    d[s * stride] = __float2bfloat16((float)dig);
    X = (X - dig) >> bits;
  }
}

// x 2^shift (x in (-1/2, 1/2)) as n fp16 values: x 2^shift = d_0 + d_1 + ...,
// each the fp16 rounding of what the previous left
__device__ __forceinline__ void tc_fp16_split(double x, int n, int shift, __half* d, int64_t stride) {
  x = ldexp(x, shift);
  for (int s = 0; s < n; ++s) {
    const __half h = __double2half(x);
    d[s * stride] = h;
    x -= (double)__half2float(h);
  }
}

// Blocked layout of nsl slices of W: element (s, i, j) at
//   (((i / 8) * nch + j / 64) * nsl + s) * 512 + (i % 8) * 64 + j % 64;
// rows and columns past N hold zeros.
__host__ __device__ inline int64_t tc_wsl_index(int s, int64_t i, int64_t j, int64_t nch, int nsl) {
  return (((i >> 3) * nch + j / TC_KC) * nsl + s) * (8 * TC_KC) + (i & 7) * TC_KC + j % TC_KC;
}
template <typename T>
__global__ void tc_slice_w_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl, int64_t ldw, int64_t N,
                                  int64_t nch, int64_t ngroups, int nsl, int bits, const int* __restrict__ ex,
                                  T* __restrict__ S) {
  const int64_t cols = nch * TC_KC;
  const int64_t n = ngroups * 8 * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    const double w = (i < N && j < N) ? ldexp(df_to_double(Wh[i * ldw + j], Wl[i * ldw + j]), -ex[i]) : 0.0;
    if constexpr (std::is_same<T, __half>::value)
      tc_fp16_split(w, nsl, bits, S + tc_wsl_index(0, i, j, nch, nsl), 8 * TC_KC);   // bits: the shift
    else
      tc_digits(w, nsl, bits, S + tc_wsl_index(0, i, j, nch, nsl), 8 * TC_KC);
  }
}

// column maxima of |P| (N x kb row-major): per-block maxima combined by an
// atomic maximum on their bit patterns (the order of non-negative doubles)
__global__ void tc_col_max_kernel(const double* __restrict__ P, int64_t N, int kb,
                                  unsigned long long* __restrict__ mx) {
  __shared__ unsigned long long sm[256];
  const int64_t n = N * kb;
  unsigned long long m = 0;
  // a stride that is a multiple of kb keeps each thread on one column
  const int64_t stride = (int64_t)gridDim.x * 256 / kb * kb;
  const int64_t start = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (start < stride)
    for (int64_t e = start; e < n; e += stride) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(P[e]));
      m = b > m ? b : m;
    }
  sm[threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.x < kb) {
    // column c gathers the threads t with (block offset + t) = c mod kb
    const int shift = (int)(((int64_t)blockIdx.x * 256) % kb);
    unsigned long long r = 0;
    for (int t = 0; t < 256; ++t)
      if ((shift + t) % kb == (int)threadIdx.x) r = sm[t] > r ? sm[t] : r;
    atomicMax(&mx[threadIdx.x], r);
  }
}

// P slices by chunk: element (u, c, j) at ((j / 64 * np + u) * 16 + c) * 64 + j % 64
// (vectors c >= kb and entries j >= N stay zero); column exponents f_c from
// the maxima as for the rows of W
template <typename T>
__global__ void tc_slice_p_kernel(const double* __restrict__ P, int64_t N, int kb, int np, int bits,
                                  const unsigned long long* __restrict__ mx, int* __restrict__ fx,
                                  T* __restrict__ S) {
  const int64_t n = N * kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / kb;
    const int c = (int)(e - j * kb);
    const double m = __longlong_as_double((long long)mx[c]);
    int f = 0;
    if (m > 0.0) frexp(m, &f);
    f = m > 0.0 ? f + 1 : 0;
    if (j == 0) fx[c] = f;
    T* d = S + ((j / TC_KC) * np * TC_NV + c) * TC_KC + j % TC_KC;
    if constexpr (std::is_same<T, __half>::value)
      tc_fp16_split(ldexp(P[e], -f), np, bits, d, TC_NV * TC_KC);   // bits: the shift
    else
      tc_digits(ldexp(P[e], -f), np, bits, d, TC_NV * TC_KC);
  }
}

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

// ---- the product -------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(192, 1) tc_matvec_kernel(const __grid_constant__ CUtensorMap tmW,
                                                           const __grid_constant__ CUtensorMap tmP, int N,
                                                           int nchunks_all, int cps, int kb,
                                                           const int* __restrict__ ex, const int* __restrict__ fx,
                                                           double* __restrict__ split_part,
                                                           const int* __restrict__ stop, int* __restrict__ err) {
  constexpr int ST = C::STAGES;
  if (*stop) return;
  extern __shared__ unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(base + ST * C::STAGE);   // copy landed
  uint64_t* empty = full + ST;                          // its MMAs done
  uint64_t* accfull = empty + ST;                       // a window's sums final
  uint64_t* accempty = accfull + 1;                     // a window's sums read
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
                 "r"(C::TMEM) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int st = 0; st < ST; ++st) {
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
    // ---- producer: the copies of chunk t once the MMAs of chunk t - ST are done
    if (lane == 0) {
      const long long expire = g_tc_expire_ns;
      if (expire > 0 && !tc_wait_never(expire)) *s_fail = 1;
      for (int t = 0; *s_fail == 0 && t < nchunks; ++t) {
        const int st = t % ST;
        if (t >= ST && !tc_wait(&empty[st], (uint32_t)((t / ST - 1) & 1), s_fail)) {
          *s_fail = 1;
          break;
        }
        unsigned char* sw = base + st * C::STAGE;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(&full[st])),
                     "r"(C::STAGE) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
            ::"r"(tc_smem(sw)), "l"((uint64_t)&tmW), "r"(0), "r"(0), "r"(0), "r"(chunk0 + t), "r"(row0 >> 3),
            "r"(tc_smem(&full[st])) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            ::"r"(tc_smem(sw + C::STAGE_W)), "l"((uint64_t)&tmP), "r"(0), "r"(0), "r"(0), "r"(chunk0 + t),
            "r"(tc_smem(&full[st])) : "memory");
        *s_issued = t + 1;
      }
    }
  } else if (warp == 4) {
    // ---- MMA issuer: one MMA per W slice and K step, B = the P slices paired with it
    if (lane == 0) {
      for (int t = 0; t < nchunks; ++t) {
        const int st = t % ST;
        const int w = t / TC_WIN;
        const bool first = t % TC_WIN == 0;
        if (!tc_wait(&full[st], (uint32_t)((t / ST) & 1), s_fail) ||
            (first && w > 0 && !tc_wait(accempty, (uint32_t)((w - 1) & 1), s_fail))) {
          *s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sw = tc_smem(base + st * C::STAGE);
        const uint32_t sp = sw + C::STAGE_W;
        for (int k = 0; k < TC_KC / 16; ++k)
#pragma unroll
          for (int sl = 1; sl <= C::NW; ++sl) {
            // slice s of the copied tiles: one 8-row group every NW tiles
            const uint64_t ad = tc_desc(sw + (uint32_t)((sl - 1) * 8 * TC_ROWB) + 32u * k, C::NW * 8 * TC_ROWB);
            const uint64_t bd = tc_desc(sp + 32u * k, 8 * TC_ROWB);
            const uint32_t ty = C::F16 ? 0u : 1u;   // operand type: 0 fp16, 1 bf16 (A and B alike)
            const uint32_t idesc = (1u << 4) | (ty << 7) | (ty << 10) | ((uint32_t)(TC_NV * C::nu(sl) >> 3) << 17) |
                                   ((uint32_t)(TC_ROWS >> 4) << 24);
            const uint32_t en = (first && k == 0) ? 0u : 1u;
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(taddr + (uint32_t)C::off(sl)), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
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
      if constexpr (C::FLOATING) {
        // floating values at one scale: the sums W P_u add into the double-float sums
#pragma unroll
        for (int u = 1; u <= C::NP; ++u) {
          uint32_t r[16];
          tc_ld16(taddr + lanes + (uint32_t)(TC_NV * (u - 1)), r);
#pragma unroll
          for (int c = 0; c < TC_NV; ++c) {
            float sh, e;
            two_sum(acch[c], __uint_as_float(r[c]), sh, e);
            acch[c] = sh;
            accl[c] += e;
          }
        }
      }
      // level by level: the pair sums (integers below 2^30) add exactly in
      // 32-bit integers; the sum v enters the double-float accumulator as its
      // FP32 rounding plus what that missed
#pragma unroll
      for (int l = 2; l <= (C::FLOATING ? 1 : C::LMAX); ++l) {
        int lv[TC_NV];
#pragma unroll
        for (int c = 0; c < TC_NV; ++c) lv[c] = 0;
#pragma unroll
        for (int sl = 1; sl <= C::NW; ++sl) {
          const int u = l - sl;
          if (u < 1 || u > C::nu(sl)) continue;
          uint32_t r[16];
          tc_ld16(taddr + lanes + (uint32_t)(C::off(sl) + TC_NV * (u - 1)), r);
#pragma unroll
          for (int c = 0; c < TC_NV; ++c) lv[c] += __float2int_rn(__uint_as_float(r[c]));
        }
        const float sc = ldexpf(1.0f, -C::BITS * l);
#pragma unroll
        for (int c = 0; c < TC_NV; ++c) {
          const float hi = __int2float_rn(lv[c]);
          const int lo = lv[c] - __float2int_rn(hi);
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
              ldexp((double)acch[c] + (double)accl[c], e + fx[c] - (C::FLOATING ? 2 * C::FSHIFT : 0));
        }
      }
    }
  } else if (tid == 0) {
    // let the copies and the MMAs still in flight finish (bounded) before the
    // shared memory and the accumulators are given back
    const int taken = *s_taken, issued = *s_issued;
    for (int u = taken; u < issued; ++u) tc_wait(&full[u % ST], (uint32_t)((u / ST) & 1), nullptr);
    if (taken > 0) tc_wait(&empty[(taken - 1) % ST], (uint32_t)(((taken - 1) / ST) & 1), nullptr);
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(C::TMEM) : "memory");
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
cudaError_t set_matvec_tc_expire_ns(long long ns) {
  return cudaMemcpyToSymbol(g_tc_expire_ns, &ns, sizeof(ns));
}

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

// 16-bit tensor of `rank` dims (dims[0] innermost), byte strides of dims 1.., one box
static cudaError_t encode16(CUtensorMap* map, bool f16, const void* base, int rank, const cuuint64_t* dims,
                            const cuuint64_t* strides, const cuuint32_t* box) {
  auto fn = tc_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, (void*)base,
                  dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int64_t tc_nch(int64_t N) { return (N + TC_KC - 1) / TC_KC; }
static int64_t tc_ngroups(int64_t N) { return (N + 7) / 8; }
static size_t tc_wsl_elems(int64_t N, int nsl) { return (size_t)tc_ngroups(N) * 8 * tc_nch(N) * TC_KC * nsl; }
static size_t tc_psl_elems(int64_t N, int np) { return (size_t)tc_nch(N) * np * TC_NV * TC_KC; }

// W slices, nsl stored per tile; boxes of the first nw of them x 16 row groups
static cudaError_t encode_w_slices(CUtensorMap* map, bool f16, const void* base, int64_t N, int nsl, int nw) {
  const int64_t nch = tc_nch(N), ngr = tc_ngroups(N);
  // (column in chunk, row in group, slice, chunk, row group)
  const cuuint64_t dims[5] = {TC_KC, 8, (cuuint64_t)nsl, (cuuint64_t)nch, (cuuint64_t)ngr};
  const cuuint64_t strides[4] = {TC_ROWB, 8 * TC_ROWB, (cuuint64_t)nsl * 8 * TC_ROWB,
                                 (cuuint64_t)nch * nsl * 8 * TC_ROWB};
  const cuuint32_t box[5] = {TC_KC, 8, (cuuint32_t)nw, 1, TC_ROWS / 8};
  return encode16(map, f16, base, 5, dims, strides, box);
}

template <class C>
static cudaError_t tc_set_attr() {
  return cudaFuncSetAttribute(tc_matvec_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
}

// per device, once: the shared memory of both products (outside any capture)
static cudaError_t tc_init_device() {
  static std::mutex mu;
  static std::vector<int> ready;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (std::find(ready.begin(), ready.end(), dev) != ready.end()) return cudaSuccess;
  cudaError_t e = tc_set_attr<TcDF>();
  if (e == cudaSuccess) e = tc_set_attr<TcF16>();
  if (e == cudaSuccess) ready.push_back(dev);
  return e;
}

size_t tc_slices_bytes(const DevGeom& g, int prec) {
  return (prec == 0 ? tc_wsl_elems(g.ndof, TC_NSTORE) : tc_wsl_elems(g.ndof, 1)) * 2 + sizeof(int) * g.ndof;
}

// the row exponents (shared by both slicings) and the slices of one precision
cudaError_t ensure_w_slices(DevGeom& g, int prec, cudaStream_t s) {
  if (g.ndof == 0) return cudaSuccess;
  if ((prec == 0 && g.d_wsl) || (prec == 1 && g.d_wf16)) return cudaSuccess;
  cudaError_t e = tc_init_device();
  if (e != cudaSuccess) return e;
  const int64_t N = g.ndof, nch = tc_nch(N), ngr = tc_ngroups(N);
  const int64_t n = ngr * 8 * nch * TC_KC;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 64);
  if (!g.d_wexp) {
    if ((e = pool_alloc((void**)&g.d_wexp, sizeof(int) * N, g.pool, s)) != cudaSuccess) return e;
    tc_row_exp_kernel<<<(unsigned)N, 256, 0, s>>>(g.d_Wh, g.ldw, N, g.d_wexp);
    ++g.launches;
  }
  if (prec == 0) {
    if ((e = pool_alloc((void**)&g.d_wsl, tc_wsl_elems(N, TC_NSTORE) * 2, g.pool, s)) != cudaSuccess) return e;
    tc_slice_w_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, N, nch, ngr, TC_NSTORE,
                                                            TcDF::BITS, g.d_wexp, (__nv_bfloat16*)g.d_wsl);
    ++g.launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return encode_w_slices(&g.tm_wsl, false, g.d_wsl, N, TC_NSTORE, TcDF::NW);
  }
  if ((e = pool_alloc((void**)&g.d_wf16, tc_wsl_elems(N, 1) * 2, g.pool, s)) != cudaSuccess) return e;
  tc_slice_w_kernel<__half><<<blocks, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, N, nch, ngr, 1, TcF16::FSHIFT,
                                                   g.d_wexp, (__half*)g.d_wf16);
  ++g.launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return encode_w_slices(&g.tm_wf16, true, g.d_wf16, N, 1, 1);
}

void drop_w_slices(DevGeom& g, cudaStream_t s) {
  for (void* p : {(void*)g.d_wsl, (void*)g.d_wf16, (void*)g.d_wexp})
    if (p) cudaFreeAsync(p, s);
  g.d_wsl = nullptr;
  g.d_wf16 = nullptr;
  g.d_wexp = nullptr;
}

// Column splits for order N (a function of N only, so that a vector's product
// never depends on the batch): the count that fills the last wave of
// (row block x split) CTAs best, one CTA per SM on 152 SMs, with a slight
// preference for fewer splits; every split keeps at least two fold windows.
static int tc_split(int64_t N) {
  const int64_t nchunks = tc_nch(N);
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
  return tc_psl_elems(g.ndof, TcDF::NP) * 2 + sizeof(double) * (size_t)tc_split(g.ndof) * g.ndof * TC_NV + 1024;
}

template <class C>
static cudaError_t launch_cfg(DevGeom& g, const CUtensorMap& tmW, int kb, const double* P, double* Q, double* part,
                              const int* stop, int* err, void* work, cudaStream_t s) {
  const int64_t N = g.ndof;
  const int split = tc_split(N);
  char* cur = (char*)(((uintptr_t)work + 255) & ~(uintptr_t)255);
  void* ps = cur;
  const size_t pbytes = tc_psl_elems(N, C::NP) * 2;
  cur += (pbytes + 255) / 256 * 256;
  unsigned long long* mx = (unsigned long long*)cur;   // 16 maxima, then 16 exponents
  int* fx = (int*)(cur + 128);
  cur += 256;
  double* sp = (double*)cur;
  CUtensorMap tmP;
  // (column in chunk, vector, slice, chunk); one chunk per box
  const cuuint64_t dims[4] = {TC_KC, TC_NV, (cuuint64_t)C::NP, (cuuint64_t)tc_nch(N)};
  const cuuint64_t strides[3] = {TC_ROWB, TC_NV * TC_ROWB, (cuuint64_t)C::NP * TC_NV * TC_ROWB};
  const cuuint32_t box[4] = {TC_KC, TC_NV, (cuuint32_t)C::NP, 1};
  cudaError_t e = encode16(&tmP, C::F16, ps, 4, dims, strides, box);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(ps, 0, pbytes, s);
  cudaMemsetAsync(mx, 0, 256, s);
  const unsigned pblocks = (unsigned)std::min<int64_t>((N * kb + 255) / 256, 152 * 16);
  tc_col_max_kernel<<<(unsigned)std::min<int64_t>((N * kb + 255) / 256, 152), 256, 0, s>>>(P, N, kb, mx);
  if constexpr (C::F16)
    tc_slice_p_kernel<__half><<<pblocks, 256, 0, s>>>(P, N, kb, C::NP, C::FSHIFT, mx, fx, (__half*)ps);
  else
    tc_slice_p_kernel<__nv_bfloat16><<<pblocks, 256, 0, s>>>(P, N, kb, C::NP, C::BITS, mx, fx, (__nv_bfloat16*)ps);
  const int nchunks = (int)tc_nch(N);
  const int cps = (nchunks + split - 1) / split;
  const int nsplit = (nchunks + cps - 1) / cps;
  const dim3 grid((unsigned)((N + TC_ROWS - 1) / TC_ROWS), (unsigned)nsplit);
  tc_matvec_kernel<C><<<grid, 192, C::SMEM, s>>>(tmW, tmP, (int)N, nchunks, cps, kb, g.d_wexp, fx, sp, stop, err);
  static_assert(TC_PART_ROWS == 16, "blocks of the p.q partial sums");
  tc_combine_kernel<<<(unsigned)((N + TC_PART_ROWS - 1) / TC_PART_ROWS), 256, 0, s>>>(sp, nsplit, (int)N, kb, P, Q,
                                                                                      part, stop);
  g.launches += 4;
  return cudaGetLastError();
}

// Q (N x kb) and the partial sums of p.q (layout of launch_matvec) from P
// (N x kb, row-major double); prec 0 double-float, 1 scaled FP16; work:
// tc_work_bytes(g) of scratch; the slices of that precision must exist.
cudaError_t launch_matvec_tc(DevGeom& g, int prec, int kb, const double* P, double* Q, double* part,
                             const int* stop, int* err, void* work, cudaStream_t s) {
  const int64_t N = g.ndof;
  if (N <= 0 || N > 0x7fffffff || kb < 1 || kb > TC_NV || !g.d_wexp) return cudaErrorInvalidValue;
  if (prec == 0) {
    if (!g.d_wsl) return cudaErrorInvalidValue;
    return launch_cfg<TcDF>(g, g.tm_wsl, kb, P, Q, part, stop, err, work, s);
  }
  if (!g.d_wf16) return cudaErrorInvalidValue;
  return launch_cfg<TcF16>(g, g.tm_wf16, kb, P, Q, part, stop, err, work, s);
}

}  // namespace msbem
