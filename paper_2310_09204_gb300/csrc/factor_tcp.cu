// The rank-32 update of the double-float blocked Gauss-Jordan set-up (Sec.
// 5, eq. jumpSplit: the face, wire-basket and coarse blocks of M(H;h)
// inverted explicitly) on the tcgen05 tensor cores, as one persistent kernel
// per step.
//
// One step updates every entry of an active matrix from the left operand L
// (row r: the scaled pivot row P[r - k0] for the 32 pivot rows K, else the
// panel row C'_r) and the right operand R (the old pivot rows A[K][c]):
//   A[r][c] = L(r)[c - k0]                          for c in K,
//   A[r][c] = [r not in K] A[r][c] + L(r) . R[:, c]   otherwise.
// The product L R is formed exactly in integers: each row of L is scaled by a
// power of two 2^-e_r into (-1/2, 1/2), rounded to 48 bits and cut into six
// balanced base-256 digits (each exact in bf16); each column of R likewise
// with 2^-f_c.  Then (L R)[r][c] = 2^(e_r + f_c) sum_l 2^(-8(l+2)) Q_l[r][c]
// with Q_l = sum_{s+t=l} a_s b_t, a product of integer matrices that a
// kind::f16 MMA (bf16 operands, FP32 accumulators in tensor memory) forms
// exactly (K = 32 terms of at most 2^14, at most 6 slice pairs per level:
// below 2^22).  Levels 0 .. 6 are kept (26 slice pairs; what is left out lies
// below 2^-51 of the operands' scales), each in its own accumulator, and
// folded into double-float sums.
//
// Per step, two slicing kernels write the digits of every row of L (tiles of
// 128 rows) and every column of R (tiles of 32 columns) in the tensor cores'
// shared-memory order (128-byte rows under the 128-byte swizzle; K positions
// 0 .. 31).  Then one persistent kernel, one CTA per SM, takes a contiguous
// range of 128 x 32 output tiles (row-major in each matrix, so consecutive
// tiles share their left digits) with its warps specialised:
//   warp 0  (one lane) brings in the digit tiles by bulk asynchronous copies:
//           the right digits of each tile into one of two stages, the left
//           digits only when the row tile changes;
//   warp 1  owns the tensor memory (two accumulator sets of 7 x 32 columns)
//           and issues each tile's 52 MMAs from one lane;
//   warps 2 .. 17 (one tile row per thread, 8 columns each) read their old
//           entries of A, fold the level accumulators of the tile and store
//           the updated entries back.
// Copies, MMAs and the epilogue of neighbouring tiles overlap.  Every wait is
// bounded (an error flag, the work in flight drained, the tensor memory
// freed).
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

namespace {

constexpr int KG = 32;            // pivot panel width of the recursion
constexpr int TR = 128;           // rows of an output tile (TMEM lanes)
constexpr int DROW = 128;         // bytes of one digit row (64 K positions; 0 .. 31 used)
constexpr int LBLK = TR * DROW;   // bytes of one left digit tile
constexpr int NEPI = 16;          // epilogue warps (four per TMEM lane quarter)
constexpr int NTHREADS = 32 * (2 + NEPI);

// double-float set-up: FP64 matrices, float-pair operands; levels 0 .. 6 in
// seven exact accumulators
struct CfgDF {
  static constexpr int ND = 6, LEVELS = 7, TN = 32;
  using Elem = double;
  using Op = float2;
};
template <class Cfg>
struct Lay {
  static constexpr int RBLK = Cfg::TN * DROW;                     // one right digit tile
  static constexpr int LB = Cfg::ND * LBLK;                       // left digits of a row tile
  static constexpr int RB = Cfg::ND * RBLK;                       // right digits of a tile
  static constexpr int OFF_R = LB;                                // two right stages
  static constexpr int OFF_BAR = LB + 2 * RB;
  static constexpr int SMEM = 1024 + OFF_BAR + 128;
  static constexpr int TCOLS = Cfg::LEVELS * Cfg::TN;             // accumulator columns of one set
  static_assert(2 * TCOLS <= 512, "two accumulator sets fit in tensor memory");
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

template <class Elem>
__host__ __device__ __forceinline__ int64_t tcp_ld(int64_t n) {
  return sizeof(Elem) == 4 ? ((n + 3) & ~(int64_t)3) : n;   // FP32 rows padded to 16 bytes
}

__device__ __forceinline__ double tcp_value(float2 v) { return widen(v.x) + widen(v.y); }
__device__ __forceinline__ float tcp_hi(float2 v) { return v.x; }

__device__ __forceinline__ int tcp_find(const int64_t* pre, int active, int64_t t) {
  int lo = 0, hi = active - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// e with |x| < 2^(e-1) for every x of a row whose largest |hi| is m
// (0 for a zero row, whose digits are all zero)
__device__ __forceinline__ int tcp_exp(float m) {
  if (!(m > 0.f)) return 0;
  int k = 0;
  frexpf(m, &k);   // m in [2^(k-1), 2^k)
  return k + 1;
}

// the ND balanced base-256 digits of x (|x| < 1/2): x = sum_i d[i] 2^(-8(i+1))
// + r with |r| <= 2^-(8 ND + 1), d[0] the most significant (|d[0]| <= 128)
template <int ND>
__device__ __forceinline__ void tcp_digits(double x, int* d) {
  long long v = llrint(ldexp(x, 8 * ND));
#pragma unroll
  for (int i = ND - 1; i >= 1; --i) {
    const long long r = ((v + 128) & 255) - 128;   // in [-128, 127]
    d[i] = (int)r;
    v = (v - r) >> 8;                               // exact: v - r is a multiple of 256
  }
  d[0] = (int)v;
}
// Chunk j (K positions 8j .. 8j+7, j < 4) of one row (left) or column (right)
// of an operand: its K = 32 values (kb of them used, the rest zero), scaled by
// the exponent of the whole row, as ND 16-byte digit chunks in the swizzled
// order of row `row` of tiles digit_stride bytes apart.  K positions 32 .. 63
// of a digit row are never read by the MMAs and are not written.
template <class Cfg>
__device__ __forceinline__ int tcp_slice_chunk(const typename Cfg::Op* v, int64_t vstride, int kb,
                                               unsigned char* base, size_t digit_stride, int row, int j) {
  constexpr int ND = Cfg::ND;
  float m = 0.f;
  for (int k = 0; k < kb; ++k) m = fmaxf(m, fabsf(tcp_hi(v[k * vstride])));
  const int e = tcp_exp(m);
  unsigned short h[ND][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = 8 * j + q;
    int d[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) d[i] = 0;
    if (k < kb && m > 0.f) {   // (e = 0 is also the exponent of a row whose largest |hi| is in [1/4, 1/2))
      tcp_digits<ND>(ldexp(tcp_value(v[k * vstride]), -e), d);
    }
#pragma unroll
    for (int i = 0; i < ND; ++i) h[i][q] = __bfloat16_as_ushort(__float2bfloat16((float)d[i]));
  }
  const uint32_t o = (uint32_t)(row * DROW + ((j ^ (row & 7)) << 4));
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    uint4 w;
    w.x = h[i][0] | ((uint32_t)h[i][1] << 16);
    w.y = h[i][2] | ((uint32_t)h[i][3] << 16);
    w.z = h[i][4] | ((uint32_t)h[i][5] << 16);
    w.w = h[i][6] | ((uint32_t)h[i][7] << 16);
    *(uint4*)(base + (size_t)i * digit_stride + o) = w;
  }
  return e;
}

template <class Cfg>
using Args = TcpDev<typename Cfg::Elem, typename Cfg::Op>;

// left operand: four threads (one per chunk) per row of the active matrices
// (rows padded to 128)
template <class Cfg>
__global__ void __launch_bounds__(128) tcp_left_kernel(Args<Cfg> g, int active, int64_t k0) {
  const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = tt >> 2;
  const int j = (int)(tt & 3);
  if (t >= g.pl[active]) return;
  const int a = tcp_find(g.pl, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int64_t r = t - g.pl[a];
  const int kb = (int)(n - k0 < KG ? n - k0 : KG);
  unsigned char* base = g.Lsl + (size_t)(t / TR) * Cfg::ND * LBLK;
  using Op = typename Cfg::Op;
  const Op zero[1] = {Op{}};
  const Op* v = zero;
  int64_t vs = 0;
  int kk = 0;
  if (r < n) {
    kk = kb;
    vs = 1;
    v = (r >= k0 && r < k0 + kb) ? g.Pf + (int64_t)a * KG * KG + (r - k0) * KG : g.Cf + g.soff[a] + r * KG;
  }
  const int e = tcp_slice_chunk<Cfg>(v, vs, kk, base, LBLK, (int)(t % TR), j);
  if (j == 0) g.exL[t] = e;
}

// right operand: four threads per column of the active matrices (padded to TN)
template <class Cfg>
__global__ void __launch_bounds__(128) tcp_right_kernel(Args<Cfg> g, int active, int64_t k0) {
  constexpr int TN = Cfg::TN;
  const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = tt >> 2;
  const int j = (int)(tt & 3);
  if (t >= g.pr[active]) return;
  const int a = tcp_find(g.pr, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int64_t c = t - g.pr[a];
  const int kb = (int)(n - k0 < KG ? n - k0 : KG);
  unsigned char* base = g.Rsl + (size_t)(t / TN) * Cfg::ND * Lay<Cfg>::RBLK;
  using Op = typename Cfg::Op;
  const Op zero[1] = {Op{}};
  const Op* v = zero;
  int64_t vs = 0;
  int kk = 0;
  if (c < n) {
    kk = kb;
    vs = n;
    v = g.Rf + g.soff[a] + c;
  }
  const int e = tcp_slice_chunk<Cfg>(v, vs, kk, base, Lay<Cfg>::RBLK, (int)(t % TN), j);
  if (j == 0) g.exR[t] = e;
}

// ---- waits, descriptors, tensor-memory loads --------------------------------

__device__ __forceinline__ uint32_t tcp_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tcp_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the phase of the barrier with the given parity to complete; false
// after ~2 s, after 2^24 tries, or once another role has given up (*abort;
// abort may be NULL)
__device__ __noinline__ bool tcp_wait(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  const uint64_t t0 = tcp_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t ok;
    // suspended in hardware until the phase completes, for at most ~1 ms per
    // try, instead of spinning on the issue slots the other warps need
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0,1,0,p;\n}\n"
        : "=r"(ok) : "r"(tcp_smem(bar)), "r"(parity), "r"(1000000u) : "memory");
    if (ok) return true;
    if ((abort && *abort) || tcp_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// shared-memory matrix descriptor: K-major, 128-byte rows under the 128-byte
// swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t tcp_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tcp_ld16(uint32_t addr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(addr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :: "memory");
}

__device__ __forceinline__ void tcp_ld8(uint32_t addr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :: "memory");
}
template <int NC>
__device__ __forceinline__ void tcp_ldn(uint32_t addr, uint32_t* r) {
  if constexpr (NC == 8) tcp_ld8(addr, r); else tcp_ld16(addr, r);
}

// 2^s as a float for -126 <= s <= 127
__device__ __forceinline__ float tcp_pow2(int s) { return __int_as_float((s + 127) << 23); }


// Where tile t of the step lies: matrix (sorted position a, id b, order n,
// row stride ld), its first row and column, its left and right digit tiles.
template <class Cfg>
struct TileAt {
  int a, b, kb;
  int64_t n, ld, r0, c0, Lt, Rt;
  __device__ __forceinline__ TileAt(const Args<Cfg>& g, int active, int64_t k0, int64_t t) {
    constexpr int TN = Cfg::TN;
    a = tcp_find(g.pt, active, t);
    b = g.order[a];
    n = g.bsize[b];
    ld = tcp_ld<typename Cfg::Elem>(n);
    const int ntn = (int)((n + TN - 1) / TN), loc = (int)(t - g.pt[a]);   // tiles of a matrix < 2^31
    r0 = (int64_t)(loc / ntn) * TR;
    c0 = (int64_t)(loc % ntn) * TN;
    kb = (int)(n - k0 < KG ? n - k0 : KG);
    Lt = (g.pl[a] + r0) / TR;
    Rt = (g.pr[a] + c0) / TN;
  }
};

template <class Cfg>
__global__ void __launch_bounds__(NTHREADS, 1) tcp_update_kernel(Args<Cfg> g, int active, int64_t k0,
                                                                 int64_t tiles) {
  using L = Lay<Cfg>;
  using Elem = typename Cfg::Elem;
  constexpr int TN = Cfg::TN, ND = Cfg::ND, LEVELS = Cfg::LEVELS;
  extern __shared__ unsigned char tcp_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcp_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sL = base;
  unsigned char* sR = base + L::OFF_R;                  // stage s at + s * RB
  uint64_t* bars = (uint64_t*)(base + L::OFF_BAR);
  uint64_t* full = bars;          // [2] digits of a stage landed
  uint64_t* empty = bars + 2;     // [2] the MMAs reading a stage (and the left digits) are done
  uint64_t* tfull = bars + 4;     // [2] an accumulator set is complete
  uint64_t* tempty = bars + 6;    // [2] the epilogue has read an accumulator set
  uint32_t* tbase = (uint32_t*)(bars + 8);
  volatile int* abort_ = (volatile int*)(bars + 9);
  volatile int* issued = (volatile int*)(bars + 10);   // [0] tiles copied, [1] tiles whose MMAs were committed
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tb = tiles * blockIdx.x / gridDim.x, te = tiles * (blockIdx.x + 1) / gridDim.x;
  const int cnt = (int)(te - tb);

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tcp_smem(tbase)),
                 "r"(512) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 8; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tcp_smem(&bars[i])),
                   "r"(i >= 6 ? NEPI : 1) : "memory");
    *abort_ = 0;
    issued[0] = 0;
    issued[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tbase;

  if (warp == 0) {
    // ---- producer: digit tiles by bulk asynchronous copies
    if (lane == 0) {
      int64_t prevLt = -1;
      for (int i = 0; i < cnt; ++i) {
        const TileAt<Cfg> T(g, active, k0, tb + i);
        const int s = i & 1;
        if (i >= 2 && !tcp_wait(&empty[s], ((i - 2) >> 1) & 1, abort_)) { *abort_ = 1; break; }
        const bool newrow = T.Lt != prevLt;
        // the left digits are replaced only once the MMAs of the previous tile are done
        if (newrow && i >= 1 && !tcp_wait(&empty[(i - 1) & 1], ((i - 1) >> 1) & 1, abort_)) { *abort_ = 1; break; }
        const uint32_t bytes = (uint32_t)L::RB + (newrow ? (uint32_t)L::LB : 0u);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tcp_smem(&full[s])),
                     "r"(bytes) : "memory");
        if (newrow)
          for (int d = 0; d < ND; ++d)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(tcp_smem(sL + d * LBLK)), "l"(g.Lsl + ((size_t)T.Lt * ND + d) * LBLK), "r"(LBLK),
                         "r"(tcp_smem(&full[s])) : "memory");
        for (int d = 0; d < ND; ++d)
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       ::"r"(tcp_smem(sR + s * L::RB + d * L::RBLK)),
                       "l"(g.Rsl + ((size_t)T.Rt * ND + d) * L::RBLK), "r"(L::RBLK), "r"(tcp_smem(&full[s]))
                       : "memory");
        issued[0] = i + 1;
        prevLt = T.Lt;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: level l of tile i into accumulator set i & 1, columns l TN ..
    if (lane == 0) {
      // bf16 A and B, FP32 accumulators, M = 128, N = TN
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TR >> 4) << 24);
      for (int i = 0; i < cnt; ++i) {
        const int s = i & 1;
        if (!tcp_wait(&full[s], (i >> 1) & 1, abort_)) { *abort_ = 1; break; }
        if (i >= 2 && !tcp_wait(&tempty[s], ((i - 2) >> 1) & 1, abort_)) { *abort_ = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dset = taddr + (uint32_t)(s * L::TCOLS);
        for (int l = 0; l < LEVELS; ++l) {
          uint32_t en = 0;                     // the level's first MMA overwrites its accumulator
          for (int x = 0; x < ND && x <= l; ++x) {
            const int y = l - x;
            if (y >= ND) continue;
            for (int kk = 0; kk < KG / 16; ++kk) {
              const uint64_t ad = tcp_desc(tcp_smem(sL + x * LBLK) + 32u * kk);
              const uint64_t bd = tcp_desc(tcp_smem(sR + s * L::RB + y * L::RBLK) + 32u * kk);
              asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                           " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                           ::"r"(dset + (uint32_t)(l * TN)), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
              en = 1;
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tcp_smem(&empty[s])) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tcp_smem(&tfull[s])) : "memory");
        issued[1] = i + 1;
      }
    }
  } else {
    // ---- epilogue: sixteen warps; warp w owns TMEM lanes 32 (w mod 4) .. +31
    // (one tile row per thread) and the tile columns col0 .. col0 + CW - 1.
    // Each thread reads its old entries of A before it waits for the
    // accumulators, updates them in registers and stores them back.
    constexpr int CW = TN / 4;
    const int ew = warp - 2;
    const int qd = warp & 3;
    const int row = 32 * qd + lane;
    const int col0 = (ew >> 2) * CW;
    const uint32_t lanes = (uint32_t)(32 * qd) << 16;
    for (int i = 0; i < cnt; ++i) {
      const TileAt<Cfg> T(g, active, k0, tb + i);
      const int64_t r = T.r0 + row;
      const int64_t cb = T.c0 + col0;
      const bool rin = r < T.n, rK = r >= k0 && r < k0 + T.kb;
      // no pivot column and no column past the matrix among this thread's
      const bool plain = cb + CW <= T.n && (cb + CW <= k0 || cb >= k0 + T.kb);
      Elem* Arow = g.Ap[T.b] + (rin ? r : 0) * T.ld + cb;
      Elem old[CW];
#pragma unroll
      for (int j = 0; j < CW; ++j) old[j] = (Elem)0;
      if (rin && !rK) {
#pragma unroll
        for (int j = 0; j < CW; ++j)
          if (plain || cb + j < T.n) old[j] = Arow[j];
      }
      const int eL = g.exL[T.Lt * TR + row];
      const int* exc = g.exR + T.Rt * TN + col0;   // the same for every lane: broadcast loads
      // one lane per warp waits for the accumulators
      int got = 0;
      if (lane == 0) got = tcp_wait(&tfull[i & 1], (i >> 1) & 1, abort_) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        *abort_ = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dset = taddr + lanes + (uint32_t)((i & 1) * L::TCOLS + col0);
      // sum_l Q_l 2^(-8(l+2)) in double-float, smallest level first; every
      // term is exact (Q_l an integer below 2^22 times a power of two)
      float sh[CW], sl[CW];
      uint32_t q[CW];
      tcp_ldn<CW>(dset + (uint32_t)((LEVELS - 1) * TN), q);
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        sh[j] = __uint_as_float(q[j]) * tcp_pow2(-8 * (LEVELS + 1));
        sl[j] = 0.f;
      }
#pragma unroll
      for (int l = LEVELS - 2; l >= 0; --l) {
        tcp_ldn<CW>(dset + (uint32_t)(l * TN), q);
        const float w = tcp_pow2(-8 * (l + 2));
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          float s2, e2;
          two_sum(sh[j], __uint_as_float(q[j]) * w, s2, e2);
          sh[j] = s2;
          sl[j] += e2;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tcp_smem(&tempty[i & 1])) : "memory");
      if (!rin) continue;
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const int64_t c = cb + j;
        if (!plain && c >= T.n) continue;
        Elem v;
        if (!plain && c >= k0 && c < k0 + T.kb) {
          // a pivot column takes the left operand itself
          const auto Lv = rK ? g.Pf[(int64_t)T.a * KG * KG + (r - k0) * KG + (c - k0)]
                             : g.Cf[g.soff[T.a] + r * KG + (c - k0)];
          v = tcp_value(Lv);
        } else {
          const int sc = eL + exc[j];
          const bool normal = sc >= -126 && sc <= 127;
          const float f = tcp_pow2(normal ? sc : 0);
          const float ph = normal ? sh[j] * f : ldexpf(sh[j], sc);
          const float pl = normal ? sl[j] * f : ldexpf(sl[j], sc);
          v = old[j] + (widen(ph) + widen(pl));
        }
        Arow[j] = v;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_) {
    // give up: let the copies and the MMAs in flight finish, bounded, before
    // the shared memory and the tensor memory are given back
    atomicExch(g.err, 1);
    const int ni = issued[0], nm = issued[1];
    for (int i = ni >= 2 ? ni - 2 : 0; i < ni; ++i) tcp_wait(&full[i & 1], (i >> 1) & 1, nullptr);
    for (int i = nm >= 2 ? nm - 2 : 0; i < nm; ++i) tcp_wait(&empty[i & 1], (i >> 1) & 1, nullptr);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(512) : "memory");
}

template <class Cfg>
cudaError_t tcp_launch(const Args<Cfg>& d, int active, int64_t k0, int64_t rows, int64_t cols, int64_t tiles,
                       int sms, cudaStream_t s) {
  if (rows <= 0 || tiles <= 0) return cudaSuccess;
  if (rows / 32 > 0x7fffffff || cols / 32 > 0x7fffffff) return cudaErrorInvalidValue;
  tcp_left_kernel<Cfg><<<(unsigned)((4 * rows + 127) / 128), 128, 0, s>>>(d, active, k0);
  tcp_right_kernel<Cfg><<<(unsigned)((4 * cols + 127) / 128), 128, 0, s>>>(d, active, k0);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
  tcp_update_kernel<Cfg><<<grid, NTHREADS, Lay<Cfg>::SMEM, s>>>(d, active, k0, tiles);
  return cudaGetLastError();
}

}  // namespace

size_t tcp_slice_bytes(int64_t rows, int64_t cols) { return (size_t)(rows + cols) * CfgDF::ND * DROW; }

int tcp_tile_cols() { return CfgDF::TN; }

cudaError_t tcp_init(int* sms) {
  static std::mutex mu;
  static std::vector<std::pair<int, int>> ready;   // (device, SM count)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& r : ready)
    if (r.first == dev) {
      *sms = r.second;
      return cudaSuccess;
    }
  int n = 0;
  if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tcp_update_kernel<CfgDF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Lay<CfgDF>::SMEM)) != cudaSuccess)
    return e;
  ready.emplace_back(dev, n);
  *sms = n;
  return cudaSuccess;
}

cudaError_t launch_tcp_update(const TcpDev<double, float2>& d, int active, int64_t k0, int64_t rows, int64_t cols,
                              int64_t tiles, int sms, cudaStream_t s) {
  return tcp_launch<CfgDF>(d, active, k0, rows, cols, tiles, sms, s);
}

}  // namespace msbem
