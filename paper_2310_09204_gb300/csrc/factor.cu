// Set-up of the two-level additive Schwarz preconditioner (Sec. 2.1 Remark
// "Bound on the number of PCG iterations", Sec. 5 eq. jumpSplit):
//
//   M r = sum_F R_F^T A_F^{-1} R_F r + R_W^T A_W^{-1} R_W r + P A_H^{-1} P^T r,
//   A_F = W[F,F], A_W = W[W,W], A_H = P^T W P.
//
// Every block is gathered into one packed buffer and inverted explicitly, so
// that each PCG iteration applies M with dense matrix-vector products instead
// of sequential triangular solves.  The inversion is Gauss-Jordan elimination
// without pivoting, which is stable for symmetric positive definite blocks; a
// non-positive or non-finite pivot is reported as a breakdown.
#include <algorithm>
#include <cstring>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

__global__ void gather_blocks_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl,
                                     int64_t ldw,
                                     const int64_t* __restrict__ bptr,
                                     const int32_t* __restrict__ bdofs,
                                     const int64_t* __restrict__ boff,
                                     const int64_t* __restrict__ prefix2, int nblk, int wb_block,
                                     int wb_diag, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prefix2[nblk]) return;
  // the block of entry t: largest b with prefix2[b] <= t (binary search)
  int b = 0, hi = nblk - 1;
  while (b < hi) {
    const int mid = (b + hi + 1) >> 1;
    if (prefix2[mid] <= t) b = mid; else hi = mid - 1;
  }
  const int64_t n = bptr[b + 1] - bptr[b];
  const int64_t e = t - prefix2[b];
  const int64_t i = e / n, j = e % n;
  const int64_t di = bdofs[bptr[b] + i], dj = bdofs[bptr[b] + j];
  double v = df_to_double(Wh[di * ldw + dj], Wl[di * ldw + dj]);
  if (b == wb_block && wb_diag) v = (i == j) ? 1.0 / v : 0.0;
  out[boff[b] + e] = v;
}

// W P  (transposed, NH x N) from the CSC form of P:  (W P)^T[mu][i] = sum_nu P[nu,mu] W[nu][i],
// accumulated in double-float (W and P values are float pairs)
__global__ void wp_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl, int64_t ldw,
                          int64_t N, const int64_t* __restrict__ cptr,
                          const int32_t* __restrict__ crow, const float2* __restrict__ cval,
                          double* __restrict__ WPt) {
  const int64_t mu = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float acch = 0.f, accl = 0.f;
  for (int64_t k = cptr[mu]; k < cptr[mu + 1]; ++k) {
    const int64_t o = (int64_t)crow[k] * ldw + i;
    const float2 c = cval[k];
    df_fma_acc(c.x, c.y, Wh[o], Wl[o], acch, accl);
  }
  WPt[mu * N + i] = df_to_double(acch, accl);
}

__global__ void ah_kernel(const double* __restrict__ WPt, int64_t N, int64_t NH,
                          const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                          const double* __restrict__ cval, double* __restrict__ AH) {
  const int64_t mu = blockIdx.x, nu = threadIdx.x + (int64_t)blockIdx.y * blockDim.x;
  if (nu >= NH) return;
  double acc = 0.0;
  for (int64_t k = cptr[mu]; k < cptr[mu + 1]; ++k) acc = fma(cval[k], WPt[nu * N + crow[k]], acc);
  AH[mu * NH + nu] = acc;
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion of a batch of SPD matrices, in place.
// Pivot panels of GB = 32 rows/columns K; for every active matrix:
//   P = A_KK^{-1}                       (bgj_pivot_kernel, double-float in shared memory)
//   C'_I = -A_IK P,  R_J = A_KJ (old)   (bgj_panel_kernel, double-float)
//   A_IJ += C'_I R_J, A_KJ = P R_J, A_IK = C'_I, A_KK = P
//                                       (bgj_update_kernel, double-float tiles;
//                                        factor_tcp.cu on the tensor cores for
//                                        matrices of order >= kTcMinOrder)
// which is the scalar Gauss-Jordan recursion applied 32 pivots at a time; after
// the last panel A holds A^{-1}.  Rank-32 updates run as double-float products
// on the FP32 pipe (GB300 FP64 is ~1/70 of FP32) or as exact integer-slice
// products on the tensor cores, and P in double-float on the FP32 pipe.
// ---------------------------------------------------------------------------
#define GB 32

struct BgjArgs {
  double* const* Ap;      // per matrix id: the matrix (row-major, bsize x bsize)
  const int64_t* bsize;   // per matrix id
  const int32_t* order;   // matrix ids sorted by size (descending)
  const int64_t* pt1;     // prefix over sorted matrices of tiles per side
  const int64_t* pt2;     // prefix of tiles^2
  const int64_t* soff;    // prefix of n * GB (scratch panels), sorted order
  float2* Pf;             // [sorted][GB*GB]
  float2* Cf;             // [soff] n x GB
  float2* Rf;             // [soff] GB x n
  int* flag;              // per matrix id: 1 when a pivot was not positive
};

__device__ __forceinline__ int find_prefix(const int64_t* pre, int active, int64_t t) {
  int lo = 0, hi = active - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(1024) bgj_pivot_kernel(BgjArgs g, int64_t k0) {
  // the scalar recursion on the 32 x 32 pivot block in double-float on the
  // FP32 pipe (GB300's FP64 pipe would make these 32 dependent steps the
  // critical path of every panel step); one thread per entry, so that the
  // latency of each step's chain is hidden by 32 warps
  __shared__ float2 S[GB][GB + 1];
  __shared__ float2 rowk[GB], colk[GB];  // pivot row scaled by 1/p, pivot column
  __shared__ float2 s_ip;
  const int a = blockIdx.x;
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int kb = (int)(n - k0 < GB ? n - k0 : GB);
  const double* A = g.Ap[b];
  for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) {
    const int i = e / GB, j = e % GB;
    const double v = (i < kb && j < kb) ? A[(k0 + i) * n + k0 + j] : (i == j ? 1.0 : 0.0);
    float h, l;
    split_df(v, h, l);
    S[i][j] = make_float2(h, l);
  }
  __syncthreads();
  for (int k = 0; k < GB; ++k) {
    // one warp forms 1/p, the scaled pivot row and the pivot column
    if (threadIdx.x < 32) {
      const float2 pk = S[k][k];
      // 1/p in double-float without the FP64 pipe: the correctly rounded FP32
      // reciprocal r, then one Newton step on the residual 1 - p r formed
      // with an exact FMA product (relative error ~2^-46)
      const float r = __frcp_rn(pk.x);
      const float t = fmaf(-pk.y, r, fmaf(-pk.x, r, 1.0f));
      float iph, ipl;
      two_sum(r, r * t, iph, ipl);
      if (threadIdx.x == 0) {
        s_ip = make_float2(iph, ipl);
        if (!(pk.x > 0.f && isfinite(pk.x))) g.flag[b] = 1;
      }
      const float2 skj = S[k][threadIdx.x];
      float rh, rl;
      df_mul(skj.x, skj.y, iph, ipl, rh, rl);
      rowk[threadIdx.x] = make_float2(rh, rl);
      colk[threadIdx.x] = S[threadIdx.x][k];
    }
    __syncthreads();
    const float2 ip = s_ip;
    for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) {
      const int i = e / GB, j = e % GB;
      float2 v;
      if (i == k) {
        v = (j == k) ? ip : rowk[j];
      } else if (j == k) {
        float rh, rl;
        df_mul(colk[i].x, colk[i].y, ip.x, ip.y, rh, rl);
        v = make_float2(-rh, -rl);
      } else {
        float h = S[i][j].x, l = S[i][j].y;
        df_fma_acc(-colk[i].x, -colk[i].y, rowk[j].x, rowk[j].y, h, l);
        const float sh = h + l;
        v = make_float2(sh, l - (sh - h));
      }
      S[i][j] = v;
    }
    __syncthreads();
  }
  float2* P = g.Pf + (int64_t)a * GB * GB;
  for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) P[e] = S[e / GB][e % GB];
}

__global__ void __launch_bounds__(256) bgj_panel_kernel(BgjArgs g, int active, int64_t k0) {
  __shared__ float2 sP[GB][GB + 1];
  __shared__ float2 sA[GB][GB + 1];
  const int64_t t = blockIdx.x;
  const int a = find_prefix(g.pt1, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int I = (int)(t - g.pt1[a]);
  const int kb = (int)(n - k0 < GB ? n - k0 : GB);
  const double* A = g.Ap[b];
  float2* C = g.Cf + g.soff[a];
  float2* R = g.Rf + g.soff[a];
  const int64_t r0 = (int64_t)I * GB;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // old row panel: R[m][col] = A[k0+m][col], col in tile I
  for (int m = ty; m < kb; m += 8) {
    int64_t col = r0 + tx;
    if (col < n) {
      float h, l;
      split_df(A[(k0 + m) * n + col], h, l);
      R[m * n + col] = make_float2(h, l);
    }
  }
  if (r0 == k0) return;
  // C'_I = -A_IK P
  const float2* P = g.Pf + (int64_t)a * GB * GB;
  for (int e = threadIdx.x; e < GB * GB; e += blockDim.x) sP[e / GB][e % GB] = P[e];
  for (int i = ty; i < GB; i += 8) {
    int64_t row = r0 + i;
    float h = 0.f, l = 0.f;
    if (row < n && tx < kb) split_df(A[row * n + k0 + tx], h, l);
    sA[i][tx] = make_float2(h, l);
  }
  __syncthreads();
  for (int i = ty; i < GB; i += 8) {
    int64_t row = r0 + i;
    if (row >= n || tx >= kb) continue;
    float acch = 0.f, accl = 0.f;
    for (int m = 0; m < kb; ++m) df_fma_acc(sA[i][m].x, sA[i][m].y, sP[m][tx].x, sP[m][tx].y, acch, accl);
    C[row * GB + tx] = make_float2(-acch, -accl);
  }
}

// tiles tile0 + blockIdx.x of the active matrices' 32 x 32 tiles
__global__ void __launch_bounds__(256) bgj_update_kernel(BgjArgs g, int active, int64_t k0, int64_t tile0) {
  __shared__ float2 sL[GB][GB + 1];
  __shared__ float2 sR[GB][GB + 1];
  const int64_t t = tile0 + blockIdx.x;
  const int a = find_prefix(g.pt2, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int nti = (int)((n + GB - 1) / GB);
  const int64_t loc = t - g.pt2[a];
  const int I = (int)(loc / nti), J = (int)(loc % nti);
  const int kt = (int)(k0 / GB);
  const int kb = (int)(n - k0 < GB ? n - k0 : GB);
  double* A = g.Ap[b];
  const float2* C = g.Cf + g.soff[a];
  const float2* R = g.Rf + g.soff[a];
  const float2* P = g.Pf + (int64_t)a * GB * GB;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)I * GB, c0 = (int64_t)J * GB;
  if (I == kt && J == kt) {
    for (int i = ty; i < kb; i += 8)
      if (tx < kb) A[(k0 + i) * n + k0 + tx] = df_to_double(P[i * GB + tx].x, P[i * GB + tx].y);
    return;
  }
  if (J == kt) {
    for (int i = ty; i < GB; i += 8) {
      int64_t row = r0 + i;
      if (row < n && tx < kb) {
        float2 v = C[row * GB + tx];
        A[row * n + k0 + tx] = df_to_double(v.x, v.y);
      }
    }
    return;
  }
  // left factor: P (row panel) or C'_I; right factor: R_KJ
  for (int i = ty; i < GB; i += 8) {
    float2 v = make_float2(0.f, 0.f);
    if (I == kt) {
      if (i < kb && tx < kb) v = P[i * GB + tx];
    } else {
      int64_t row = r0 + i;
      if (row < n && tx < kb) v = C[row * GB + tx];
    }
    sL[i][tx] = v;
    float2 w = make_float2(0.f, 0.f);
    int64_t col = c0 + tx;
    if (i < kb && col < n) w = R[i * n + col];
    sR[i][tx] = w;
  }
  __syncthreads();
  // rows ty, ty + 8, ty + 16, ty + 24 of the tile at once: one read of the
  // right factor per m, four independent accumulators
  const int64_t col = c0 + tx;
  float acch[4] = {0.f, 0.f, 0.f, 0.f}, accl[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = 0; m < kb; ++m) {
    const float2 r = sR[m][tx];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 l = sL[ty + 8 * q][m];
      df_fma_acc(l.x, l.y, r.x, r.y, acch[q], accl[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = ty + 8 * q;
    const int64_t row = r0 + i;
    if (row >= n || col >= n) continue;
    if (I == kt && i >= kb) continue;
    const double upd = df_to_double(acch[q], accl[q]);
    A[row * n + col] = (I == kt) ? upd : A[row * n + col] + upd;
  }
}

// ---------------------------------------------------------------------------
// The same blocked Gauss-Jordan recursion in FP32, for the face and
// wire-basket blocks of a preconditioner that only the mixed-precision solves
// read (their inner PCG applies the FP32 inverses; the refinement's residual
// uses W alone, so the preconditioner's precision sets the inner convergence
// rate, not the accuracy of the result).  One FP32 FMA per update term instead
// of a double-float product of 13 FP32 operations, and the matrices stay in
// FP32 (half the bytes per pass).  The result is symmetrised.
// ---------------------------------------------------------------------------
// row stride of the FP32 copies: n rounded up to 4 floats, so that every row
// starts on a 16-byte boundary (vector accesses in the update)
__host__ __device__ __forceinline__ int64_t f32_ld(int64_t n) { return (n + 3) & ~(int64_t)3; }

struct Bgj32Args {
  float* const* Ap;       // per matrix id: the matrix (row-major FP32, bsize x bsize)
  const int64_t* bsize;   // per matrix id
  const int32_t* order;   // matrix ids sorted by size (descending)
  const int64_t* pt1;     // prefix over sorted matrices of tiles per side
  const int64_t* pt3;     // prefix of 128 x 128 update tiles
  const int64_t* soff;    // prefix of n * GB (scratch panels), sorted order
  float* Pf;              // [sorted][GB*GB]
  float* Cf;              // [soff] n x GB
  float* Rf;              // [soff] GB x n
  int* flag;              // per matrix id: 1 when a pivot was not positive
};

// The 32 x 32 pivot block inverted by one warp: lane j holds column j of the
// block in registers; per pivot k the warp forms 1/p, scales row k and
// eliminates column k, the column entries S[i][k] broadcast by shuffles.  Rows
// / columns past kb hold the identity.  P[i][j] is written to sP (row stride
// GB + 1); the result is false if a pivot was not positive.
__device__ __forceinline__ bool pivot32_warp(const float* A, int64_t ld, int64_t k0, int kb, float* sP) {
  const int j = threadIdx.x & 31;
  float s[GB];
#pragma unroll
  for (int i = 0; i < GB; ++i) s[i] = (i < kb && j < kb) ? A[(k0 + i) * ld + k0 + j] : (i == j ? 1.0f : 0.0f);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < GB; ++k) {
    const float pk = __shfl_sync(0xffffffffu, s[k], k);
    ok = ok && pk > 0.f && isfinite(pk);
    const float ip = 1.0f / pk;
    const float rk = (j == k) ? ip : s[k] * ip;   // the new row k
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      if (i == k) continue;
      const float cik = __shfl_sync(0xffffffffu, s[i], k);   // S[i][k] before the step
      s[i] = (j == k) ? -cik * ip : fmaf(-cik, rk, s[i]);
    }
    s[k] = rk;
  }
#pragma unroll
  for (int i = 0; i < GB; ++i) sP[i * (GB + 1) + j] = s[i];
  return ok;
}

// One step's panels, one CTA per 32-row tile of every active matrix: warp 0
// inverts the pivot block (each CTA for itself: no separate launch, no
// dependency between CTAs), while the other warps copy the old pivot rows R
// over the tile's 32 columns; then C'_I = -A_IK P for the tile's rows.  The
// CTA of the pivot tile writes P (read by the update for the rows in K) and
// the breakdown flag.
__global__ void __launch_bounds__(256) bgj32_panel_kernel(Bgj32Args g, int active, int64_t k0) {
  __shared__ float sP[GB][GB + 1];
  __shared__ float sA[GB][GB + 1];
  const int64_t t = blockIdx.x;
  const int a = find_prefix(g.pt1, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int I = (int)(t - g.pt1[a]);
  const int kb = (int)(n - k0 < GB ? n - k0 : GB);
  const float* A = g.Ap[b];
  const int64_t ld = f32_ld(n);
  float* C = g.Cf + g.soff[a];
  float* R = g.Rf + g.soff[a];
  const int64_t r0 = (int64_t)I * GB;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (ty == 0) {
    const bool ok = pivot32_warp(A, ld, k0, kb, &sP[0][0]);
    if (r0 == k0) {
      float* P = g.Pf + (int64_t)a * GB * GB;
#pragma unroll 4
      for (int i = 0; i < GB; ++i) P[i * GB + tx] = sP[i][tx];
      if (tx == 0 && !ok) g.flag[b] = 1;
    }
  } else {
    for (int m = ty - 1; m < kb; m += 7) {
      const int64_t col = r0 + tx;
      if (col < n) R[m * n + col] = A[(k0 + m) * ld + col];
    }
    for (int i = ty - 1; i < GB; i += 7) {
      const int64_t row = r0 + i;
      sA[i][tx] = (row < n && tx < kb) ? A[row * ld + k0 + tx] : 0.f;
    }
  }
  if (r0 == k0) return;
  __syncthreads();
  for (int i = ty; i < GB; i += 8) {
    const int64_t row = r0 + i;
    if (row >= n || tx >= kb) continue;
    float acc = 0.f;
    for (int m = 0; m < kb; ++m) acc = fmaf(sA[i][m], sP[m][tx], acc);
    C[row * GB + tx] = -acc;
  }
}

// Update of one 128 x 128 tile per CTA, 8 x 8 outputs per thread.  With K
// the pivot rows / columns [k0, k0 + kb), L(r) = P[r - k0] for r in K, else
// C'_r, and R[m][c] the old A[k0 + m][c]:
//   A[r][c] = L(r)[c - k0]                         for c in K,
//   A[r][c] = [r not in K] A[r][c] + L(r) . R[:, c]  otherwise,
// which is the scalar Gauss-Jordan step on 32 pivots at once.  The tile of A
// comes in by 16-byte asynchronous copies at the start (rows start on 16-byte
// boundaries), so that the pass over the matrix overlaps the panel loads and
// the products; two CTAs per SM.
#define UT 128
constexpr int UT_LDL = UT + 4;    // row stride of sLT (16-byte rows, 4-way conflicts on the transposing stores)
constexpr size_t UT_SMEM = sizeof(float) * ((size_t)GB * UT_LDL + (size_t)GB * UT + (size_t)UT * UT);
__global__ void __launch_bounds__(256, 2) bgj32_update_kernel(Bgj32Args g, int active, int64_t k0) {
  extern __shared__ __align__(16) float sm32[];
  float* sLT = sm32;                     // sLT[m * UT_LDL + i] = L(r0 + i)[m]
  float* sR = sm32 + GB * UT_LDL;        // sR[m * UT + j] = R[m][c0 + j]
  float* sT = sR + GB * UT;              // sT[i * UT + j] = A[r0 + i][c0 + j]
  const int64_t t = blockIdx.x;
  const int a = find_prefix(g.pt3, active, t);
  const int b = g.order[a];
  const int64_t n = g.bsize[b];
  const int nt = (int)((n + UT - 1) / UT);
  const int64_t loc = t - g.pt3[a];
  const int64_t r0 = (loc / nt) * UT, c0 = (loc % nt) * UT;
  const int kb = (int)(n - k0 < GB ? n - k0 : GB);
  float* A = g.Ap[b];
  const float* C = g.Cf + g.soff[a];
  const float* R = g.Rf + g.soff[a];
  const float* P = g.Pf + (int64_t)a * GB * GB;
  const int tid = threadIdx.x;
  const int64_t ld = f32_ld(n);
  for (int e = tid; e < UT * UT / 4; e += 256) {
    const int i = e / (UT / 4), q = e % (UT / 4);   // consecutive threads: consecutive 16-byte chunks of a row
    const int64_t r = r0 + i, c = c0 + 4 * q;
    if (r < n && c < ld && !(r >= k0 && r < k0 + kb))
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sT + i * UT + 4 * q)),
                   "l"(A + r * ld + c) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  // the panels: all 32 loads of a thread in flight before its stores
  constexpr int PQ = GB * UT / 256;
  float lq[PQ], rq[PQ];
#pragma unroll
  for (int q = 0; q < PQ; ++q) {
    const int e = tid + 256 * q;
    const int i = e / GB, m = e % GB;           // consecutive threads: consecutive m (one row of L)
    const int64_t r = r0 + i;
    lq[q] = 0.f;
    if (r < n && m < kb) lq[q] = (r >= k0 && r < k0 + kb) ? P[(r - k0) * GB + m] : C[r * GB + m];
    const int mm = e / UT, jj = e % UT;         // consecutive threads: consecutive columns
    const int64_t c = c0 + jj;
    rq[q] = (mm < kb && c < n) ? R[mm * n + c] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < PQ; ++q) {
    const int e = tid + 256 * q;
    sLT[(e % GB) * UT_LDL + e / GB] = lq[q];
    sR[e] = rq[q];                              // (e / UT) * UT + e % UT
  }
  __syncthreads();
  // rows 4ty + u and 64 + 4ty + u, columns 4tx + v and 64 + 4tx + v
  const int ty = tid >> 4, tx = tid & 15;
  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  // the panel entries past kb are zero, so a full 32-term loop (unrolled) is
  // exact for every step
#pragma unroll 8
  for (int m = 0; m < GB; ++m) {
    const float4 l0 = *(const float4*)&sLT[m * UT_LDL + 4 * ty];
    const float4 l1 = *(const float4*)&sLT[m * UT_LDL + 64 + 4 * ty];
    const float4 q0 = *(const float4*)&sR[m * UT + 4 * tx];
    const float4 q1 = *(const float4*)&sR[m * UT + 64 + 4 * tx];
    const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
    const float rv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(lv[u], rv[v], acc[u][v]);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (c0 + UT <= n && (c0 + UT <= k0 || c0 >= k0 + kb)) {
    // no pivot column and no column past the matrix in this tile
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = (u < 4 ? 0 : 64) + 4 * ty + (u & 3);
      const int64_t r = r0 + i;
      if (r >= n) continue;
      const bool rK = r >= k0 && r < k0 + kb;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jb = 64 * h + 4 * tx;
        const float4 o = rK ? make_float4(0.f, 0.f, 0.f, 0.f) : *(const float4*)&sT[i * UT + jb];
        *(float4*)(A + r * ld + c0 + jb) = make_float4(o.x + acc[u][4 * h], o.y + acc[u][4 * h + 1],
                                                      o.z + acc[u][4 * h + 2], o.w + acc[u][4 * h + 3]);
      }
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int i = (u < 4 ? 0 : 64) + 4 * ty + (u & 3);
    const int64_t r = r0 + i;
    if (r >= n) continue;
    const bool rK = r >= k0 && r < k0 + kb;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jb = 64 * h + 4 * tx;
      const int64_t cb = c0 + jb;
      if (cb >= n) continue;
      const float4 o = rK ? make_float4(0.f, 0.f, 0.f, 0.f) : *(const float4*)&sT[i * UT + jb];
      float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t c = cb + v;
        ov[v] = (c >= k0 && c < k0 + kb) ? sLT[(c - k0) * UT_LDL + i] : ov[v] + acc[u][4 * h + v];
      }
      float* dst = A + r * ld + cb;
      if (cb + 3 < n) {
        *(float4*)dst = make_float4(ov[0], ov[1], ov[2], ov[3]);   // 16-byte aligned
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (cb + v < n) dst[v] = ov[v];
      }
    }
  }
}

// FP32 copies of the listed matrices (from FP64) and back (symmetrised):
// one CTA row per matrix, entries strided
__global__ void f64_to_f32_kernel(double* const* src, float* const* dst, const int64_t* bsize,
                                  const int32_t* ids) {
  const int b = ids[blockIdx.y];
  const int64_t n = bsize[b], ld = f32_ld(n);
  const double* s = src[b];
  float* d = dst[b];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    d[i * ld + j] = (float)s[e];
  }
}

__global__ void f32_sym_to_f64_kernel(float* const* src, double* const* dst, const int64_t* bsize,
                                      const int32_t* ids) {
  const int b = ids[blockIdx.y];
  const int64_t n = bsize[b];
  const float* s = src[b];
  double* d = dst[b];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n, ld = f32_ld(n);
    d[e] = 0.5 * ((double)s[i * ld + j] + (double)s[j * ld + i]);
  }
}


__global__ void to_float_pairs_kernel(const double* __restrict__ x, float2* __restrict__ xf, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float h, l;
    split_df(x[i], h, l);
    xf[i] = make_float2(h, l);
  }
}

namespace {
// Scratch of one call: buffers taken from the pool, all returned (stream
// ordered) when the object goes out of scope, on every return path.
class PoolScratch {
 public:
  PoolScratch(cudaMemPool_t pool, cudaStream_t s) : pool_(pool), s_(s) {}
  PoolScratch(const PoolScratch&) = delete;
  PoolScratch& operator=(const PoolScratch&) = delete;
  ~PoolScratch() {
    for (void* q : held_) cudaFreeAsync(q, s_);
  }
  template <class T>
  cudaError_t take(T** d, size_t n) {
    void* q = nullptr;
    cudaError_t e = pool_alloc(&q, sizeof(T) * std::max<size_t>(1, n), pool_, s_);
    if (e != cudaSuccess) return e;
    held_.push_back(q);
    *d = (T*)q;
    return cudaSuccess;
  }
  template <class T>
  cudaError_t put(T** d, const std::vector<T>& h) {
    cudaError_t e = take(d, h.size());
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s_);
  }

 private:
  cudaMemPool_t pool_;
  cudaStream_t s_;
  std::vector<void*> held_;
};

template <class T>
cudaError_t upload(T** d, const std::vector<T>& h, cudaMemPool_t pool, cudaStream_t s) {
  cudaError_t e = pool_alloc((void**)d, sizeof(T) * std::max<size_t>(1, h.size()), pool, s);
  if (e != cudaSuccess) return e;
  if (h.empty()) return cudaSuccess;
  return cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
}
}  // namespace

namespace {

// Symmetric power-of-two equilibration of the double-float inversions:
// A <- S A S with S = diag(2^x_i), x_i = -floor(k_i / 2) for A_ii in
// [2^(k_i - 1), 2^k_i), so that the scaled diagonal lies in [1/2, 2); after the
// recursion the same S gives A^-1 = S (S A S)^-1 S.  Every product by a power
// of two is exact.  The point is the tensor-core update: its error is relative
// to the largest entries of the row of one operand and the column of the other,
// which for a graded matrix (D B D with D spanning many binades) would be far
// above the entries themselves; after the scaling the rows and columns of an
// SPD matrix have comparable scales (|a_ij| <= sqrt(a_ii a_jj) < 2).
__global__ void equil_exp_kernel(double* const* Ap, const int64_t* bsize, const int32_t* order,
                                 const int64_t* prow, int nb, int* ex) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prow[nb]) return;
  const int a = find_prefix(prow, nb, t);
  const int b = order[a];
  const int64_t n = bsize[b], i = t - prow[a];
  const double d = Ap[b][i * n + i];
  int k = 0;
  if (d > 0.0 && isfinite(d)) frexp(d, &k);   // d in [2^(k-1), 2^k)
  ex[t] = -(k >= 0 ? k / 2 : -((1 - k) / 2));  // -floor(k / 2); 0 for a pivot the recursion will reject
}

// one block per row of the matrices: A_ij <- 2^(x_i + x_j) A_ij
__global__ void __launch_bounds__(128) equil_scale_kernel(double* const* Ap, const int64_t* bsize,
                                                          const int32_t* order, const int64_t* prow, int nb,
                                                          const int* ex) {
  const int64_t t = blockIdx.x;
  const int a = find_prefix(prow, nb, t);
  const int b = order[a];
  const int64_t n = bsize[b], i = t - prow[a];
  double* row = Ap[b] + i * n;
  const int xi = ex[t];
  const int* xr = ex + prow[a];
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) row[j] = ldexp(row[j], xi + xr[j]);
}

// Inverts the FP32 matrices of `ids` (their FP64 copies in plan.ptr, in place:
// converted to FP32, inverted, symmetrised and written back).
cudaError_t invert_f32(const InvPlan& plan, const std::vector<int32_t>& ids, cudaMemPool_t pool, cudaStream_t s,
                       std::vector<int>& bad, int64_t* launches) {
  const int nm = (int)plan.size.size();
  std::vector<int32_t> order(ids);
  if (order.empty()) return cudaSuccess;
  const std::vector<int64_t>& bsize = plan.size;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bsize[a] > bsize[b]; });
  const int nb = (int)order.size();
  std::vector<int64_t> pt1(nb + 1, 0), pt3(nb + 1, 0), soff(nb + 1, 0);
  int64_t elems = 0;
  for (int a = 0; a < nb; ++a) {
    const int64_t n = bsize[order[a]];
    const int64_t nti = (n + GB - 1) / GB;
    pt1[a + 1] = pt1[a] + nti;
    const int64_t ntu = (n + UT - 1) / UT;
    pt3[a + 1] = pt3[a] + ntu * ntu;
    soff[a + 1] = soff[a] + n * GB;
    elems += n * f32_ld(n);
  }
  PoolScratch scratch(pool, s);
  cudaError_t e;
  float* mats = nullptr;
  if ((e = scratch.take(&mats, (size_t)elems)) != cudaSuccess) return e;
  std::vector<float*> fptr(nm, nullptr);
  int64_t off = 0;
  for (int a = 0; a < nb; ++a) {
    fptr[order[a]] = mats + off;
    off += bsize[order[a]] * f32_ld(bsize[order[a]]);
  }
  Bgj32Args args{};
  double** d_dptr = nullptr;
  float** d_fptr = nullptr;
  int64_t *d_bsize = nullptr, *d_pt1 = nullptr, *d_pt3 = nullptr, *d_soff = nullptr;
  int32_t* d_order = nullptr;
  if ((e = scratch.put(&d_dptr, plan.ptr)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_pt3, pt3)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_fptr, fptr)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_bsize, bsize)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_pt1, pt1)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_soff, soff)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_order, order)) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Pf, (size_t)nb * GB * GB)) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Cf, (size_t)soff[nb])) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Rf, (size_t)soff[nb])) != cudaSuccess) return e;
  if ((e = scratch.take(&args.flag, (size_t)nm)) != cudaSuccess) return e;
  cudaMemsetAsync(args.flag, 0, sizeof(int) * nm, s);
  args.Ap = d_fptr;
  args.bsize = d_bsize;
  args.order = d_order;
  args.pt1 = d_pt1;
  args.pt3 = d_pt3;
  args.soff = d_soff;
  if ((e = cudaFuncSetAttribute(bgj32_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UT_SMEM)) !=
      cudaSuccess)
    return e;
  const dim3 cgrid(std::min<unsigned>(1024u, (unsigned)((bsize[order[0]] * bsize[order[0]] + 255) / 256)),
                   (unsigned)nb);
  f64_to_f32_kernel<<<cgrid, 256, 0, s>>>(d_dptr, d_fptr, d_bsize, d_order);
  const int64_t nmax = bsize[order[0]];
  int active = nb;
  for (int64_t k0 = 0; k0 < nmax; k0 += GB) {
    while (active > 0 && bsize[order[active - 1]] <= k0) --active;
    bgj32_panel_kernel<<<(unsigned)pt1[active], 256, 0, s>>>(args, active, k0);
    bgj32_update_kernel<<<(unsigned)pt3[active], 256, UT_SMEM, s>>>(args, active, k0);
    *launches += 2;
  }
  f32_sym_to_f64_kernel<<<cgrid, 256, 0, s>>>(d_fptr, d_dptr, d_bsize, d_order);
  *launches += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::vector<int> h(nm, 0);
  if ((e = cudaMemcpyAsync(h.data(), args.flag, sizeof(int) * nm, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int m = 0; m < nm; ++m) bad[m] |= h[m];
  return cudaSuccess;
}

}  // namespace

// Order from which a matrix's double-float update runs on the tensor cores
// (the measured crossover of the two updates lies between 1536 and 2048).
constexpr int64_t kTcMinOrder = 2048;

// Inverts in place the matrices plan.inv lists (ids into plan.ptr / plan.size),
// all of them in one grouped sequence of launches: per 32-column step, the
// pivot, panel and update launches cover the tiles of every matrix still
// active (matrices sorted by order, largest first).  The double-float ones
// are equilibrated first (and unscaled after); the FP32 ones (plan.f32) go to
// invert_f32.  bad[m] = 1 for each id m
// whose recursion met a pivot that was not positive.
cudaError_t factor_invert(const InvPlan& plan, cudaMemPool_t pool, cudaStream_t s, std::vector<int>& bad,
                          int64_t* launches) {
  const int nm = (int)plan.size.size();
  bad.assign(nm, 0);
  std::vector<int32_t> order, order32;
  for (int32_t m : plan.inv)
    if (plan.size[m] > 0) (m < (int)plan.f32.size() && plan.f32[m] ? order32 : order).push_back(m);
  if (order.empty()) return invert_f32(plan, order32, pool, s, bad, launches);
  const std::vector<int64_t>& bsize = plan.size;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bsize[a] > bsize[b]; });
  const int nb = (int)order.size();
  std::vector<int64_t> pt1(nb + 1, 0), pt2(nb + 1, 0), soff(nb + 1, 0), pl(nb + 1, 0), pr(nb + 1, 0), ptc(nb + 1, 0);
  for (int a = 0; a < nb; ++a) {
    int64_t n = bsize[order[a]];
    int64_t nti = (n + GB - 1) / GB;
    pt1[a + 1] = pt1[a] + nti;
    pt2[a + 1] = pt2[a] + nti * nti;
    soff[a + 1] = soff[a] + n * GB;
    const int64_t tn = tcp_tile_cols();
    pl[a + 1] = pl[a] + (n + 127) / 128 * 128;
    pr[a + 1] = pr[a] + (n + tn - 1) / tn * tn;
    ptc[a + 1] = ptc[a] + ((n + 127) / 128) * ((n + tn - 1) / tn);
  }
  BgjArgs args{};
  double** d_ptr = nullptr;
  int64_t *d_bsize = nullptr, *d_pt1 = nullptr, *d_pt2 = nullptr, *d_soff = nullptr;
  int32_t* d_order = nullptr;
  PoolScratch scratch(pool, s);
  cudaError_t e;
  if ((e = scratch.put(&d_ptr, plan.ptr)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_bsize, bsize)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_pt1, pt1)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_pt2, pt2)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_soff, soff)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_order, order)) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Pf, (size_t)nb * GB * GB)) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Cf, (size_t)soff[nb])) != cudaSuccess) return e;
  if ((e = scratch.take(&args.Rf, (size_t)soff[nb])) != cudaSuccess) return e;
  if ((e = scratch.take(&args.flag, (size_t)nm)) != cudaSuccess) return e;
  cudaMemsetAsync(args.flag, 0, sizeof(int) * nm, s);
  args.Ap = d_ptr;
  args.bsize = d_bsize;
  args.order = d_order;
  args.pt1 = d_pt1;
  args.pt2 = d_pt2;
  args.soff = d_soff;
  // the rank-32 updates of the matrices of order >= kTcMinOrder on the
  // tensor cores (digit tiles and exponents of both operands made per step);
  // for smaller ones the three launches of a tensor-core update cost more
  // than the CUDA-core update saves
  int nbig = 0;
  while (nbig < nb && bsize[order[nbig]] >= kTcMinOrder) ++nbig;
  int sms = 0;
  if (nbig > 0 && (e = tcp_init(&sms)) != cudaSuccess) return e;
  TcpDev<double, float2> tc{};
  int64_t *d_pl = nullptr, *d_pr = nullptr, *d_ptc = nullptr;
  unsigned char* slices = nullptr;
  if ((e = scratch.put(&d_pl, pl)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_pr, pr)) != cudaSuccess) return e;
  if ((e = scratch.put(&d_ptc, ptc)) != cudaSuccess) return e;
  if ((e = scratch.take(&slices, tcp_slice_bytes(pl[nbig], pr[nbig]))) != cudaSuccess) return e;
  if ((e = scratch.take(&tc.exL, (size_t)pl[nbig])) != cudaSuccess) return e;
  if ((e = scratch.take(&tc.exR, (size_t)pr[nbig])) != cudaSuccess) return e;
  if ((e = scratch.take(&tc.err, 1)) != cudaSuccess) return e;
  cudaMemsetAsync(tc.err, 0, sizeof(int), s);
  tc.Ap = d_ptr;
  tc.bsize = d_bsize;
  tc.order = d_order;
  tc.soff = d_soff;
  tc.Pf = args.Pf;
  tc.Cf = args.Cf;
  tc.Rf = args.Rf;
  tc.pl = d_pl;
  tc.pr = d_pr;
  tc.pt = d_ptc;
  tc.Lsl = slices;
  tc.Rsl = slices + tcp_slice_bytes(pl[nbig], 0);
  // the power-of-two equilibration (prow: prefix of the orders)
  std::vector<int64_t> prow(nb + 1, 0);
  for (int a = 0; a < nb; ++a) prow[a + 1] = prow[a] + bsize[order[a]];
  int64_t* d_prow = nullptr;
  int* d_ex = nullptr;
  if ((e = scratch.put(&d_prow, prow)) != cudaSuccess) return e;
  if ((e = scratch.take(&d_ex, (size_t)prow[nb])) != cudaSuccess) return e;
  if (prow[nb] > 0x7fffffff) return cudaErrorInvalidValue;
  equil_exp_kernel<<<(unsigned)((prow[nb] + 255) / 256), 256, 0, s>>>(d_ptr, d_bsize, d_order, d_prow, nb, d_ex);
  equil_scale_kernel<<<(unsigned)prow[nb], 128, 0, s>>>(d_ptr, d_bsize, d_order, d_prow, nb, d_ex);
  *launches += 2;
  const int64_t nmax = bsize[order[0]];
  int active = nb;
  for (int64_t k0 = 0; k0 < nmax && e == cudaSuccess; k0 += GB) {
    while (active > 0 && bsize[order[active - 1]] <= k0) --active;
    bgj_pivot_kernel<<<active, GB * GB, 0, s>>>(args, k0);
    bgj_panel_kernel<<<(unsigned)pt1[active], 256, 0, s>>>(args, active, k0);
    // the matrices of order >= kTcMinOrder (sorted first) on the tensor
    // cores, the others on the CUDA cores: each matrix's arithmetic depends
    // on its own order only, whatever it is grouped with
    const int abig = std::min(active, nbig);
    *launches += 2;
    if (abig > 0) {
      e = launch_tcp_update(tc, abig, k0, pl[abig], pr[abig], ptc[abig], sms, s);
      *launches += 3;
    }
    if (active > abig) {
      bgj_update_kernel<<<(unsigned)(pt2[active] - pt2[abig]), 256, 0, s>>>(args, active, k0, pt2[abig]);
      *launches += 1;
    }
  }
  if (e != cudaSuccess) return e;
  equil_scale_kernel<<<(unsigned)prow[nb], 128, 0, s>>>(d_ptr, d_bsize, d_order, d_prow, nb, d_ex);
  *launches += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int h_err = 0;
  if ((e = cudaMemcpyAsync(&h_err, tc.err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  if (h_err) return cudaErrorTimeout;
  if ((e = cudaMemcpyAsync(bad.data(), args.flag, sizeof(int) * nm, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  return invert_f32(plan, order32, pool, s, bad, launches);
}

// Blocked Gauss-Jordan inversion of one SPD matrix A (n x n, row-major,
// device) in place, with all scratch (pivot block, the two panels, index
// arrays, breakdown flag) carved from the caller's device buffer `scratch` of
// `bytes` bytes; allocates nothing.  Needs bgj_scratch_bytes(n) bytes.
size_t bgj_scratch_bytes(int64_t n) {
  return sizeof(float2) * GB * GB + 2 * sizeof(float2) * (size_t)n * GB + 256;
}

cudaError_t bgj_invert_single(double* A, int64_t n, unsigned char* scratch, size_t bytes,
                              cudaStream_t s, int* not_spd) {
  *not_spd = 0;
  if (n < 1 || bytes < bgj_scratch_bytes(n)) return cudaErrorInvalidValue;
  const int64_t nti = (n + GB - 1) / GB;
  BgjArgs args{};
  args.Pf = (float2*)scratch;
  args.Cf = args.Pf + GB * GB;
  args.Rf = args.Cf + n * GB;
  int64_t* idx = (int64_t*)(args.Rf + n * GB);
  int32_t* tail = (int32_t*)(idx + 9);
  // ptr[1] bsize[1] pt1[2] pt2[2] soff[2] (one spare slot) | order[1] flag[1];
  // the matrix pointer travels as its 8 bytes in the first slot
  int64_t h_idx[9] = {0, n, 0, nti, 0, nti * nti, 0, n * GB, 0};
  static_assert(sizeof(double*) == sizeof(int64_t), "pointer slot");
  std::memcpy(&h_idx[0], &A, sizeof(double*));
  const int32_t h_tail[2] = {0, 0};
  args.Ap = (double* const*)idx;
  args.bsize = idx + 1;
  args.pt1 = idx + 2;
  args.pt2 = idx + 4;
  args.soff = idx + 6;
  args.order = tail;
  args.flag = tail + 1;
  cudaError_t e = cudaMemcpyAsync(idx, h_idx, sizeof(h_idx), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tail, h_tail, sizeof(h_tail), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  for (int64_t k0 = 0; k0 < n; k0 += GB) {
    bgj_pivot_kernel<<<1, GB * GB, 0, s>>>(args, k0);
    bgj_panel_kernel<<<(unsigned)nti, 256, 0, s>>>(args, 1, k0);
    bgj_update_kernel<<<(unsigned)(nti * nti), 256, 0, s>>>(args, 1, k0, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int flag = 0;
  e = cudaMemcpyAsync(&flag, args.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  *not_spd = flag;
  return cudaSuccess;
}

// Gathers face / wire-basket blocks and the coarse matrix A_H = P^T W P into
// g.d_binv and appends the matrices to invert to `plan` (owner: the tag the
// plan records for them).  bptr: block pointer (faces first, wire basket last
// if any).
cudaError_t factor_gather(DevGeom& g, const std::vector<int64_t>& bptr, int wb_diag, cudaStream_t s,
                          InvPlan& plan, int owner, int prec32) {
  const int nblk = (int)bptr.size() - 1;
  std::vector<int64_t> bsize(nblk + 1), boff(nblk + 2, 0), prefix2(nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) {
    bsize[b] = bptr[b + 1] - bptr[b];
    boff[b + 1] = boff[b] + bsize[b] * bsize[b];
    prefix2[b + 1] = prefix2[b] + bsize[b] * bsize[b];
  }
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  bsize[nblk] = NH;
  boff[nblk + 1] = boff[nblk] + NH * NH;
  cudaError_t e;
  if (g.d_binv) { cudaFreeAsync(g.d_binv, s); g.d_binv = nullptr; }
  if (g.d_boff) { cudaFreeAsync(g.d_boff, s); g.d_boff = nullptr; }
  g.binv_size = boff[nblk + 1];
  if ((e = pool_alloc((void**)&g.d_binv, sizeof(double) * std::max<int64_t>(1, g.binv_size), g.pool, s)) !=
      cudaSuccess)
    return e;
  if ((e = upload(&g.d_boff, boff, g.pool, s)) != cudaSuccess) return e;
  int64_t* d_prefix2 = nullptr;
  if ((e = upload(&d_prefix2, prefix2, g.pool, s)) != cudaSuccess) return e;
  const int wb_block = (g.n_blocks > 0 && g.wb_diag >= 0) ? nblk - 1 : -1;
  if (prefix2[nblk] > 0) ++g.launches;
  if (prefix2[nblk] > 0)
    gather_blocks_kernel<<<(unsigned)((prefix2[nblk] + 255) / 256), 256, 0, s>>>(
        g.d_Wh, g.wlo(), g.ldw, g.d_bptr, g.d_bdofs, g.d_boff, d_prefix2, nblk, wb_block, wb_diag, g.d_binv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaFreeAsync(d_prefix2, s);
  const int32_t base = (int32_t)plan.size.size();
  for (int b = 0; b <= nblk; ++b) {
    plan.ptr.push_back(g.d_binv + boff[b]);
    plan.size.push_back(bsize[b]);
    plan.owner.push_back(owner);
    plan.f32.push_back(prec32 && b < nblk ? 1 : 0);   // the coarse block stays double-float
  }
  for (int b = 0; b < nblk; ++b)
    if (!(wb_diag && b == wb_block) && bsize[b] > 0) plan.inv.push_back(base + b);
  if (NH > 0 && g.ndof > 0) {
    // A_H = P^T W P in the last slot
    dim3 grid((unsigned)((g.ndof + 255) / 256), (unsigned)NH);
    wp_kernel<<<grid, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, g.ndof, g.d_cptr, g.d_crow, g.d_cvalf, g.d_WP);
    dim3 grid2((unsigned)NH, (unsigned)((NH + 127) / 128));
    ah_kernel<<<grid2, 128, 0, s>>>(g.d_WP, g.ndof, NH, g.d_cptr, g.d_crow, g.d_cval,
                                    g.d_binv + boff[nblk]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    g.launches += 2;
    plan.inv.push_back(base + nblk);
  }
  return cudaSuccess;
}

// After the inversion: the float-pair copy of the face / wire-basket inverses
// and the 16-row tiles (block id, first row) of the multi-vector application.
cudaError_t factor_finish(DevGeom& g, const std::vector<int64_t>& bptr, cudaStream_t s) {
  const int nblk = (int)bptr.size() - 1;
  int64_t nf = 0;
  for (int b = 0; b < nblk; ++b) nf += (bptr[b + 1] - bptr[b]) * (bptr[b + 1] - bptr[b]);
  cudaError_t e;
  if (g.d_binvf) { cudaFreeAsync(g.d_binvf, s); g.d_binvf = nullptr; }
  if ((e = pool_alloc((void**)&g.d_binvf, sizeof(float2) * std::max<int64_t>(1, nf), g.pool, s)) !=
      cudaSuccess)
    return e;
  if (nf > 0) {
    to_float_pairs_kernel<<<(unsigned)std::min<int64_t>((nf + 255) / 256, 152 * 32), 256, 0, s>>>(
        g.d_binv, g.d_binvf, nf);
    ++g.launches;
  }
  std::vector<int32_t> tiles;
  for (int b = 0; b < nblk; ++b)
    for (int64_t r0 = 0; r0 < bptr[b + 1] - bptr[b]; r0 += 16) {
      tiles.push_back(b);
      tiles.push_back((int32_t)r0);
    }
  if (g.d_btile) { cudaFreeAsync(g.d_btile, s); g.d_btile = nullptr; }
  g.n_btiles = (int64_t)tiles.size() / 2;
  if ((e = upload(&g.d_btile, tiles, g.pool, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t factor_blocks(DevGeom& g, const std::vector<int64_t>& bptr, int wb_diag, cudaStream_t s,
                          int* not_spd, int prec32) {
  *not_spd = 0;
  InvPlan plan;
  cudaError_t e = factor_gather(g, bptr, wb_diag, s, plan, 0, prec32);
  if (e != cudaSuccess) return e;
  std::vector<int> bad;
  if ((e = factor_invert(plan, g.pool, s, bad, &g.launches)) != cudaSuccess) return e;
  for (int v : bad) *not_spd |= v;
  return factor_finish(g, bptr, s);
}

}  // namespace msbem
