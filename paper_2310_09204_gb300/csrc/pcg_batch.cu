// Block PCG: k independent right-hand sides on one geometry (for instance k
// Neumann data g on a cached W), each column following exactly the PCG
// recursion of pcg.cu (Sec. 2.1, Remark "Bound on the number of PCG
// iterations") with its own scalars and stopping test, while the columns share
// one pass over W per iteration:
//
//   Q = W P  (N x k), one read of W for all k columns (matvec.cu), double-float
//   on the FP32 pipe (13 k FP32 operations per element of W);
//   the preconditioner applies each block inverse to all k columns at once.
//
// Vectors are stored row-major N x KB (KB = columns of this pass, <= 16).
// A column that has converged (or broken down) stops updating; the pass ends
// when every column is done.
#include <cmath>
#include <cstddef>
#include <vector>

#include "batch.cuh"
#include "df.cuh"

namespace msbem {

// per-column partial sums of a_c . b_c  (part: kb x BRED)
__global__ void bdot_kernel(const double* __restrict__ A, const double* __restrict__ B, int64_t N,
                            int kb, double* __restrict__ part, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[256];
  const int c = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
    acc = fma(A[i * kb + c], B[i * kb + c], acc);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)c * gridDim.x + blockIdx.x] = s[0];
}

// fixed-order reduction of each column's partial sums into the field at
// byte offset `field` of its ColState
__global__ void breduce_kernel(const double* __restrict__ part, int nparts, ColState* cs, int field,
                               const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += part[(int64_t)c * nparts + i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *(double*)((char*)&cs[c] + field) = s[0];
}

// alpha_c = rz_c / pq_c (breakdown check), per active column
__global__ void balpha_kernel(ColState* cs, double* alpha_hist, int hcap, const BatchState* bs) {
  if (bs->all_done) return;
  const int c = threadIdx.x;
  if (c >= bs->kb || !col_active(cs, c)) return;
  const double pq = cs[c].pq, a = cs[c].rz / pq;
  if (!(pq > 0.0) || !isfinite(a)) {
    cs[c].done = 2;
    return;
  }
  cs[c].alpha = a;
  alpha_hist[(int64_t)c * hcap + cs[c].iter] = a;
}

// x_c += alpha_c p_c; r_c -= alpha_c q_c; per-column partial r.r
// Rf (may be null): the residual's float-pair split, written beside it for
// the block solves of the preconditioner that follow
__global__ void bupdate_xr_kernel(double* __restrict__ X, double* __restrict__ R,
                                  const double* __restrict__ P, const double* __restrict__ Q, int64_t N,
                                  int kb, const ColState* __restrict__ cs, double* __restrict__ part,
                                  float2* __restrict__ Rf, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[256];
  const int c = blockIdx.y;
  const bool act = col_active(cs, c);
  const double alpha = cs[c].alpha;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    const int64_t o = i * kb + c;
    double ri = R[o];
    if (act) {
      X[o] = fma(alpha, P[o], X[o]);
      ri = fma(-alpha, Q[o], ri);
      R[o] = ri;
    }
    if (Rf) {
      float h, l;
      split_df(ri, h, l);
      Rf[o] = make_float2(h, l);
    }
    acc = fma(ri, ri, acc);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)c * gridDim.x + blockIdx.x] = s[0];
}

// per-column stopping test; all_done when every column is done
__global__ void bcheck_kernel(ColState* cs, double* hist, int hcap, BatchState* bs) {
  if (bs->all_done) return;
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  const int c = threadIdx.x;
  if (c < bs->kb) {
    if (col_active(cs, c)) {
      const double rel = sqrt(cs[c].rr / cs[c].nL2);
      const int it = cs[c].iter + 1;
      cs[c].iter = it;
      hist[(int64_t)c * (hcap + 1) + it] = rel;
      if (bs->err) cs[c].done = 5;
      else if (!isfinite(rel)) cs[c].done = 2;
      else if (!bs->fixed && rel <= bs->rtol) cs[c].done = 1;
      else if (it >= bs->maxit) cs[c].done = (bs->fixed || rel <= bs->rtol) ? 1 : 3;
    }
    if (col_active(cs, c)) atomicAdd(&s_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_active == 0) bs->all_done = 1;
}

// float-pair copy of an N x kb block
__global__ void bto_df_kernel(const double* __restrict__ X, float2* __restrict__ Xf, int64_t n,
                              const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    float h, l;
    split_df(X[i], h, l);
    Xf[i] = make_float2(h, l);
  }
}

// Z[D_b[i]][c] = sum_j Ainv_b[i][j] R[D_b[j]][c] for all columns, in
// double-float.  One CTA per 16-row tile of a block (two rows per warp); the
// block's residual rows are gathered chunk by chunk (128 dofs x kb columns)
// into shared memory, transposed and split into hi / lo planes, so each is
// read from L2 once per tile instead of once per row; lane l takes the chunk's
// dofs 4l .. 4l+3.  F32: the hi parts of the inverses and of the residual
// only, plain FP32 accumulation (inner solves of the iterative refinement).
#define BA_KC 128
#define BA_PAD 132   // row pitch of the staged planes (keeps float4 reads aligned, staging 2-way)
template <bool F32>
__device__ __forceinline__ void block_tile_body(int tile, const float2* __restrict__ Ainv,
                                                const int64_t* __restrict__ boff,
                                                const int64_t* __restrict__ bptr,
                                                const int32_t* __restrict__ bdofs,
                                                const int32_t* __restrict__ tiles,
                                                const float2* __restrict__ Rf, double* __restrict__ Z,
                                                int kb, float* sRh, float* sRl) {
  const int b = tiles[2 * tile];
  const int64_t r0 = tiles[2 * tile + 1];
  const int64_t n = bptr[b + 1] - bptr[b];
  const int32_t* d = bdofs + bptr[b];
  const float2* A = Ainv + boff[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i0 = r0 + 2 * wid;
  const bool ok0 = i0 < n, ok1 = i0 + 1 < n;
  const float2* a0 = A + (ok0 ? i0 : 0) * n;
  const float2* a1 = A + (ok1 ? i0 + 1 : 0) * n;
  float h[2][BK], l[2][BK];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < BK; ++c) { h[r][c] = 0.f; l[r][c] = 0.f; }
  for (int64_t j0 = 0; j0 < n; j0 += BA_KC) {
    const int len = (int)((n - j0) < BA_KC ? (n - j0) : BA_KC);
    // this chunk's inverse entries first, so their latency overlaps the staging
    float2 w0[4], w1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = 4 * lane + q;
      const bool in = jj < len;
      w0[q] = (ok0 && in) ? a0[j0 + jj] : make_float2(0.f, 0.f);
      w1[q] = (ok1 && in) ? a1[j0 + jj] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BA_KC * kb; e += 256) {
      const int jj = e / kb, c = e - jj * kb;
      float2 v = make_float2(0.f, 0.f);
      if (jj < len) v = Rf[(int64_t)d[j0 + jj] * kb + c];
      sRh[c * BA_PAD + jj] = v.x;
      sRl[c * BA_PAD + jj] = v.y;
    }
    __syncthreads();
    if (F32) {
#pragma unroll
      for (int c = 0; c < BK; ++c) {
        if (c < kb) {
          const float4 rh = *(const float4*)(sRh + c * BA_PAD + 4 * lane);
          h[0][c] = fmaf(w0[0].x, rh.x, h[0][c]);
          h[1][c] = fmaf(w1[0].x, rh.x, h[1][c]);
          l[0][c] = fmaf(w0[1].x, rh.y, l[0][c]);
          l[1][c] = fmaf(w1[1].x, rh.y, l[1][c]);
          h[0][c] = fmaf(w0[2].x, rh.z, h[0][c]);
          h[1][c] = fmaf(w1[2].x, rh.z, h[1][c]);
          l[0][c] = fmaf(w0[3].x, rh.w, l[0][c]);
          l[1][c] = fmaf(w1[3].x, rh.w, l[1][c]);
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < BK; ++c) {
        if (c < kb) {
          const float4 rh = *(const float4*)(sRh + c * BA_PAD + 4 * lane);
          const float4 rl = *(const float4*)(sRl + c * BA_PAD + 4 * lane);
          df_fma_acc(w0[0].x, w0[0].y, rh.x, rl.x, h[0][c], l[0][c]);
          df_fma_acc(w1[0].x, w1[0].y, rh.x, rl.x, h[1][c], l[1][c]);
          df_fma_acc(w0[1].x, w0[1].y, rh.y, rl.y, h[0][c], l[0][c]);
          df_fma_acc(w1[1].x, w1[1].y, rh.y, rl.y, h[1][c], l[1][c]);
          df_fma_acc(w0[2].x, w0[2].y, rh.z, rl.z, h[0][c], l[0][c]);
          df_fma_acc(w1[2].x, w1[2].y, rh.z, rl.z, h[1][c], l[1][c]);
          df_fma_acc(w0[3].x, w0[3].y, rh.w, rl.w, h[0][c], l[0][c]);
          df_fma_acc(w1[3].x, w1[3].y, rh.w, rl.w, h[1][c], l[1][c]);
        }
      }
    }
  }
  // the 2 rows x 16 vectors of sums at once (transposed butterfly: 31
  // shuffles, each sum over the same lane pairs as a plain butterfly); lane L
  // ends with the sum of row L / 16, vector L % 16
  float* hh = &h[0][0];
  float* ll = &l[0][0];
  if (F32) {
#pragma unroll
    for (int v = 0; v < 2 * BK; ++v) hh[v] += ll[v];
  }
  warp_xreduce<2 * BK, 16, !F32>(hh, ll, lane);
  {
    const int r = lane / BK, c = lane % BK;
    const bool ok = r == 0 ? ok0 : ok1;
    if (ok && c < kb) Z[(int64_t)d[i0 + r] * kb + c] = F32 ? (double)hh[0] : df_to_double(hh[0], ll[0]);
  }
}

template <bool F32>
__global__ void __launch_bounds__(256) bblock_tile_kernel(const float2* __restrict__ Ainv,
                                                          const int64_t* __restrict__ boff,
                                                          const int64_t* __restrict__ bptr,
                                                          const int32_t* __restrict__ bdofs,
                                                          const int32_t* __restrict__ tiles,
                                                          const float2* __restrict__ Rf,
                                                          double* __restrict__ Z, int kb,
                                                          const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ __align__(16) float sRh[BK * BA_PAD];
  __shared__ __align__(16) float sRl[BK * BA_PAD];
  block_tile_body<F32>(blockIdx.x, Ainv, boff, bptr, bdofs, tiles, Rf, Z, kb, sRh, sRl);
}

// T[mu][c] = sum_k P[row_k, mu] R[row_k][c]  (block per coarse dof)
__device__ __forceinline__ void restrict_body(int64_t mu, const int64_t* __restrict__ cptr,
                                              const int32_t* __restrict__ crow, const double* __restrict__ cval,
                                              const double* __restrict__ R, int kb, double* __restrict__ T,
                                              double (*s)[BK]) {
  double acc[BK];
#pragma unroll
  for (int c = 0; c < BK; ++c) acc[c] = 0.0;
  for (int64_t k = cptr[mu] + threadIdx.x; k < cptr[mu + 1]; k += blockDim.x) {
    const double v = cval[k];
    const double* r = R + (int64_t)crow[k] * kb;
#pragma unroll
    for (int c = 0; c < BK; ++c)
      if (c < kb) acc[c] = fma(v, r[c], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < BK; ++c) {
    double v = acc[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kb) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s[w][threadIdx.x];
    T[mu * kb + threadIdx.x] = v;
  }
}

__global__ void brestrict_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                 const double* __restrict__ cval, const double* __restrict__ R, int kb,
                                 double* __restrict__ T, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[8][BK];
  restrict_body(blockIdx.x, cptr, crow, cval, R, kb, T, s);
}

// The subspace solves and the coarse restriction in one launch: CTAs below
// ntiles apply the block inverses to their tiles, the others restrict the
// residual onto one coarse dof each (the two read the residual and write
// disjoint outputs).
template <bool F32>
__global__ void __launch_bounds__(256) bblock_restrict_kernel(
    const float2* __restrict__ Ainv, const int64_t* __restrict__ boff, const int64_t* __restrict__ bptr,
    const int32_t* __restrict__ bdofs, const int32_t* __restrict__ tiles, int ntiles,
    const float2* __restrict__ Rf, double* __restrict__ Z, int kb, const int64_t* __restrict__ cptr,
    const int32_t* __restrict__ crow, const double* __restrict__ cval, const double* __restrict__ R,
    double* __restrict__ T, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ __align__(16) float sRh[BK * BA_PAD];
  __shared__ __align__(16) float sRl[BK * BA_PAD];
  if ((int)blockIdx.x < ntiles) {
    block_tile_body<F32>(blockIdx.x, Ainv, boff, bptr, bdofs, tiles, Rf, Z, kb, sRh, sRl);
  } else {
    restrict_body((int64_t)blockIdx.x - ntiles, cptr, crow, cval, R, kb, T, (double (*)[BK])sRh);
  }
}

// U = AHinv T  (thread per (row, column))
__global__ void bcoarse_kernel(const double* __restrict__ AHinv, int64_t NH, const double* __restrict__ T,
                               int kb, double* __restrict__ U, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NH * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  double acc = 0.0;
  for (int64_t j = 0; j < NH; ++j) acc = fma(AHinv[i * NH + j], T[j * kb + c], acc);
  U[i * kb + c] = acc;
}

// Z[i][c] += sum P[i, mu] U[mu][c]
__global__ void bprolong_kernel(const int64_t* __restrict__ pptr, const int32_t* __restrict__ pcol,
                                const double* __restrict__ pval, int64_t N, const double* __restrict__ U,
                                int kb, double* __restrict__ Z, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  double acc = 0.0;
  for (int64_t k = pptr[i]; k < pptr[i + 1]; ++k) acc = fma(pval[k], U[(int64_t)pcol[k] * kb + c], acc);
  Z[e] += acc;
}

// Z[i][c] += sum P[i, mu] U[mu][c], and the per-block partial sums of
// R[:, c] . Z[:, c] over the same row partition as bdot_kernel (the coarse
// prolongation fused with the r.z reduction that follows it; the same
// arithmetic in the same order as the two kernels)
__global__ void bprolong_dot_kernel(const int64_t* __restrict__ pptr, const int32_t* __restrict__ pcol,
                                    const double* __restrict__ pval, int64_t N, const double* __restrict__ U,
                                    int kb, double* __restrict__ Z, const double* __restrict__ R,
                                    double* __restrict__ part, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[256];
  const int c = blockIdx.y;
  double dot = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    const int64_t o = i * kb + c;
    double acc = 0.0;
    for (int64_t k = pptr[i]; k < pptr[i + 1]; ++k) acc = fma(pval[k], U[(int64_t)pcol[k] * kb + c], acc);
    const double z = Z[o] + acc;
    Z[o] = z;
    dot = fma(R[o], z, dot);
  }
  s[threadIdx.x] = dot;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)c * gridDim.x + blockIdx.x] = s[0];
}

__global__ void bcopy_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t n,
                             const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256)
    dst[i] = src[i];
}

// beta_c = rz_new_c / rz_c; rz_c = rz_new_c (active columns)
__global__ void bbeta_kernel(ColState* cs, double* beta_hist, int hcap, const BatchState* bs) {
  if (bs->all_done) return;
  const int c = threadIdx.x;
  if (c >= bs->kb || !col_active(cs, c)) return;
  const double b = cs[c].rz_new / cs[c].rz;
  cs[c].beta = b;
  cs[c].rz = cs[c].rz_new;
  beta_hist[(int64_t)c * hcap + cs[c].iter - 1] = b;
}

// p_c = z_c + beta_c p_c (active columns) and its float-pair copy, stored
// transposed as planes Pf[plane][c][i] (plane 0 hi, 1 lo; leading dimension ldp)
__global__ void bupdate_p_kernel(double* __restrict__ P, float* __restrict__ Pf, int64_t ldp,
                                 const double* __restrict__ Z, int64_t N, int kb,
                                 const ColState* __restrict__ cs, int first,
                                 const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256) {
    const int64_t i = e / kb;
    const int c = (int)(e - i * kb);
    double v;
    if (first) v = Z[e];
    else if (col_active(cs, c)) v = fma(cs[c].beta, P[e], Z[e]);
    else v = P[e];
    P[e] = v;
    float h, l;
    split_df(v, h, l);
    Pf[(int64_t)c * ldp + i] = h;
    Pf[(int64_t)(kb + c) * ldp + i] = l;
  }
}

// R[i][c] = L_c[i] for constant data g_c (rows of the curl/RHS lists)
__global__ void brhs_kernel(const int64_t* __restrict__ jptr, const double* __restrict__ jrhs, int64_t N,
                            const double* __restrict__ gv, int kb, double* __restrict__ R) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  double acc = 0.0;
  for (int64_t k = jptr[i]; k < jptr[i + 1]; ++k)
    acc += jrhs[3 * k] * gv[3 * c] + jrhs[3 * k + 1] * gv[3 * c + 1] + jrhs[3 * k + 2] * gv[3 * c + 2];
  R[e] = acc;
}

// X_out[c][i] = X[i][c]
__global__ void btranspose_kernel(const double* __restrict__ X, int64_t N, int kb, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  out[(int64_t)c * N + i] = X[e];
}


void apply_M_batch(DevGeom& g, const BatchBuffers& b, int kb, int precondition, int f32, cudaStream_t s,
                   bool in_iteration) {
  const int64_t N = g.ndof;
  const dim3 rgrid(BRED, kb);
  if (!precondition) {
    bcopy_kernel<<<kStrideBlocks, 256, 0, s>>>(b.Z, b.R, N * kb, b.bs);
    ++g.launches;
    if (in_iteration) {
      bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.Z, N, kb, b.part, b.bs);
      ++g.launches;
    }
    return;
  }
  // in an iteration the residual's float-pair split was written by the update
  if (!in_iteration) {
    bto_df_kernel<<<kStrideBlocks, 256, 0, s>>>(b.R, b.Rf, N * kb, b.bs);
    ++g.launches;
  }
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  // block solves and coarse restriction: one launch
  const unsigned nt = (unsigned)g.n_btiles, grid = nt + (unsigned)NH;
  if (grid > 0) {
    if (f32)
      bblock_restrict_kernel<true><<<grid, 256, 0, s>>>(g.d_binvf, g.d_boff, g.d_bptr, g.d_bdofs, g.d_btile, (int)nt,
                                                        b.Rf, b.Z, kb, g.d_cptr, g.d_crow, g.d_cval, b.R, b.T, b.bs);
    else
      bblock_restrict_kernel<false><<<grid, 256, 0, s>>>(g.d_binvf, g.d_boff, g.d_bptr, g.d_bdofs, g.d_btile,
                                                         (int)nt, b.Rf, b.Z, kb, g.d_cptr, g.d_crow, g.d_cval, b.R,
                                                         b.T, b.bs);
    ++g.launches;
  }
  if (NH > 0) {
    bcoarse_kernel<<<(unsigned)((NH * kb + 127) / 128), 128, 0, s>>>(g.d_AHinv, NH, b.T, kb, b.U, b.bs);
    if (in_iteration)
      bprolong_dot_kernel<<<rgrid, 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, b.U, kb, b.Z, b.R, b.part, b.bs);
    else
      bprolong_kernel<<<(unsigned)((N * kb + 255) / 256), 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, b.U,
                                                                        kb, b.Z, b.bs);
    g.launches += 2;
  } else if (in_iteration) {
    bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.Z, N, kb, b.part, b.bs);
    ++g.launches;
  }
}

// ---- small kernels of the drivers ------------------------------------------
// out[c] = sum of the nparts partial sums of column c (fixed order)
__global__ void bsum_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double sm[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) acc += part[(int64_t)c * nparts + i];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sm[0];
}

// Rm = R with the columns flagged in skip[] set to zero
__global__ void bmask_kernel(const double* __restrict__ R, int64_t n, int kb, const int* __restrict__ skip,
                             double* __restrict__ Rm) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
    Rm[e] = skip[e % kb] ? 0.0 : R[e];
}

// X += D
__global__ void baxpy_kernel(double* __restrict__ X, const double* __restrict__ D, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
    X[e] += D[e];
}

// float-pair planes of an N x kb block, transposed: Xf[plane][c][i]
__global__ void bsplit_kernel(const double* __restrict__ X, float* __restrict__ Xf, int64_t ldp, int64_t N,
                              int kb) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < N * kb; e += (int64_t)gridDim.x * 256) {
    const int64_t i = e / kb;
    const int c = (int)(e - i * kb);
    float h, l;
    split_df(X[e], h, l);
    Xf[(int64_t)c * ldp + i] = h;
    Xf[(int64_t)(kb + c) * ldp + i] = l;
  }
}

// R = L - Q
__global__ void bresid_kernel(const double* __restrict__ L, const double* __restrict__ Q, int64_t n,
                              double* __restrict__ R) {
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
    R[e] = L[e] - Q[e];
}


void enqueue_batch_iteration(DevGeom& g, const BatchBuffers& b, int kb, int precondition, int mv_mode,
                             const CUtensorMap& tmP, int split, void* scratch, int hcap, cudaStream_t s) {
  const int64_t N = g.ndof;
  const dim3 rgrid(BRED, kb);
  double* rel_h = b.hist;
  double* alpha_h = rel_h + (size_t)kb * (hcap + 1);
  double* beta_h = alpha_h + (size_t)kb * hcap;
  if (mv_mode >= 3) {
    launch_matvec_tc(g, mv_mode - 3, kb, b.P, b.Q, b.part, &b.bs->all_done, &b.bs->err, scratch, s);
  } else {
    const CUtensorMap& tmW = mv_mode == 0 ? g.tm_W : g.tm_Whi;
    launch_matvec(mv_mode, tmW, tmP, N, kb, b.P, b.Q, b.part, &b.bs->all_done, &b.bs->err, s, split, scratch);
  }
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, (int)matvec_blocks(N, mv_mode == 1 ? 1 : 0), b.cs,
                                    offsetof(ColState, pq), b.bs);
  balpha_kernel<<<1, BK, 0, s>>>(b.cs, alpha_h, hcap, b.bs);
  bupdate_xr_kernel<<<rgrid, 256, 0, s>>>(b.X, b.R, b.P, b.Q, N, kb, b.cs, b.part, precondition ? b.Rf : nullptr,
                                          b.bs);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rr), b.bs);
  bcheck_kernel<<<1, 32, 0, s>>>(b.cs, rel_h, hcap, b.bs);
  // z = M r and the partial sums of r . z (its last launch carries them)
  apply_M_batch(g, b, kb, precondition, mv_mode == 1 || mv_mode == 4, s, true);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rz_new), b.bs);
  bbeta_kernel<<<1, BK, 0, s>>>(b.cs, beta_h, hcap, b.bs);
  bupdate_p_kernel<<<kStrideBlocks, 256, 0, s>>>(b.P, b.Pf, g.ldw, b.Z, N, kb, b.cs, 0, b.bs);
  g.launches += mv_mode >= 3 ? 8 : 9 + (split > 1 ? 1 : 0);   // (the tensor-core product counts its own)
}

// PCG from X = 0 on the kb right-hand sides Rin (device, N x kb row-major);
// the iterates are written to X (device, N x kb).  mv_mode 0: double-float
// products with W; 1: FP32 products with the hi plane (inner solves of the
// iterative refinement); 3: double-float products on the tensor cores; 4:
// scaled-FP16 products on the tensor cores (inner solves).  The block inverses
// are applied in FP32 with modes 1 and 4, in double-float otherwise.  Each
// column's relative residual is measured against its own ||Rin_c||.
static cudaError_t pcg_batch_core(DevGeom& g, int kb, double rtol, int maxit, int fixed, int precondition,
                                  int mv_mode, const double* Rin, double* X, std::vector<PcgOut>& outs,
                                  cudaStream_t s) {
  const int64_t N = g.ndof;
  outs.assign(kb, PcgOut());
  const int64_t NH = std::max<int64_t>(g.n_coarse, 1);
  const bool tc = mv_mode >= 3;
  cudaError_t e;
  if (tc && (e = ensure_w_slices(g, mv_mode - 3, s)) != cudaSuccess) return e;
  const unsigned gemv_blocks = matvec_blocks(N, mv_mode == 1 ? 1 : 0);
  const size_t nvec = (size_t)N * kb;
  const size_t nparts = (size_t)kb * std::max<unsigned>(gemv_blocks, BRED);
  const size_t hsz = (size_t)kb * (maxit + 1) + 2 * (size_t)kb * maxit;
  const int split = tc ? 1 : matvec_split_of(g, mv_mode);
  const size_t scr_bytes = tc ? tc_work_bytes(g) : matvec_scratch_bytes(N, kb, split);
  const size_t bytes = sizeof(double) * (4 * nvec + 2 * NH * kb + nparts + hsz) +
                       sizeof(float) * 2 * kb * g.ldw + sizeof(float2) * nvec + sizeof(ColState) * kb +
                       sizeof(BatchState) + scr_bytes + 512;
  char* base = nullptr;
  if ((e = pool_alloc((void**)&base, bytes, g.pool, s)) != cudaSuccess) return e;
  Carver cv{base};
  BatchBuffers b;
  b.X = X;
  b.R = cv.take<double>(nvec);
  b.Z = cv.take<double>(nvec);
  b.P = cv.take<double>(nvec);
  b.Q = cv.take<double>(nvec);
  b.T = cv.take<double>(NH * kb);
  b.U = cv.take<double>(NH * kb);
  b.part = cv.take<double>(nparts);
  b.hist = cv.take<double>(hsz);
  b.gv = nullptr;
  b.Pf = cv.take<float>(2 * kb * g.ldw);
  b.Rf = cv.take<float2>(nvec);
  b.cs = cv.take<ColState>(kb);
  b.bs = cv.take<BatchState>(1);
  char* scratch = cv.take<char>(scr_bytes);
  std::vector<ColState> h_cs(kb);
  for (auto& c : h_cs) c = ColState{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  BatchState h_bs{0, kb, maxit, fixed, rtol, 0};
  CUtensorMap tmP;   // the FP32 planes of P read by the CUDA-core products
  const int planes = mv_mode == 1 ? 1 : 2;
  if ((e = encode_planes(&tmP, b.Pf, g.ldw, kb, kb * g.ldw, planes, matvec_pad(kb))) != cudaSuccess) {
    cudaFreeAsync(base, s);
    return e;
  }
  cudaMemsetAsync(b.Pf, 0, sizeof(float) * 2 * kb * g.ldw, s);
  cudaMemcpyAsync(b.cs, h_cs.data(), sizeof(ColState) * kb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b.bs, &h_bs, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(b.X, 0, sizeof(double) * nvec, s);
  cudaMemcpyAsync(b.R, Rin, sizeof(double) * nvec, cudaMemcpyDeviceToDevice, s);
  const dim3 rgrid(BRED, kb);
  bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.R, N, kb, b.part, b.bs);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, nL2), b.bs);
  apply_M_batch(g, b, kb, precondition, mv_mode == 1 || mv_mode == 4, s, false);
  bupdate_p_kernel<<<kStrideBlocks, 256, 0, s>>>(b.P, b.Pf, g.ldw, b.Z, N, kb, b.cs, 1, b.bs);
  bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.Z, N, kb, b.part, b.bs);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rz), b.bs);
  g.launches += 6;
  // columns with zero data are finished before the first iteration
  auto drop = [&](cudaError_t err) {  // error exit: the buffer goes back to the pool
    cudaFreeAsync(base, s);
    return err;
  };
  if ((e = cudaMemcpyAsync(h_cs.data(), b.cs, sizeof(ColState) * kb, cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return drop(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
  int zero_cols = 0;
  for (int c = 0; c < kb; ++c)
    if (h_cs[c].nL2 == 0.0) {
      h_cs[c].done = 4;  // marks "no data": solution 0, no iterations
      ++zero_cols;
    }
  if (zero_cols) {
    if (zero_cols == kb) h_bs.all_done = 1;
    cudaMemcpyAsync(b.cs, h_cs.data(), sizeof(ColState) * kb, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b.bs, &h_bs, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  }
  int enq = 0;
  while (enq < maxit && !h_bs.all_done) {
    const int chunk = std::min(4, maxit - enq);
    for (int it = 0; it < chunk; ++it)
      enqueue_batch_iteration(g, b, kb, precondition, mv_mode, tmP, split, scratch, maxit, s);
    enq += chunk;
    if ((e = cudaGetLastError()) != cudaSuccess) return drop(e);
    if ((e = cudaMemcpyAsync(&h_bs, b.bs, sizeof(BatchState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return drop(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
  }
  std::vector<double> h(hsz);
  cudaMemcpyAsync(h.data(), b.hist, sizeof(double) * hsz, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_cs.data(), b.cs, sizeof(ColState) * kb, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(base, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int c = 0; c < kb; ++c) {
    PcgOut& o = outs[c];
    const int it = h_cs[c].iter;
    o.iters = it;
    o.hist.assign(1, h_cs[c].done == 4 ? 0.0 : 1.0);
    for (int k = 1; k <= it; ++k) o.hist.push_back(h[(size_t)c * (maxit + 1) + k]);
    o.alpha.assign(h.begin() + (size_t)kb * (maxit + 1) + (size_t)c * maxit,
                   h.begin() + (size_t)kb * (maxit + 1) + (size_t)c * maxit + it);
    const int nbeta = it - 1;  // the Lanczos matrix of `it` steps uses it - 1 betas
    const size_t boff_ = (size_t)kb * (maxit + 1) + (size_t)kb * maxit + (size_t)c * maxit;
    o.beta.assign(h.begin() + boff_, h.begin() + boff_ + std::max(0, nbeta));
    const int d = h_cs[c].done;
    o.status = d == 5 ? MSBEM_DEVICE_TIMEOUT
             : d == 2 ? MSBEM_BREAKDOWN
             : (d == 3 || d == 0) ? MSBEM_NOT_CONVERGED
                                  : MSBEM_OK;
  }
  return cudaSuccess;
}

// densities out: column c of X (row-major N x kb) -> X_out[c][i]
static cudaError_t copy_out(DevGeom& g, const double* X, int64_t N, int kb, double* X_out, bool on_device,
                            cudaStream_t s) {
  if (!X_out) return cudaSuccess;
  const size_t nvec = (size_t)N * kb;
  if (on_device) {
    btranspose_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(X, N, kb, X_out);
    ++g.launches;
    return cudaStreamSynchronize(s);
  }
  std::vector<double> xh(nvec);
  cudaMemcpyAsync(xh.data(), X, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < kb; ++c)
    for (int64_t i = 0; i < N; ++i) X_out[(size_t)c * N + i] = xh[(size_t)i * kb + c];
  return cudaSuccess;
}

// L (N x kb) for the data g_c
static cudaError_t batch_rhs(DevGeom& g, const double* gvecs, int kb, double* gv_dev, double* L, cudaStream_t s) {
  const size_t nvec = (size_t)g.ndof * kb;
  cudaMemcpyAsync(gv_dev, gvecs, sizeof(double) * 3 * kb, cudaMemcpyHostToDevice, s);
  brhs_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(g.d_jptr, g.d_jrhs, g.ndof, gv_dev, kb, L);
  ++g.launches;
  return cudaGetLastError();
}

cudaError_t run_pcg_batch(DevGeom& g, const double* gvecs, int kb, double rtol, int maxit, int fixed,
                          int precondition, double* X_out, bool out_on_device, std::vector<PcgOut>& outs,
                          cudaStream_t s, int tensor) {
  const int64_t N = g.ndof;
  outs.assign(kb, PcgOut());
  if (kb < 1 || kb > BK) return cudaErrorInvalidValue;
  if (N == 0) {
    for (auto& o : outs) { o.hist.push_back(0.0); o.status = MSBEM_OK; }
    return cudaStreamSynchronize(s);
  }
  const size_t nvec = (size_t)N * kb;
  char* base = nullptr;
  cudaError_t e = pool_alloc((void**)&base, sizeof(double) * (2 * nvec + 3 * kb) + 64, g.pool, s);
  if (e != cudaSuccess) return e;
  Carver cv{base};
  double* L = cv.take<double>(nvec);
  double* X = cv.take<double>(nvec);
  double* gv = cv.take<double>(3 * kb);
  if ((e = batch_rhs(g, gvecs, kb, gv, L, s)) == cudaSuccess)
    e = pcg_batch_core(g, kb, rtol, maxit, fixed, precondition, tensor ? 3 : 0, L, X, outs, s);
  if (e == cudaSuccess) e = copy_out(g, X, N, kb, X_out, out_on_device, s);
  cudaFreeAsync(base, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : e2;
}

// Mixed precision (iterative refinement): the correction equation W D = R is
// solved by the PCG above with FP32 products (hi plane of W) to the relative
// tolerance inner_rtol, X += D, and the residual R = L - W X is recomputed
// with the double-float product, until ||R_c|| <= rtol ||L_c|| for every
// column.  tensor: the residual's double-float product on the tensor cores;
// inner_fp16: the inner products in scaled FP16 on the tensor cores.  Reported per column: the inner iterations summed, the true relative
// residual after every refinement step (hist), and the Lanczos coefficients
// of the first inner solve.
cudaError_t run_ir_batch(DevGeom& g, const double* gvecs, int kb, double rtol, int maxit, double inner_rtol,
                         int precondition, double* X_out, bool out_on_device, std::vector<PcgOut>& outs,
                         int* refinements, cudaStream_t s, int tensor, int inner_fp16, double density_tol) {
  const int64_t N = g.ndof;
  outs.assign(kb, PcgOut());
  if (refinements) *refinements = 0;
  if (kb < 1 || kb > BK) return cudaErrorInvalidValue;
  if (N == 0) {
    for (auto& o : outs) { o.hist.push_back(0.0); o.status = MSBEM_OK; }
    return cudaStreamSynchronize(s);
  }
  cudaError_t e;
  if (tensor && (e = ensure_w_slices(g, 0, s)) != cudaSuccess) return e;
  const unsigned gemv_blocks = matvec_blocks(N, 0);
  const size_t nvec = (size_t)N * kb;
  const size_t nparts = (size_t)kb * std::max<unsigned>(gemv_blocks, BRED);
  const int split = tensor ? 1 : matvec_split_of(g, 0);
  const size_t scr_bytes = tensor ? tc_work_bytes(g) : matvec_scratch_bytes(N, kb, split);
  const size_t bytes = sizeof(double) * (5 * nvec + nparts + 3 * kb + 4 * kb) + sizeof(float) * 2 * kb * g.ldw +
                       sizeof(int) * kb + sizeof(BatchState) + scr_bytes + 256;
  char* base = nullptr;
  if ((e = pool_alloc((void**)&base, bytes, g.pool, s)) != cudaSuccess) return e;
  Carver cv{base};
  double* L = cv.take<double>(nvec);
  double* X = cv.take<double>(nvec);
  double* R = cv.take<double>(nvec);
  double* D = cv.take<double>(nvec);
  double* Q = cv.take<double>(nvec);
  double* part = cv.take<double>(nparts);
  double* gv = cv.take<double>(3 * kb);
  double* nrm = cv.take<double>(4 * kb);     // ||L||^2, ||R||^2, ||D||^2, ||X||^2 per column
  float* Xf = cv.take<float>(2 * kb * g.ldw);
  int* skip = cv.take<int>(kb);
  BatchState* fl = cv.take<BatchState>(1);   // all_done = 0 throughout; err from the product
  char* scratch = cv.take<char>(scr_bytes);
  auto finish = [&](cudaError_t err) {
    cudaFreeAsync(base, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    return err != cudaSuccess ? err : e2;
  };
  CUtensorMap tmX;
  if ((e = encode_planes(&tmX, Xf, g.ldw, kb, kb * g.ldw, 2, matvec_pad(kb))) != cudaSuccess) return finish(e);
  BatchState h_fl{0, kb, 0, 0, 0.0, 0};
  cudaMemcpyAsync(fl, &h_fl, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(Xf, 0, sizeof(float) * 2 * kb * g.ldw, s);
  cudaMemsetAsync(X, 0, sizeof(double) * nvec, s);
  if ((e = batch_rhs(g, gvecs, kb, gv, L, s)) != cudaSuccess) return finish(e);
  cudaMemcpyAsync(R, L, sizeof(double) * nvec, cudaMemcpyDeviceToDevice, s);
  const dim3 rgrid(BRED, kb);
  bdot_kernel<<<rgrid, 256, 0, s>>>(L, L, N, kb, part, fl);
  bsum_kernel<<<kb, 256, 0, s>>>(part, BRED, nrm);
  g.launches += 2;
  std::vector<double> h_nrm(4 * kb, 0.0), dprev(kb, 0.0);
  std::vector<int> h_skip(kb, 0), inner_total(kb, 0), st(kb, MSBEM_OK);
  std::vector<char> conv(kb, 0);
  const int max_outer = 12;
  int outer = 0;
  for (;; ++outer) {
    bdot_kernel<<<rgrid, 256, 0, s>>>(R, R, N, kb, part, fl);
    bsum_kernel<<<kb, 256, 0, s>>>(part, BRED, nrm + kb);
    g.launches += 2;
    cudaMemcpyAsync(h_nrm.data(), nrm, sizeof(double) * 4 * kb, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return finish(e);
    bool all = true;
    for (int c = 0; c < kb; ++c) {
      const double nl = h_nrm[c];
      const double rel = nl > 0.0 ? std::sqrt(h_nrm[kb + c] / nl) : 0.0;
      if (!conv[c]) outs[c].hist.push_back(rel);
      // density test (density_tol > 0): the error of X_{k+1} = X_k + D_k is
      // estimated from the contraction eta of consecutive corrections,
      // eta = ||D_k|| / ||D_{k-1}||, as eta / (1 - eta) ||D_k|| (the error of
      // X_k is at most ||D_k|| / (1 - eta), and the next one eta times that)
      bool dens = density_tol <= 0.0;
      if (!conv[c] && !dens && outer >= 2) {
        const double dn = std::sqrt(h_nrm[2 * kb + c]), xn = std::sqrt(h_nrm[3 * kb + c]);
        const double eta = dprev[c] > 0.0 ? dn / dprev[c] : 1.0;
        const double est = eta < 1.0 ? eta / (1.0 - eta) * dn : INFINITY;
        outs[c].err_est = xn > 0.0 ? est / xn : 0.0;
        dens = est <= density_tol * xn;
      }
      if (!conv[c] && outer >= 1) dprev[c] = std::sqrt(h_nrm[2 * kb + c]);
      if (!conv[c] && (nl == 0.0 || (rel <= rtol && dens))) conv[c] = 1;
      if (!std::isfinite(rel)) { conv[c] = 1; st[c] = MSBEM_BREAKDOWN; }
      all = all && conv[c];
    }
    if (all) break;
    int budget = maxit;
    for (int c = 0; c < kb; ++c)
      if (!conv[c]) budget = std::min(budget, maxit - inner_total[c]);
    if (outer >= max_outer || budget < 1) {
      for (int c = 0; c < kb; ++c)
        if (!conv[c]) st[c] = MSBEM_NOT_CONVERGED;
      break;
    }
    for (int c = 0; c < kb; ++c) h_skip[c] = conv[c];
    cudaMemcpyAsync(skip, h_skip.data(), sizeof(int) * kb, cudaMemcpyHostToDevice, s);
    bmask_kernel<<<kStrideBlocks, 256, 0, s>>>(R, (int64_t)nvec, kb, skip, Q);
    ++g.launches;
    std::vector<PcgOut> in;
    if ((e = pcg_batch_core(g, kb, inner_rtol, budget, 0, precondition, inner_fp16 ? 4 : 1, Q, D, in, s)) !=
        cudaSuccess)
      return finish(e);
    for (int c = 0; c < kb; ++c) {
      if (conv[c]) continue;
      inner_total[c] += in[c].iters;
      if (outer == 0) {
        outs[c].alpha = in[c].alpha;
        outs[c].beta = in[c].beta;
      }
      if (in[c].status == MSBEM_DEVICE_TIMEOUT) st[c] = MSBEM_DEVICE_TIMEOUT;
    }
    baxpy_kernel<<<kStrideBlocks, 256, 0, s>>>(X, D, (int64_t)nvec);
    if (density_tol > 0.0) {
      bdot_kernel<<<rgrid, 256, 0, s>>>(D, D, N, kb, part, fl);
      bsum_kernel<<<kb, 256, 0, s>>>(part, BRED, nrm + 2 * kb);
      bdot_kernel<<<rgrid, 256, 0, s>>>(X, X, N, kb, part, fl);
      bsum_kernel<<<kb, 256, 0, s>>>(part, BRED, nrm + 3 * kb);
      g.launches += 4;
    }
    if (tensor) {
      launch_matvec_tc(g, 0, kb, X, Q, part, &fl->all_done, &fl->err, scratch, s);
    } else {
      bsplit_kernel<<<kStrideBlocks, 256, 0, s>>>(X, Xf, g.ldw, N, kb);
      launch_matvec(0, g.tm_W, tmX, N, kb, X, Q, part, &fl->all_done, &fl->err, s, split, scratch);
      g.launches += 2;
    }
    bresid_kernel<<<kStrideBlocks, 256, 0, s>>>(L, Q, (int64_t)nvec, R);
    g.launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return finish(e);
  }
  cudaMemcpyAsync(&h_fl, fl, sizeof(BatchState), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return finish(e);
  for (int c = 0; c < kb; ++c) {
    outs[c].iters = inner_total[c];
    outs[c].status = h_fl.err ? MSBEM_DEVICE_TIMEOUT : st[c];
    if (h_nrm[c] == 0.0) outs[c].hist.assign(1, 0.0);
  }
  if (refinements) *refinements = outer;
  e = copy_out(g, X, N, kb, X_out, out_on_device, s);
  return finish(e);
}

// X[i][c] = Xin[c][i]  (k x N  ->  N x k)
__global__ void btranspose_in_kernel(const double* __restrict__ Xin, int64_t N, int kb, double* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * kb) return;
  const int64_t i = e / kb;
  const int c = (int)(e % kb);
  X[e] = Xin[(int64_t)c * N + i];
}

// Y = W X for kb <= 16 vectors (rows of X_in, k x N, host or device); mode 0
// double-float products, 1 FP32 products with the hi plane, 2 the plain FP64
// copy (one vector at a time), 3 double-float from integer slices on the
// tensor cores, 4 scaled FP16 on the tensor cores.  *kernel_ms receives the device time of the
// product kernel(s) alone.
cudaError_t apply_w(DevGeom& g, const double* X_in, bool in_dev, int kb, int mode, double* Y_out, bool out_dev,
                    float* kernel_ms, cudaStream_t s) {
  const int64_t N = g.ndof;
  if (kb < 1 || kb > BK) return cudaErrorInvalidValue;
  if (N == 0) return cudaSuccess;
  cudaError_t e;
  if (mode == 2 && (e = ensure_w64(g, s)) != cudaSuccess) return e;
  if (mode >= 3 && (e = ensure_w_slices(g, mode - 3, s)) != cudaSuccess) return e;
  const unsigned gemv_blocks = matvec_blocks(N, 0);
  const size_t nvec = (size_t)N * kb;
  const size_t nparts = (size_t)kb * std::max<unsigned>(gemv_blocks, (unsigned)((N + 15) / 16));
  const int split = mode >= 2 ? 1 : matvec_split_of(g, mode);
  const size_t scr_bytes = mode >= 3 ? tc_work_bytes(g) : matvec_scratch_bytes(N, kb, split);
  const size_t bytes = sizeof(double) * (3 * nvec + nparts) + sizeof(float) * 2 * kb * g.ldw +
                       sizeof(BatchState) + scr_bytes + 256;
  char* base = nullptr;
  if ((e = pool_alloc((void**)&base, bytes, g.pool, s)) != cudaSuccess) return e;
  Carver cv{base};
  double* Xin = cv.take<double>(nvec);
  double* X = cv.take<double>(nvec);
  double* Q = cv.take<double>(nvec);
  double* part = cv.take<double>(nparts);
  float* Xf = cv.take<float>(2 * kb * g.ldw);
  BatchState* fl = cv.take<BatchState>(1);
  char* scratch = cv.take<char>(scr_bytes);
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  BatchState h_fl{0, kb, 0, 0, 0.0, 0};
  cudaMemcpyAsync(fl, &h_fl, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(Xin, X_in, sizeof(double) * nvec, in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  btranspose_in_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(Xin, N, kb, X);
  ++g.launches;
  if (mode == 2) {
    // plain FP64: column by column with the comparator's kernel (its layout is a
    // contiguous vector), so the input stays k x N
    cudaEventRecord(ev[0], s);
    for (int c = 0; c < kb; ++c)
      launch_gemv64(g, Xin + (size_t)c * N, Q + (size_t)c * N, part, &fl->all_done, s);
    cudaEventRecord(ev[1], s);
    g.launches += kb;
    e = cudaMemcpyAsync(Y_out, Q, sizeof(double) * nvec, out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        s);
  } else if (mode >= 3) {
    cudaEventRecord(ev[0], s);
    e = launch_matvec_tc(g, mode - 3, kb, X, Q, part, &fl->all_done, &fl->err, scratch, s);
    cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = copy_out(g, Q, N, kb, Y_out, out_dev, s);
  } else {
    CUtensorMap tmX;
    const int planes = mode == 0 ? 2 : 1;
    e = encode_planes(&tmX, Xf, g.ldw, kb, kb * g.ldw, planes, matvec_pad(kb));
    if (e == cudaSuccess) {
      cudaMemsetAsync(Xf, 0, sizeof(float) * 2 * kb * g.ldw, s);
      bsplit_kernel<<<kStrideBlocks, 256, 0, s>>>(X, Xf, g.ldw, N, kb);
      cudaEventRecord(ev[0], s);
      e = launch_matvec(mode, mode == 0 ? g.tm_W : g.tm_Whi, tmX, N, kb, X, Q, part, &fl->all_done, &fl->err, s,
                        split, scratch);
      cudaEventRecord(ev[1], s);
      g.launches += 2;
    }
    if (e == cudaSuccess) e = copy_out(g, Q, N, kb, Y_out, out_dev, s);
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && kernel_ms) cudaEventElapsedTime(kernel_ms, ev[0], ev[1]);
  if (e == cudaSuccess) {
    cudaMemcpy(&h_fl, fl, sizeof(BatchState), cudaMemcpyDeviceToHost);
    if (h_fl.err) e = cudaErrorTimeout;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaFreeAsync(base, s);
  e2 = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace msbem
