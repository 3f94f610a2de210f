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

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define BK 16                 // columns per pass
#define BRED 128              // blocks of the column reductions
static constexpr unsigned kStrideBlocks = 512;

struct ColState {
  double rz, pq, alpha, rr, rz_new, beta, nL2;
  int done, iter, pad0, pad1;
};
struct BatchState {
  int all_done;
  int kb;
  int maxit;
  int fixed;
  double rtol;
  int err;      // set by the matrix-vector product when a copy never completed
};

__device__ __forceinline__ bool col_active(const ColState* cs, int c) { return cs[c].done == 0; }

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
__global__ void bupdate_xr_kernel(double* __restrict__ X, double* __restrict__ R,
                                  const double* __restrict__ P, const double* __restrict__ Q, int64_t N,
                                  int kb, const ColState* __restrict__ cs, double* __restrict__ part,
                                  const BatchState* __restrict__ bs) {
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

// Z[D_b[i]][c] = sum_j Ainv_b[i][j] R[D_b[j]][c] for all columns (warp per row)
__global__ void __launch_bounds__(256) bblock_apply_kernel(const float2* __restrict__ Ainv,
                                                           const int64_t* __restrict__ boff,
                                                           const int64_t* __restrict__ bptr,
                                                           const int32_t* __restrict__ bdofs, int nblk,
                                                           int64_t N, const float2* __restrict__ Rf,
                                                           double* __restrict__ Z, int kb,
                                                           const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  const int lane = threadIdx.x & 31;
  const int64_t rho = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (rho >= N) return;
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (bptr[mid] <= rho) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int64_t n = bptr[b + 1] - bptr[b];
  const int64_t i = rho - bptr[b];
  const float2* a = Ainv + boff[b] + i * n;
  const int32_t* d = bdofs + bptr[b];
  float h[BK], l[BK];
#pragma unroll
  for (int c = 0; c < BK; ++c) { h[c] = 0.f; l[c] = 0.f; }
  for (int64_t j = lane; j < n; j += 32) {
    const float2 x = a[j];
    const float2* rr = Rf + (int64_t)d[j] * kb;
#pragma unroll
    for (int c = 0; c < BK; ++c)
      if (c < kb) df_fma_acc(x.x, x.y, rr[c].x, rr[c].y, h[c], l[c]);
  }
#pragma unroll
  for (int c = 0; c < BK; ++c) {
    if (c >= kb) break;
    float acch = h[c], accl = l[c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      float oh = __shfl_xor_sync(0xffffffffu, acch, off);
      float ol = __shfl_xor_sync(0xffffffffu, accl, off);
      float sh, se;
      two_sum(acch, oh, sh, se);
      acch = sh;
      accl = accl + ol + se;
    }
    if (lane == 0) Z[(int64_t)d[i] * kb + c] = df_to_double(acch, accl);
  }
}

// T[mu][c] = sum_k P[row_k, mu] R[row_k][c]  (block per coarse dof)
__global__ void brestrict_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                 const double* __restrict__ cval, const double* __restrict__ R, int kb,
                                 double* __restrict__ T, const BatchState* __restrict__ bs) {
  if (bs->all_done) return;
  __shared__ double s[8][BK];
  const int64_t mu = blockIdx.x;
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

namespace {
struct BatchBuffers {
  double *X, *R, *Z, *P, *Q, *T, *U, *part, *gv, *hist;
  float* Pf;     // [2][kb][ldw]
  float2* Rf;
  ColState* cs;
  BatchState* bs;
};
}  // namespace

static void apply_M_batch(DevGeom& g, const BatchBuffers& b, int kb, int precondition, cudaStream_t s) {
  const int64_t N = g.ndof;
  if (!precondition) {
    bcopy_kernel<<<kStrideBlocks, 256, 0, s>>>(b.Z, b.R, N * kb, b.bs);
    ++g.launches;
    return;
  }
  bto_df_kernel<<<kStrideBlocks, 256, 0, s>>>(b.R, b.Rf, N * kb, b.bs);
  bblock_apply_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(g.d_binvf, g.d_boff, g.d_bptr, g.d_bdofs,
                                                               (int)g.n_blocks, N, b.Rf, b.Z, kb, b.bs);
  g.launches += 2;
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  if (NH > 0) {
    brestrict_kernel<<<(unsigned)NH, 256, 0, s>>>(g.d_cptr, g.d_crow, g.d_cval, b.R, kb, b.T, b.bs);
    bcoarse_kernel<<<(unsigned)((NH * kb + 127) / 128), 128, 0, s>>>(g.d_AHinv, NH, b.T, kb, b.U, b.bs);
    bprolong_kernel<<<(unsigned)((N * kb + 255) / 256), 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, b.U,
                                                                      kb, b.Z, b.bs);
    g.launches += 3;
  }
}

cudaError_t run_pcg_batch(DevGeom& g, const double* gvecs, int kb, double rtol, int maxit, int fixed,
                          int precondition, double* X_out, bool out_on_device, std::vector<PcgOut>& outs,
                          cudaStream_t s) {
  const int64_t N = g.ndof;
  outs.assign(kb, PcgOut());
  if (kb < 1 || kb > BK) return cudaErrorInvalidValue;
  if (N == 0) {
    for (auto& o : outs) { o.hist.push_back(0.0); o.status = MSBEM_OK; }
    return cudaStreamSynchronize(s);
  }
  const int64_t NH = std::max<int64_t>(g.n_coarse, 1);
  const unsigned gemv_blocks = matvec_blocks(N);
  const size_t nvec = (size_t)N * kb;
  const size_t nparts = (size_t)kb * std::max<unsigned>(gemv_blocks, BRED);
  const size_t hsz = (size_t)kb * (maxit + 1) + 2 * (size_t)kb * maxit;
  const size_t bytes = sizeof(double) * (5 * nvec + 2 * NH * kb + nparts + 3 * kb + hsz) +
                       sizeof(float) * 2 * kb * g.ldw + sizeof(float2) * nvec + sizeof(ColState) * kb +
                       sizeof(BatchState) + 512;
  char* base = nullptr;
  cudaError_t e = pool_alloc((void**)&base, bytes, g.pool, s);
  if (e != cudaSuccess) return e;
  BatchBuffers b;
  char* cur = base;
  auto take = [&](size_t n) { char* p = cur; cur += (n + 15) / 16 * 16; return p; };
  b.X = (double*)take(sizeof(double) * nvec);
  b.R = (double*)take(sizeof(double) * nvec);
  b.Z = (double*)take(sizeof(double) * nvec);
  b.P = (double*)take(sizeof(double) * nvec);
  b.Q = (double*)take(sizeof(double) * nvec);
  b.T = (double*)take(sizeof(double) * NH * kb);
  b.U = (double*)take(sizeof(double) * NH * kb);
  b.part = (double*)take(sizeof(double) * nparts);
  b.gv = (double*)take(sizeof(double) * 3 * kb);
  b.hist = (double*)take(sizeof(double) * hsz);
  b.Pf = (float*)take(sizeof(float) * 2 * kb * g.ldw);
  b.Rf = (float2*)take(sizeof(float2) * nvec);
  b.cs = (ColState*)take(sizeof(ColState) * kb);
  b.bs = (BatchState*)take(sizeof(BatchState));
  double* rel_h = b.hist;                                   // kb x (maxit+1)
  double* alpha_h = rel_h + (size_t)kb * (maxit + 1);       // kb x maxit
  double* beta_h = alpha_h + (size_t)kb * maxit;            // kb x maxit
  std::vector<ColState> h_cs(kb);
  for (auto& c : h_cs) c = ColState{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  BatchState h_bs{0, kb, maxit, fixed, rtol, 0};
  CUtensorMap tmP;
  if ((e = encode_planes(&tmP, b.Pf, g.ldw, kb, kb * g.ldw, 2, kb)) != cudaSuccess) {
    cudaFreeAsync(base, s);
    return e;
  }
  cudaMemsetAsync(b.Pf, 0, sizeof(float) * 2 * kb * g.ldw, s);
  cudaMemcpyAsync(b.gv, gvecs, sizeof(double) * 3 * kb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b.cs, h_cs.data(), sizeof(ColState) * kb, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(b.bs, &h_bs, sizeof(BatchState), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(b.X, 0, sizeof(double) * nvec, s);
  brhs_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(g.d_jptr, g.d_jrhs, N, b.gv, kb, b.R);
  const dim3 rgrid(BRED, kb);
  bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.R, N, kb, b.part, b.bs);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, nL2), b.bs);
  apply_M_batch(g, b, kb, precondition, s);
  bupdate_p_kernel<<<kStrideBlocks, 256, 0, s>>>(b.P, b.Pf, g.ldw, b.Z, N, kb, b.cs, 1, b.bs);
  bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.Z, N, kb, b.part, b.bs);
  breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rz), b.bs);
  g.launches += 7;
  // columns with zero data are finished before the first iteration
  if ((e = cudaMemcpyAsync(h_cs.data(), b.cs, sizeof(ColState) * kb, cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
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
    for (int it = 0; it < chunk; ++it) {
      launch_matvec(0, g.tm_W, tmP, N, kb, b.P, b.Q, b.part, &b.bs->all_done, &b.bs->err, s);
      breduce_kernel<<<kb, 256, 0, s>>>(b.part, (int)gemv_blocks, b.cs, offsetof(ColState, pq), b.bs);
      balpha_kernel<<<1, BK, 0, s>>>(b.cs, alpha_h, maxit, b.bs);
      bupdate_xr_kernel<<<rgrid, 256, 0, s>>>(b.X, b.R, b.P, b.Q, N, kb, b.cs, b.part, b.bs);
      breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rr), b.bs);
      bcheck_kernel<<<1, 32, 0, s>>>(b.cs, rel_h, maxit, b.bs);
      apply_M_batch(g, b, kb, precondition, s);
      bdot_kernel<<<rgrid, 256, 0, s>>>(b.R, b.Z, N, kb, b.part, b.bs);
      breduce_kernel<<<kb, 256, 0, s>>>(b.part, BRED, b.cs, offsetof(ColState, rz_new), b.bs);
      bbeta_kernel<<<1, BK, 0, s>>>(b.cs, beta_h, maxit, b.bs);
      bupdate_p_kernel<<<kStrideBlocks, 256, 0, s>>>(b.P, b.Pf, g.ldw, b.Z, N, kb, b.cs, 0, b.bs);
      g.launches += 10;
    }
    enq += chunk;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&h_bs, b.bs, sizeof(BatchState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  }
  std::vector<double> h(hsz);
  cudaMemcpyAsync(h.data(), b.hist, sizeof(double) * hsz, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h_cs.data(), b.cs, sizeof(ColState) * kb, cudaMemcpyDeviceToHost, s);
  // densities, column c of X (row-major N x kb) -> X_out[c][i]
  std::vector<double> xh;
  if (X_out && out_on_device) {
    btranspose_kernel<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(b.X, N, kb, X_out);
    ++g.launches;
  } else if (X_out) {
    xh.resize(nvec);
    cudaMemcpyAsync(xh.data(), b.X, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s);
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  cudaFreeAsync(base, s);
  if (X_out && !out_on_device)
    for (int c = 0; c < kb; ++c)
      for (int64_t i = 0; i < N; ++i) X_out[(size_t)c * N + i] = xh[(size_t)i * kb + c];
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

}  // namespace msbem
