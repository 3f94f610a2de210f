// Preconditioned conjugate gradients for W Phi = L (Sec. 2.1, Remark "Bound on
// the number of PCG iterations"), entirely on the device:
//
//   q = W p; alpha = (r.z)/(p.q); x += alpha p; r -= alpha q;
//   stop if ||r|| <= rtol ||L||;  z = M r; beta = (r.z)_new/(r.z); p = z + beta p
//
// with M the two-level additive Schwarz operator (face blocks, wire basket,
// coarse space) applied through the explicit block inverses.  Reductions are
// two-pass (fixed order), so results are bitwise reproducible run to run.
// The host reads back three scalars per iteration for the stopping test and the
// residual history.
#include <cmath>
#include <vector>

#include "msbem_internal.h"

namespace msbem {

#define RED_BLOCKS 256

// q = W p, partial sums of p.q per block
__global__ void __launch_bounds__(256) gemv_kernel(const double* __restrict__ W, int64_t N,
                                                   const double* __restrict__ p,
                                                   double* __restrict__ q,
                                                   double* __restrict__ part) {
  __shared__ double s_part[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * 8 + wid;
  double pq = 0.0;
  if (row < N) {
    const double* w = W + row * N;
    double acc = 0.0;
    for (int64_t j = lane; j < N; j += 32) acc = fma(w[j], p[j], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) q[row] = acc;
    pq = acc * p[row];
  }
  if (lane == 0) s_part[wid] = pq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += s_part[k];
    part[blockIdx.x] = s;
  }
}

// fixed-order final reduction of n partial sums into *out
__global__ void reduce_kernel(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) acc += part[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// partial sums of a.b (grid of RED_BLOCKS blocks)
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t N,
                           double* __restrict__ part) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
    acc = fma(a[i], b[i], acc);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// scal layout: 0 rz, 1 pq, 2 alpha, 3 rr, 4 rz_new, 5 beta, 6 nL2
__global__ void alpha_kernel(double* scal) {
  scal[2] = scal[0] / scal[1];
}

// x += alpha p; r -= alpha q; partial r.r
__global__ void update_xr_kernel(double* __restrict__ x, double* __restrict__ r,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ scal, int64_t N,
                                 double* __restrict__ part) {
  __shared__ double s[256];
  const double alpha = scal[2];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// z[D_b[i]] = sum_j Ainv_b[i][j] r[D_b[j]]  (warp per row, rows of all blocks)
__global__ void __launch_bounds__(256) block_apply_kernel(const double* __restrict__ Ainv,
                                                          const int64_t* __restrict__ boff,
                                                          const int64_t* __restrict__ bptr,
                                                          const int32_t* __restrict__ bdofs,
                                                          int nblk, int64_t N,
                                                          const double* __restrict__ r,
                                                          double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t rho = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (rho >= N) return;
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {  // last block with bptr[b] <= rho
    int mid = (lo + hi + 1) >> 1;
    if (bptr[mid] <= rho) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int64_t n = bptr[b + 1] - bptr[b];
  const int64_t i = rho - bptr[b];
  const double* a = Ainv + boff[b] + i * n;
  const int32_t* d = bdofs + bptr[b];
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(a[j], r[d[j]], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) z[d[i]] = acc;
}

// t = P^T r (CSC of P), warp per coarse dof
__global__ void restrict_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                const double* __restrict__ cval, int64_t NH,
                                const double* __restrict__ r, double* __restrict__ t) {
  const int lane = threadIdx.x & 31;
  const int64_t mu = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (mu >= NH) return;
  double acc = 0.0;
  for (int64_t k = cptr[mu] + lane; k < cptr[mu + 1]; k += 32) acc = fma(cval[k], r[crow[k]], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) t[mu] = acc;
}

// u = AHinv t (warp per row)
__global__ void coarse_solve_kernel(const double* __restrict__ AHinv, int64_t NH,
                                    const double* __restrict__ t, double* __restrict__ u) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= NH) return;
  double acc = 0.0;
  for (int64_t j = lane; j < NH; j += 32) acc = fma(AHinv[i * NH + j], t[j], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) u[i] = acc;
}

// z += P u (CSR of P by fine row)
__global__ void prolong_kernel(const int64_t* __restrict__ pptr, const int32_t* __restrict__ pcol,
                               const double* __restrict__ pval, int64_t N,
                               const double* __restrict__ u, double* __restrict__ z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int64_t k = pptr[i]; k < pptr[i + 1]; ++k) acc = fma(pval[k], u[pcol[k]], acc);
  z[i] += acc;
}

// beta = rz_new / rz; rz = rz_new
__global__ void beta_kernel(double* scal) {
  scal[5] = scal[4] / scal[0];
  scal[0] = scal[4];
}

// p = z + beta p
__global__ void update_p_kernel(double* __restrict__ p, const double* __restrict__ z,
                                const double* __restrict__ scal, int64_t N) {
  const double beta = scal[5];
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void copy_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
    dst[i] = src[i];
}

static void apply_M(DevGeom& g, const double* r, double* z, double* t, double* u, int precondition,
                    cudaStream_t s) {
  const int64_t N = g.ndof;
  if (!precondition) {
    copy_kernel<<<RED_BLOCKS, 256, 0, s>>>(z, r, N);
    ++g.launches;
    return;
  }
  ++g.launches;
  block_apply_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(g.d_binv, g.d_boff, g.d_bptr, g.d_bdofs,
                                                              (int)g.n_blocks, N, r, z);
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  if (NH > 0) {
    restrict_kernel<<<(unsigned)((NH + 7) / 8), 256, 0, s>>>(g.d_cptr, g.d_crow, g.d_cval, NH, r, t);
    coarse_solve_kernel<<<(unsigned)((NH + 7) / 8), 256, 0, s>>>(g.d_AHinv, NH, t, u);
    prolong_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, u, z);
    g.launches += 3;
  }
}

cudaError_t run_pcg(DevGeom& g, const double gvec[3], double rtol, int maxit, int fixed,
                    int precondition, double* x_out, PcgOut& out, cudaStream_t s) {
  const int64_t N = g.ndof;
  out = PcgOut();
  double* x = g.d_vec;
  double* r = x + N;
  double* z = r + N;
  double* p = z + N;
  double* q = p + N;
  double* t = q + N;          // coarse scratch (NH)
  double* u = t + std::max<int64_t>(g.n_coarse, 1);
  double* scal = g.d_scal;    // 8 scalars
  double* part = scal + 8;    // partial sums (>= max(RED_BLOCKS, N/8+1))
  const unsigned gemv_blocks = (unsigned)((N + 7) / 8);
  cudaError_t e;
  if (N == 0) {  // nothing to solve (no launch may have an empty grid)
    out.hist.push_back(0.0);
    out.status = MSBEM_OK;
    return cudaStreamSynchronize(s);
  }
  cudaMemsetAsync(x, 0, sizeof(double) * N, s);
  if ((e = launch_rhs(g, gvec, r, s)) != cudaSuccess) return e;
  dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, r, N, part);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 6);
  apply_M(g, r, z, t, u, precondition, s);
  copy_kernel<<<RED_BLOCKS, 256, 0, s>>>(p, z, N);
  dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, z, N, part);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 0);
  g.launches += 5 + (N > 0);
  double h[8];
  if ((e = cudaMemcpyAsync(h, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  const double nL = std::sqrt(h[6]);
  out.hist.push_back(nL > 0 ? 1.0 : 0.0);
  if (nL == 0.0) {
    if (x_out != x) cudaMemcpyAsync(x_out, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    out.status = MSBEM_OK;
    return cudaStreamSynchronize(s);
  }
  out.status = MSBEM_NOT_CONVERGED;
  for (int it = 0; it < maxit; ++it) {
    gemv_kernel<<<gemv_blocks, 256, 0, s>>>(g.d_W, N, p, q, part);
    reduce_kernel<<<1, 256, 0, s>>>(part, gemv_blocks, scal + 1);
    alpha_kernel<<<1, 1, 0, s>>>(scal);
    update_xr_kernel<<<RED_BLOCKS, 256, 0, s>>>(x, r, p, q, scal, N, part);
    reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 3);
    apply_M(g, r, z, t, u, precondition, s);
    dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, z, N, part);
    reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 4);
    beta_kernel<<<1, 1, 0, s>>>(scal);
    update_p_kernel<<<RED_BLOCKS, 256, 0, s>>>(p, z, scal, N);
    g.launches += 9;
    if ((e = cudaMemcpyAsync(h, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const double pq = h[1], alpha = h[2], rel = std::sqrt(h[3]) / nL, beta = h[5];
    out.iters = it + 1;
    if (!(pq > 0.0) || !std::isfinite(alpha) || !std::isfinite(rel)) {
      out.status = MSBEM_BREAKDOWN;
      break;
    }
    out.alpha.push_back(alpha);
    out.hist.push_back(rel);
    if (rel <= rtol) {
      out.status = MSBEM_OK;
      if (!fixed) break;
    }
    if (it + 1 == maxit) break;
    out.beta.push_back(beta);
  }
  if (x_out != x) cudaMemcpyAsync(x_out, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  if (fixed && out.iters == maxit && out.status != MSBEM_BREAKDOWN) out.status = MSBEM_OK;
  return cudaStreamSynchronize(s);
}

}  // namespace msbem
