// Preconditioned conjugate gradients for W Phi = L (Sec. 2.1, Remark "Bound on
// the number of PCG iterations"), entirely on the device:
//
//   q = W p; alpha = (r.z)/(p.q); x += alpha p; r -= alpha q;
//   stop if ||r|| <= rtol ||L||;  z = M r; beta = (r.z)_new/(r.z); p = z + beta p
//
// with M the two-level additive Schwarz operator (face blocks, wire basket,
// coarse space) applied through the explicit block inverses.  Reductions are
// two-pass (fixed order), so results are bitwise reproducible run to run.
// The stopping test runs on the device: it records the residual history and
// the PCG coefficients and raises a `done` flag that turns every later kernel
// into a no-op, so the host enqueues iterations in chunks and synchronises once
// per chunk instead of once per iteration.
#include <cmath>
#include <vector>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define RED_BLOCKS 256
#define PCG_CHUNK 4

// device-side solver state (ints), next to the FP64 scalars
struct PcgState {
  int done;    // 0 running, 1 converged / fixed count reached, 2 breakdown, 3 maxit,
               // 5 device timeout (a matrix copy never completed)
  int iter;    // completed iterations
  int maxit;
  int fixed;
  int err;     // set by the matrix-vector product when a copy never completed
};

// scal layout: 0 rz, 1 pq, 2 alpha, 3 rr, 4 rz_new, 5 beta, 6 |L|^2, 7 rtol

// q = W p: matvec.cu (TMA-fed, double-float on the FP32 pipe, 8 bytes of W
// per entry from HBM), with per-block partial sums of p.q.

// fixed-order final reduction of n partial sums into *out
__global__ void reduce_kernel(const double* __restrict__ part, int64_t n, double* __restrict__ out,
                              const PcgState* __restrict__ st) {
  if (st->done) return;
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
                           double* __restrict__ part, const PcgState* __restrict__ st) {
  if (st->done) return;
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

// alpha = (r.z)/(p.q); breakdown if p.q <= 0 or not finite
__global__ void alpha_kernel(double* scal, PcgState* st, double* alpha_hist) {
  if (st->done) return;
  const double pq = scal[1];
  const double a = scal[0] / pq;
  if (!(pq > 0.0) || !isfinite(a)) {
    st->done = 2;
    return;
  }
  scal[2] = a;
  alpha_hist[st->iter] = a;
}

// x += alpha p; r -= alpha q; partial r.r
// rf (may be null): r's float-pair split, written beside it for the block
// solves of the preconditioner that follow
__global__ void update_xr_kernel(double* __restrict__ x, double* __restrict__ r,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ scal, int64_t N,
                                 double* __restrict__ part, float2* __restrict__ rf,
                                 const PcgState* __restrict__ st) {
  if (st->done) return;
  __shared__ double s[256];
  const double alpha = scal[2];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    x[i] = fma(alpha, p[i], x[i]);
    double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    if (rf) {
      float h, l;
      split_df(ri, h, l);
      rf[i] = make_float2(h, l);
    }
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

// stopping test: relres = ||r|| / ||L||, history, iteration count, done flag
__global__ void check_kernel(const double* scal, PcgState* st, double* hist) {
  if (st->done) return;
  const double rel = sqrt(scal[3] / scal[6]);
  const int it = st->iter + 1;
  st->iter = it;
  hist[it] = rel;
  if (st->err) st->done = 5;
  else if (!isfinite(rel)) st->done = 2;
  else if (!st->fixed && rel <= scal[7]) st->done = 1;
  else if (it >= st->maxit) st->done = (st->fixed || rel <= scal[7]) ? 1 : 3;
}

// z[D_b[i]] = sum_j Ainv_b[i][j] r[D_b[j]]  (warp per row, rows of all blocks),
// in double-float from float-pair copies of the block inverses and of r
__device__ __forceinline__ void block_apply_body(int64_t cta, const float2* __restrict__ Ainv,
                                                 const int64_t* __restrict__ boff, const int64_t* __restrict__ bptr,
                                                 const int32_t* __restrict__ bdofs, int nblk, int64_t N,
                                                 const float2* __restrict__ rf, double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t rho = cta * 8 + (threadIdx.x >> 5);
  if (rho >= N) return;
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {  // last block with bptr[b] <= rho
    int mid = (lo + hi + 1) >> 1;
    if (bptr[mid] <= rho) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int64_t n = bptr[b + 1] - bptr[b];
  const int64_t i = rho - bptr[b];
  const float2* a = Ainv + boff[b] + i * n;
  const int32_t* d = bdofs + bptr[b];
  float acch = 0.f, accl = 0.f;
  for (int64_t j = lane; j < n; j += 32) {
    const float2 x = a[j], y = rf[d[j]];
    df_fma_acc(x.x, x.y, y.x, y.y, acch, accl);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, acch, off);
    float ol = __shfl_xor_sync(0xffffffffu, accl, off);
    float sh, se;
    two_sum(acch, oh, sh, se);
    acch = sh;
    accl = accl + ol + se;
  }
  if (lane == 0) z[d[i]] = df_to_double(acch, accl);
}

__global__ void __launch_bounds__(256) block_apply_kernel(const float2* __restrict__ Ainv,
                                                          const int64_t* __restrict__ boff,
                                                          const int64_t* __restrict__ bptr,
                                                          const int32_t* __restrict__ bdofs,
                                                          int nblk, int64_t N,
                                                          const float2* __restrict__ rf,
                                                          double* __restrict__ z,
                                                          const PcgState* __restrict__ st) {
  if (st->done) return;
  block_apply_body(blockIdx.x, Ainv, boff, bptr, bdofs, nblk, N, rf, z);
}

// ---- plain FP64 comparator: W and the block inverses read as FP64 -----------
// q = W p with an FP64 copy of W (N x N), warp per row pair, FP64 FMAs
__global__ void __launch_bounds__(256) gemv64_kernel(const double* __restrict__ W, int64_t N,
                                                     const double* __restrict__ p,
                                                     double* __restrict__ q,
                                                     double* __restrict__ part,
                                                     const PcgState* __restrict__ st) {
  if (st->done) return;
  __shared__ double s_part[16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * 16 + 2 * wid;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int64_t row = row0 + rr;
    double acc = 0.0;
    if (row < N) {
      const double* w = W + row * N;
      int64_t j = lane;
      for (; j + 96 < N; j += 128) {
        const double a0 = w[j], a1 = w[j + 32], a2 = w[j + 64], a3 = w[j + 96];
        acc = fma(a0, p[j], acc);
        acc = fma(a1, p[j + 32], acc);
        acc = fma(a2, p[j + 64], acc);
        acc = fma(a3, p[j + 96], acc);
      }
      for (; j < N; j += 32) acc = fma(w[j], p[j], acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    double pq = 0.0;
    if (row < N) {
      if (lane == 0) q[row] = acc;
      pq = acc * p[row];
    }
    if (lane == 0) s_part[2 * wid + rr] = pq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 16; ++k) t += s_part[k];
    part[blockIdx.x] = t;
  }
}

// z[D_b[i]] = sum_j Ainv_b[i][j] r[D_b[j]] with the FP64 inverses
__global__ void __launch_bounds__(256) block_apply64_kernel(const double* __restrict__ Ainv,
                                                            const int64_t* __restrict__ boff,
                                                            const int64_t* __restrict__ bptr,
                                                            const int32_t* __restrict__ bdofs,
                                                            int nblk, int64_t N,
                                                            const double* __restrict__ r,
                                                            double* __restrict__ z,
                                                            const PcgState* __restrict__ st) {
  if (st->done) return;
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
  const double* a = Ainv + boff[b] + i * n;
  const int32_t* d = bdofs + bptr[b];
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(a[j], r[d[j]], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) z[d[i]] = acc;
}

// float-pair copy of a vector
__global__ void to_df_kernel(const double* __restrict__ x, float2* __restrict__ xf, int64_t N,
                             const PcgState* __restrict__ st) {
  if (st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    float h, l;
    split_df(x[i], h, l);
    xf[i] = make_float2(h, l);
  }
}

// t = P^T r (CSC of P), one block per coarse dof (columns of P hold
// thousands of fine entries)
__device__ __forceinline__ void restrict_body1(int64_t mu, const int64_t* __restrict__ cptr,
                                               const int32_t* __restrict__ crow, const double* __restrict__ cval,
                                               const double* __restrict__ r, double* __restrict__ t, double* s) {
  double acc = 0.0;
  for (int64_t k = cptr[mu] + threadIdx.x; k < cptr[mu + 1]; k += blockDim.x)
    acc = fma(cval[k], r[crow[k]], acc);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s[w];
    t[mu] = v;
  }
}

__global__ void restrict_kernel(const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                                const double* __restrict__ cval, int64_t NH,
                                const double* __restrict__ r, double* __restrict__ t,
                                const PcgState* __restrict__ st) {
  if (st->done) return;
  __shared__ double s[8];
  restrict_body1(blockIdx.x, cptr, crow, cval, r, t, s);
}

// The block solves (CTAs below nba, 8 rows each) and the coarse restriction
// (one CTA per coarse dof after them) in one launch: both read r, their
// outputs are disjoint.
__global__ void __launch_bounds__(256) block_restrict_kernel(
    const float2* __restrict__ Ainv, const int64_t* __restrict__ boff, const int64_t* __restrict__ bptr,
    const int32_t* __restrict__ bdofs, int nblk, int64_t N, const float2* __restrict__ rf, double* __restrict__ z,
    int64_t nba, const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
    const double* __restrict__ cval, const double* __restrict__ r, double* __restrict__ t,
    const PcgState* __restrict__ st) {
  if (st->done) return;
  __shared__ double s[8];
  if ((int64_t)blockIdx.x < nba)
    block_apply_body(blockIdx.x, Ainv, boff, bptr, bdofs, nblk, N, rf, z);
  else
    restrict_body1((int64_t)blockIdx.x - nba, cptr, crow, cval, r, t, s);
}

// u = AHinv t (warp per row)
__global__ void coarse_solve_kernel(const double* __restrict__ AHinv, int64_t NH,
                                    const double* __restrict__ t, double* __restrict__ u,
                                    const PcgState* __restrict__ st) {
  if (st->done) return;
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
                               const double* __restrict__ u, double* __restrict__ z,
                               const PcgState* __restrict__ st) {
  if (st->done) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int64_t k = pptr[i]; k < pptr[i + 1]; ++k) acc = fma(pval[k], u[pcol[k]], acc);
  z[i] += acc;
}

// z += P u, and the per-block partial sums of r . z over dot_kernel's row
// partition (the prolongation fused with the reduction that follows it; the
// same arithmetic in the same order as the two kernels)
__global__ void prolong_dot_kernel(const int64_t* __restrict__ pptr, const int32_t* __restrict__ pcol,
                                   const double* __restrict__ pval, int64_t N, const double* __restrict__ u,
                                   double* __restrict__ z, const double* __restrict__ r,
                                   double* __restrict__ part, const PcgState* __restrict__ st) {
  if (st->done) return;
  __shared__ double s[256];
  double dot = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    double acc = 0.0;
    for (int64_t k = pptr[i]; k < pptr[i + 1]; ++k) acc = fma(pval[k], u[pcol[k]], acc);
    const double zi = z[i] + acc;
    z[i] = zi;
    dot = fma(r[i], zi, dot);
  }
  s[threadIdx.x] = dot;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// beta = rz_new / rz; rz = rz_new
__global__ void beta_kernel(double* scal, const PcgState* st, double* beta_hist) {
  if (st->done) return;
  const double b = scal[4] / scal[0];
  scal[5] = b;
  scal[0] = scal[4];
  beta_hist[st->iter - 1] = b;
}

// p = z + beta p (and its float-pair copy for the matrix-vector product)
__global__ void update_p_kernel(double* __restrict__ p, float* __restrict__ pf, int64_t ldp,
                                const double* __restrict__ z, const double* __restrict__ scal,
                                int64_t N, int first, const PcgState* __restrict__ st) {
  if (st->done) return;
  const double beta = first ? 0.0 : scal[5];
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256) {
    const double v = first ? z[i] : fma(beta, p[i], z[i]);
    p[i] = v;
    float h, l;
    split_df(v, h, l);
    pf[i] = h;
    pf[ldp + i] = l;
  }
}

__global__ void copy_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t N,
                            const PcgState* __restrict__ st) {
  if (st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
    dst[i] = src[i];
}

// z = M r.  in_iteration: inside a PCG iteration -- r's float-pair split is
// already in g.d_rf (written by the residual update), and the last launch
// also leaves the partial sums of r . z in part (dot_kernel's layout).
static void apply_M(DevGeom& g, const double* r, double* z, double* t, double* u, int precondition,
                    bool plain, const PcgState* st, cudaStream_t s, bool in_iteration = false,
                    double* part = nullptr) {
  const int64_t N = g.ndof;
  if (!precondition) {
    copy_kernel<<<RED_BLOCKS, 256, 0, s>>>(z, r, N, st);
    ++g.launches;
    if (in_iteration) {
      dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, z, N, part, st);
      ++g.launches;
    }
    return;
  }
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  const int64_t nba = (N + 7) / 8;
  if (plain) {
    block_apply64_kernel<<<(unsigned)nba, 256, 0, s>>>(g.d_binv, g.d_boff, g.d_bptr, g.d_bdofs,
                                                        (int)g.n_blocks, N, r, z, st);
    g.launches += 1;
    if (NH > 0) {
      restrict_kernel<<<(unsigned)NH, 256, 0, s>>>(g.d_cptr, g.d_crow, g.d_cval, NH, r, t, st);
      ++g.launches;
    }
  } else {
    if (!in_iteration) {
      to_df_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, g.d_rf, N, st);
      ++g.launches;
    }
    // block solves and coarse restriction: one launch
    block_restrict_kernel<<<(unsigned)(nba + NH), 256, 0, s>>>(g.d_binvf, g.d_boff, g.d_bptr, g.d_bdofs,
                                                               (int)g.n_blocks, N, g.d_rf, z, nba, g.d_cptr,
                                                               g.d_crow, g.d_cval, r, t, st);
    ++g.launches;
  }
  if (NH > 0) {
    coarse_solve_kernel<<<(unsigned)((NH + 7) / 8), 256, 0, s>>>(g.d_AHinv, NH, t, u, st);
    if (in_iteration)
      prolong_dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, u, z, r, part, st);
    else
      prolong_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(g.d_pptr, g.d_pcol, g.d_pval, N, u, z, st);
    g.launches += 2;
  } else if (in_iteration) {
    dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, z, N, part, st);
    ++g.launches;
  }
}

// one PCG iteration (all kernels guard on the device-side done flag); with a
// null stream only the launch counter is advanced
// count_only: add this iteration's launches to g.launches without launching
// (s may then be anything; a null s is the legacy default stream otherwise)
static void enqueue_iteration(DevGeom& g, int precondition, bool plain, double* hist, int hcap,
                              cudaStream_t s, bool count_only = false) {
  const int64_t N = g.ndof;
  double* x = g.d_vec;
  double* r = x + N;
  double* z = r + N;
  double* p = z + N;
  double* q = p + N;
  double* t = q + N;
  double* u = t + std::max<int64_t>(g.n_coarse, 1);
  double* scal = g.d_scal;
  PcgState* st = (PcgState*)(scal + 8);
  double* part = scal + 16;
  const unsigned gemv_blocks = matvec_blocks(N, 0);
  if (count_only) {
    // 9 + the product + the preconditioner's launches (which end with r . z)
    const bool coarse = precondition && g.use_coarse && g.n_coarse > 0;
    g.launches += 9 + (!precondition ? 2 : plain ? (coarse ? 4 : 2) : (coarse ? 3 : 2));
    return;
  }
  double* alpha_h = hist + hcap + 1;
  double* beta_h = alpha_h + hcap;
  if (plain)
    gemv64_kernel<<<(unsigned)((N + 15) / 16), 256, 0, s>>>(g.d_W64, N, p, q, part, st);
  else
    launch_matvec(0, g.tm_W, g.tm_p, N, 1, p, q, part, &st->done, &st->err, s);
  reduce_kernel<<<1, 256, 0, s>>>(part, plain ? (unsigned)((N + 15) / 16) : gemv_blocks, scal + 1, st);
  alpha_kernel<<<1, 1, 0, s>>>(scal, st, alpha_h);
  update_xr_kernel<<<RED_BLOCKS, 256, 0, s>>>(x, r, p, q, scal, N, part,
                                             (precondition && !plain) ? g.d_rf : nullptr, st);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 3, st);
  check_kernel<<<1, 1, 0, s>>>(scal, st, hist);
  // z = M r and the partial sums of r . z (its last launch carries them)
  apply_M(g, r, z, t, u, precondition, plain, st, s, true, part);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 4, st);
  beta_kernel<<<1, 1, 0, s>>>(scal, st, beta_h);
  update_p_kernel<<<RED_BLOCKS, 256, 0, s>>>(p, g.d_pfp, g.ldw, z, scal, N, 0, st);
  g.launches += 9;
}

void drop_pcg_graphs(DevGeom& g) {
  for (auto& ex : g.pcg_exec)
    if (ex) {
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
}

// q = W p with the FP64 copy of W (the comparator's product); stop as in PcgState.done
void launch_gemv64(const DevGeom& g, const double* p, double* q, double* part, const int* stop, cudaStream_t s) {
  gemv64_kernel<<<(unsigned)((g.ndof + 15) / 16), 256, 0, s>>>(g.d_W64, g.ndof, p, q, part,
                                                                (const PcgState*)stop);
}

cudaError_t ensure_w64(DevGeom& g, cudaStream_t s) {
  if (g.d_W64 || g.ndof == 0) return cudaSuccess;
  cudaError_t e = pool_alloc((void**)&g.d_W64, sizeof(double) * g.ndof * g.ndof, g.pool, s);
  if (e != cudaSuccess) return e;
  ++g.launches;
  return copy_rows_to_double(g, 0, g.ndof, g.d_W64, s);
}

cudaError_t run_pcg(DevGeom& g, const double gvec[3], double rtol, int maxit, int fixed,
                    int precondition, int precision, double* x_out, PcgOut& out, cudaStream_t s) {
  const bool plain = precision == 1;
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
  PcgState* st = (PcgState*)(scal + 8);
  double* part = scal + 16;   // partial sums (>= max(RED_BLOCKS, N/8+1))
  cudaError_t e;
  if (N == 0) {  // nothing to solve (no launch may have an empty grid)
    out.hist.push_back(0.0);
    out.status = MSBEM_OK;
    return cudaStreamSynchronize(s);
  }
  // residual / alpha / beta history: the persistent per-geometry buffer (laid
  // out for hist_cap iterations, so the captured graph can address it) when
  // maxit fits, else a temporary one
  const int hcap = maxit <= g.hist_cap ? g.hist_cap : maxit;
  double* hist = g.d_hist;
  if (maxit > g.hist_cap || !hist) {
    if ((e = pool_alloc((void**)&hist, sizeof(double) * (3 * (size_t)hcap + 1), g.pool, s)) != cudaSuccess)
      return e;
  }
  auto drop = [&](cudaError_t err) {  // error exit: a temporary history goes back to the pool
    if (hist != g.d_hist) cudaFreeAsync(hist, s);
    return err;
  };
  PcgState h_st = {0, 0, maxit, fixed, 0};
  cudaMemcpyAsync(st, &h_st, sizeof(PcgState), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(x, 0, sizeof(double) * N, s);
  if ((e = launch_rhs(g, gvec, r, s)) != cudaSuccess) return drop(e);
  dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, r, N, part, st);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 6, st);
  if (plain && (e = ensure_w64(g, s)) != cudaSuccess) return drop(e);
  apply_M(g, r, z, t, u, precondition, plain, st, s);
  update_p_kernel<<<RED_BLOCKS, 256, 0, s>>>(p, g.d_pfp, g.ldw, z, scal, N, 1, st);
  dot_kernel<<<RED_BLOCKS, 256, 0, s>>>(r, z, N, part, st);
  reduce_kernel<<<1, 256, 0, s>>>(part, RED_BLOCKS, scal + 0, st);
  cudaMemcpyAsync(scal + 7, &rtol, sizeof(double), cudaMemcpyHostToDevice, s);
  g.launches += 6;
  double nL2 = 0.0;
  if ((e = cudaMemcpyAsync(&nL2, scal + 6, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return drop(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
  if (nL2 == 0.0) {
    out.hist.push_back(0.0);
    out.status = MSBEM_OK;
    if (hist != g.d_hist) cudaFreeAsync(hist, s);
    if (x_out != x) cudaMemcpyAsync(x_out, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    return cudaStreamSynchronize(s);
  }
  const bool graphed = hist == g.d_hist && g.cap_stream != nullptr;
  const int gi = (precondition ? 1 : 0) + (plain ? 2 : 0);
  if (graphed && !g.pcg_exec[gi]) {
    // capture one chunk of iterations on the private stream
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(g.cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return drop(e);
    const int64_t before = g.launches;
    for (int c = 0; c < PCG_CHUNK; ++c) enqueue_iteration(g, precondition, plain, hist, hcap, g.cap_stream);
    g.launches = before;
    if ((e = cudaStreamEndCapture(g.cap_stream, &graph)) != cudaSuccess) return drop(e);
    e = cudaGraphInstantiate(&g.pcg_exec[gi], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return drop(e);
  }
  int enq = 0;
  while (enq < maxit) {
    if (graphed) {
      const int64_t before = g.launches;
      enqueue_iteration(g, precondition, plain, hist, hcap, nullptr, true);  // count only
      const int64_t per_iter = g.launches - before;
      g.launches = before + per_iter * PCG_CHUNK;
      if ((e = cudaGraphLaunch(g.pcg_exec[gi], s)) != cudaSuccess) return drop(e);
      enq += PCG_CHUNK;
    } else {
      const int chunk = std::min(PCG_CHUNK, maxit - enq);
      for (int c = 0; c < chunk; ++c) enqueue_iteration(g, precondition, plain, hist, hcap, s);
      enq += chunk;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return drop(e);
    if ((e = cudaMemcpyAsync(&h_st, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return drop(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
    if (h_st.done) break;
  }
  const int it = h_st.iter;
  std::vector<double> h(3 * (size_t)hcap + 1);
  cudaMemcpyAsync(h.data(), hist, sizeof(double) * (3 * (size_t)hcap + 1), cudaMemcpyDeviceToHost, s);
  if (hist != g.d_hist) cudaFreeAsync(hist, s);
  if (x_out != x) cudaMemcpyAsync(x_out, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  out.iters = it;
  out.hist.assign(1, 1.0);
  for (int k = 1; k <= it; ++k) out.hist.push_back(h[k]);
  out.alpha.assign(h.begin() + hcap + 1, h.begin() + hcap + 1 + it);
  const int nbeta = (h_st.done == 1 || h_st.done == 3) ? it - 1 : it;
  out.beta.assign(h.begin() + 2 * hcap + 1, h.begin() + 2 * hcap + 1 + std::max(0, nbeta));
  if (h_st.done == 2) out.status = MSBEM_BREAKDOWN;
  else if (h_st.done == 3) out.status = MSBEM_NOT_CONVERGED;
  else if (h_st.done == 5) out.status = MSBEM_DEVICE_TIMEOUT;
  else out.status = MSBEM_OK;
  return cudaSuccess;
}

}  // namespace msbem
