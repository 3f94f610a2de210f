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
#include <vector>

#include "msbem_internal.h"

namespace msbem {

__global__ void gather_blocks_kernel(const double* __restrict__ W, int64_t N,
                                     const int64_t* __restrict__ bptr,
                                     const int32_t* __restrict__ bdofs,
                                     const int64_t* __restrict__ boff,
                                     const int64_t* __restrict__ prefix2, int nblk, int wb_block,
                                     int wb_diag, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prefix2[nblk]) return;
  int b = 0;
  while (b + 1 < nblk && prefix2[b + 1] <= t) ++b;
  const int64_t n = bptr[b + 1] - bptr[b];
  const int64_t e = t - prefix2[b];
  const int64_t i = e / n, j = e % n;
  const int64_t di = bdofs[bptr[b] + i], dj = bdofs[bptr[b] + j];
  double v = W[di * N + dj];
  if (b == wb_block && wb_diag) v = (i == j) ? 1.0 / v : 0.0;
  out[boff[b] + e] = v;
}

// W P  (transposed, NH x N) from the CSC form of P:  (W P)^T[mu][i] = sum_nu P[nu,mu] W[nu][i]
__global__ void wp_kernel(const double* __restrict__ W, int64_t N, const int64_t* __restrict__ cptr,
                          const int32_t* __restrict__ crow, const double* __restrict__ cval,
                          double* __restrict__ WPt) {
  const int64_t mu = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int64_t k = cptr[mu]; k < cptr[mu + 1]; ++k) acc = fma(cval[k], W[(int64_t)crow[k] * N + i], acc);
  WPt[mu * N + i] = acc;
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

// Gauss-Jordan step k on every active block: save pivot row and column ...
__global__ void gj_save_kernel(double* __restrict__ A, const int64_t* __restrict__ boff,
                               const int64_t* __restrict__ bsize, const int32_t* __restrict__ order,
                               const int64_t* __restrict__ prefix1, int active, int64_t k,
                               double* __restrict__ save, int* __restrict__ flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prefix1[active]) return;
  int a = 0;
  while (a + 1 < active && prefix1[a + 1] <= t) ++a;
  const int b = order[a];
  const int64_t n = bsize[b];
  const int64_t e = t - prefix1[a];
  const double* M = A + boff[b];
  double v = (e < n) ? M[k * n + e] : M[(e - n) * n + k];
  save[t] = v;
  if (e == k) {
    if (!(v > 0.0) || !isfinite(v)) atomicExch(flag, 1);
  }
}

// ... then update all entries of every active block.
__global__ void gj_update_kernel(double* __restrict__ A, const int64_t* __restrict__ boff,
                                 const int64_t* __restrict__ bsize, const int32_t* __restrict__ order,
                                 const int64_t* __restrict__ prefix1,
                                 const int64_t* __restrict__ prefix2, int active, int64_t k,
                                 const double* __restrict__ save) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= prefix2[active]) return;
  int a = 0;
  while (a + 1 < active && prefix2[a + 1] <= t) ++a;
  const int b = order[a];
  const int64_t n = bsize[b];
  const int64_t e = t - prefix2[a];
  const int64_t i = e / n, j = e % n;
  const double* rowk = save + prefix1[a];
  const double* colk = rowk + n;
  const double p = rowk[k];
  const double ip = 1.0 / p;
  double* M = A + boff[b];
  double v;
  if (i == k && j == k) v = ip;
  else if (i == k) v = rowk[j] * ip;
  else if (j == k) v = -colk[i] * ip;
  else v = fma(-colk[i] * ip, rowk[j], M[e]);
  M[e] = v;
}

namespace {
template <class T>
cudaError_t upload(T** d, const std::vector<T>& h, cudaStream_t s) {
  cudaError_t e = cudaMallocAsync((void**)d, sizeof(T) * std::max<size_t>(1, h.size()), s);
  if (e != cudaSuccess) return e;
  if (h.empty()) return cudaSuccess;
  return cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
}
}  // namespace

// Inverts the blocks listed in `inv_blocks` (ids into the packed layout given by
// boff/bsize) in place.  bsize/boff are host vectors.
static cudaError_t gj_invert(double* d_A, const std::vector<int64_t>& boff,
                             const std::vector<int64_t>& bsize, std::vector<int32_t> inv_blocks,
                             cudaStream_t s, int* not_spd, int64_t* launches) {
  *not_spd = 0;
  if (inv_blocks.empty()) return cudaSuccess;
  std::sort(inv_blocks.begin(), inv_blocks.end(),
            [&](int a, int b) { return bsize[a] > bsize[b]; });
  const int nb = (int)inv_blocks.size();
  std::vector<int64_t> p1(nb + 1, 0), p2(nb + 1, 0);
  for (int a = 0; a < nb; ++a) {
    p1[a + 1] = p1[a] + 2 * bsize[inv_blocks[a]];
    p2[a + 1] = p2[a] + bsize[inv_blocks[a]] * bsize[inv_blocks[a]];
  }
  int64_t *d_boff = nullptr, *d_bsize = nullptr, *d_p1 = nullptr, *d_p2 = nullptr;
  int32_t* d_order = nullptr;
  double* d_save = nullptr;
  int* d_flag = nullptr;
  cudaError_t e;
  if ((e = upload(&d_boff, boff, s)) != cudaSuccess) return e;
  if ((e = upload(&d_bsize, bsize, s)) != cudaSuccess) return e;
  if ((e = upload(&d_p1, p1, s)) != cudaSuccess) return e;
  if ((e = upload(&d_p2, p2, s)) != cudaSuccess) return e;
  if ((e = upload(&d_order, inv_blocks, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync((void**)&d_save, sizeof(double) * p1[nb], s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync((void**)&d_flag, sizeof(int), s)) != cudaSuccess) return e;
  cudaMemsetAsync(d_flag, 0, sizeof(int), s);
  const int64_t nmax = bsize[inv_blocks[0]];
  int active = nb;
  for (int64_t k = 0; k < nmax; ++k) {
    while (active > 0 && bsize[inv_blocks[active - 1]] <= k) --active;
    gj_save_kernel<<<(unsigned)((p1[active] + 255) / 256), 256, 0, s>>>(
        d_A, d_boff, d_bsize, d_order, d_p1, active, k, d_save, d_flag);
    gj_update_kernel<<<(unsigned)((p2[active] + 255) / 256), 256, 0, s>>>(
        d_A, d_boff, d_bsize, d_order, d_p1, d_p2, active, k, d_save);
    *launches += 2;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int flag = 0;
  cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  *not_spd = flag;
  cudaFreeAsync(d_boff, s);
  cudaFreeAsync(d_bsize, s);
  cudaFreeAsync(d_p1, s);
  cudaFreeAsync(d_p2, s);
  cudaFreeAsync(d_order, s);
  cudaFreeAsync(d_save, s);
  cudaFreeAsync(d_flag, s);
  return cudaSuccess;
}

// Gathers face / wire-basket blocks and the coarse matrix into g.d_binv and
// inverts them.  bptr: block pointer (faces first, wire basket last if any).
cudaError_t factor_blocks(DevGeom& g, const std::vector<int64_t>& bptr, int wb_diag, cudaStream_t s,
                          int* not_spd) {
  *not_spd = 0;
  const int nblk = (int)bptr.size() - 1;
  const bool has_wb = g.n_blocks > 0 && nblk > 0;  // caller guarantees layout
  std::vector<int64_t> bsize(nblk + 1), boff(nblk + 2, 0), prefix2(nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) {
    bsize[b] = bptr[b + 1] - bptr[b];
    boff[b + 1] = boff[b] + bsize[b] * bsize[b];
    prefix2[b + 1] = prefix2[b] + bsize[b] * bsize[b];
  }
  const int64_t NH = g.use_coarse ? g.n_coarse : 0;
  bsize[nblk] = NH;
  boff[nblk + 1] = boff[nblk] + NH * NH;
  (void)has_wb;
  cudaError_t e;
  if (g.d_binv) { cudaFreeAsync(g.d_binv, s); g.d_binv = nullptr; }
  if (g.d_boff) { cudaFreeAsync(g.d_boff, s); g.d_boff = nullptr; }
  g.binv_size = boff[nblk + 1];
  if ((e = cudaMallocAsync((void**)&g.d_binv, sizeof(double) * std::max<int64_t>(1, g.binv_size), s)) !=
      cudaSuccess)
    return e;
  if ((e = upload(&g.d_boff, boff, s)) != cudaSuccess) return e;
  int64_t* d_prefix2 = nullptr;
  if ((e = upload(&d_prefix2, prefix2, s)) != cudaSuccess) return e;
  const int wb_block = (g.n_blocks > 0 && g.wb_diag >= 0) ? nblk - 1 : -1;
  if (prefix2[nblk] > 0) ++g.launches;
  if (prefix2[nblk] > 0)
    gather_blocks_kernel<<<(unsigned)((prefix2[nblk] + 255) / 256), 256, 0, s>>>(
        g.d_W, g.ndof, g.d_bptr, g.d_bdofs, g.d_boff, d_prefix2, nblk, wb_block, wb_diag, g.d_binv);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaFreeAsync(d_prefix2, s);
  std::vector<int32_t> inv;
  for (int b = 0; b < nblk; ++b)
    if (!(wb_diag && b == wb_block) && bsize[b] > 0) inv.push_back(b);
  if (NH > 0 && g.ndof > 0) {
    // A_H = P^T W P in the last slot
    dim3 grid((unsigned)((g.ndof + 255) / 256), (unsigned)NH);
    wp_kernel<<<grid, 256, 0, s>>>(g.d_W, g.ndof, g.d_cptr, g.d_crow, g.d_cval, g.d_WP);
    dim3 grid2((unsigned)NH, (unsigned)((NH + 127) / 128));
    ah_kernel<<<grid2, 128, 0, s>>>(g.d_WP, g.ndof, NH, g.d_cptr, g.d_crow, g.d_cval,
                                    g.d_binv + boff[nblk]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    g.launches += 2;
    inv.push_back(nblk);
  }
  std::vector<int64_t> bsz(bsize.begin(), bsize.end());
  std::vector<int64_t> bof(boff.begin(), boff.end() - 1);
  return gj_invert(g.d_binv, bof, bsz, inv, s, not_spd, &g.launches);
}

}  // namespace msbem
