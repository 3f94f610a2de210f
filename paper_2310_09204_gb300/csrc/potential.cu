// Double-layer potential of a computed jump at target points off the screen
// (Lemma lemrepDL, eq. formulaDL):
//
//   U(x) = sum_T sum_a J_{T,a} int_T n_T . (y - x) lambda_a(y) / (4 pi |x - y|^3) dy,
//   J_{T,a} = sum_nu Phi_nu (c_+ - c_-)(T, a, nu)   (the two sides of T combined),
//
// each triangle integrated by the 6-point rule, optionally on its 4^refine
// congruent sub-triangles.  FP64 throughout: the quadrature points carry
// charges q = w |T| / 4^refine sum_a J_{T,a} lambda_a(y); every thread owns a
// target and sums a range of points staged through shared memory; the point
// range is split over several CTAs when there are few targets, and a second
// kernel adds the splits in fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "msbem_internal.h"

namespace msbem {

#define DL_TILE 128   // points staged per step

// points of triangle T, sub-triangle s, rule point p:  y, n_T, charge
__global__ void dl_points_kernel(const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                                 const double* __restrict__ area, const double* __restrict__ J,
                                 const double* __restrict__ beta,   // [nsub*6][3] barycentrics in T
                                 const double* __restrict__ wq,     // [6] rule weights (sum 1)
                                 int64_t nt, int nsub, double* __restrict__ pts) {   // [npts][7]
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nsub * 6;
  if (e >= nt * per) return;
  const int64_t T = e / per;
  const int sp = (int)(e - T * per);
  const double* b = beta + 3 * sp;
  const double* X0 = xyz + 3 * tri[3 * T];
  const double* X1 = xyz + 3 * tri[3 * T + 1];
  const double* X2 = xyz + 3 * tri[3 * T + 2];
  double e1[3], e2[3], n[3];
  for (int k = 0; k < 3; ++k) {
    e1[k] = X1[k] - X0[k];
    e2[k] = X2[k] - X0[k];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double* o = pts + 7 * e;
  for (int k = 0; k < 3; ++k) o[k] = b[0] * X0[k] + b[1] * X1[k] + b[2] * X2[k];
  for (int k = 0; k < 3; ++k) o[3 + k] = n[k] / nn;
  const double* j = J + 3 * T;
  o[6] = wq[sp % 6] * area[T] / nsub * (j[0] * b[0] + j[1] * b[1] + j[2] * b[2]);
}

// partial[s][m] = sum over the points of split s of q n . (y - x_m) / (4 pi |y - x_m|^3)
__global__ void __launch_bounds__(256) dl_eval_kernel(const double* __restrict__ pts, int64_t npts,
                                                      int64_t per_split, const double* __restrict__ X,
                                                      int64_t M, double* __restrict__ partial) {
  __shared__ double sp[DL_TILE * 7];
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.y * per_split;
  const int64_t p1 = (npts < p0 + per_split) ? npts : p0 + per_split;
  double x0 = 0.0, x1 = 0.0, x2 = 0.0;
  if (m < M) {
    x0 = X[3 * m];
    x1 = X[3 * m + 1];
    x2 = X[3 * m + 2];
  }
  double acc = 0.0;
  for (int64_t c = p0; c < p1; c += DL_TILE) {
    const int len = (int)((p1 - c) < DL_TILE ? (p1 - c) : DL_TILE);
    __syncthreads();
    for (int k = threadIdx.x; k < len * 7; k += blockDim.x) sp[k] = pts[7 * c + k];
    __syncthreads();
    for (int q = 0; q < len; ++q) {
      const double* s = sp + 7 * q;
      const double d0 = s[0] - x0, d1 = s[1] - x1, d2 = s[2] - x2;
      const double r2 = fma(d0, d0, fma(d1, d1, d2 * d2));
      const double ir = rsqrt(r2);
      const double nd = fma(s[3], d0, fma(s[4], d1, s[5] * d2));
      acc = fma(s[6] * nd, ir * ir * ir, acc);
    }
  }
  if (m < M) partial[blockIdx.y * M + m] = acc * (0.25 / M_PI);
}

__global__ void dl_combine_kernel(const double* __restrict__ partial, int S, int64_t M, double* __restrict__ out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int k = 0; k < S; ++k) s += partial[k * M + m];
  out[m] = s;
}

// Barycentric coordinates in T of the 6 rule points of each of the 4^refine
// sub-triangles (uniform subdivision of the reference triangle).
static void subdivided_points(int refine, const double bary[6][3], std::vector<double>& beta) {
  const int m = 1 << refine;
  beta.clear();
  auto B = [m](int a, int b, double* o) {
    o[0] = 1.0 - (double)(a + b) / m;
    o[1] = (double)a / m;
    o[2] = (double)b / m;
  };
  auto emit = [&](const double* B0, const double* B1, const double* B2) {
    for (int p = 0; p < 6; ++p)
      for (int k = 0; k < 3; ++k) beta.push_back(bary[p][0] * B0[k] + bary[p][1] * B1[k] + bary[p][2] * B2[k]);
  };
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m - j; ++i) {
      double a0[3], a1[3], a2[3];
      B(i, j, a0);
      B(i + 1, j, a1);
      B(i, j + 1, a2);
      emit(a0, a1, a2);
      if (i + j + 1 < m) {
        double c0[3], c1[3], c2[3];
        B(i + 1, j, c0);
        B(i + 1, j + 1, c1);
        B(i, j + 1, c2);
        emit(c0, c1, c2);
      }
    }
}

cudaError_t dl_potential(DevGeom& g, const std::vector<double>& J, const double* X_dev, int64_t M, int refine,
                         double* out_dev, float* kernel_ms, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  double bary[6][3], w[6];
  six_point_rule(bary, w);
  std::vector<double> beta;
  subdivided_points(refine, bary, beta);
  const int nsub = (int)(beta.size() / 18);
  const int64_t npts = g.nt * nsub * 6;
  // split the points so that (target blocks x splits) fills about four waves
  const int64_t mblocks = (M + 255) / 256;
  int S = (int)std::min<int64_t>(64, std::max<int64_t>(1, (4 * 2 * 152 + mblocks - 1) / mblocks));
  S = (int)std::min<int64_t>(S, std::max<int64_t>(1, npts / DL_TILE));
  const int64_t per = (npts + S - 1) / S;
  const size_t bytes = sizeof(double) * (3 * g.nt + beta.size() + 6 + 7 * npts + (size_t)S * M) + 256;
  char* base = nullptr;
  cudaError_t e = pool_alloc((void**)&base, bytes, g.pool, s);
  if (e != cudaSuccess) return e;
  char* cur = base;
  auto take = [&](size_t n) { double* p = (double*)cur; cur += (sizeof(double) * n + 15) / 16 * 16; return p; };
  double* dJ = take(3 * g.nt);
  double* dB = take(beta.size());
  double* dW = take(6);
  double* dP = take(7 * npts);
  double* part = take((size_t)S * M);
  cudaMemcpyAsync(dJ, J.data(), sizeof(double) * 3 * g.nt, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dB, beta.data(), sizeof(double) * beta.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dW, w, sizeof(double) * 6, cudaMemcpyHostToDevice, s);
  dl_points_kernel<<<(unsigned)((npts + 255) / 256), 256, 0, s>>>(g.d_xyz, g.d_tri, g.d_area, dJ, dB, dW, g.nt,
                                                                   nsub, dP);
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  cudaEventRecord(ev[0], s);
  dl_eval_kernel<<<dim3((unsigned)mblocks, (unsigned)S), 256, 0, s>>>(dP, npts, per, X_dev, M, part);
  cudaEventRecord(ev[1], s);
  dl_combine_kernel<<<(unsigned)mblocks, 256, 0, s>>>(part, S, M, out_dev);
  g.launches += 3;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && kernel_ms) cudaEventElapsedTime(kernel_ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaFreeAsync(base, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace msbem
