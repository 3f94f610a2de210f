// Assembly of the hypersingular Galerkin matrix on sm_103a.
//
// a(psi~_nu, psi~_nu') = sum_{T,T'} V_{TT'} s_{T,nu} . s_{T',nu'}   (Sec. 4.3,
// eq. eval_a_phiij with Cor. corW), where s_{T,nu} is the constant surface curl
// of the jump of psi_nu on T and V_{TT'} = int_T int_T' 1/(4 pi |x-y|).
//
// Kernels:
//   far_fp64_kernel  V_{TT'} for all pairs of a 64x64 triangle tile, 6x6 points
//                    (native FP64); tiles on and above the diagonal only, the
//                    lower half written by a shared-memory transpose.
//   near_kernel /    pairs sharing a vertex: Sauter-Schwab-type rules (identical
//   near_df_kernel   (FP64 and double-float versions)
//                    6 regions, edge 4, vertex 2) with Gauss-Legendre order n.
//                    For a kernel of x - y on flat triangles the rules' integrand
//                    does not depend on some of the [0,1]^4 coordinates, and is a
//                    polynomial in the radial one; those coordinates are summed in
//                    closed form (1/3 * 1/2, 1/6, 1/3), which is exact for
//                    Gauss-Legendre of any order >= 2.  One warp per pair,
//                    warp-shuffle reduction over the quadrature points.
//   contract_kernel  W[nu,nu'] = sum_{k in J(nu)} sum_{k' in J(nu')} V[T_k,T_k'] s_k.s_k'
//                    (double-float on the FP32 pipe)
//   rhs_kernel       L_nu = sum_{k in J(nu)} (c_+ - c_-)(g.n_T)|T|/3
#include <algorithm>
#include <cstdio>

#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define FAR_TILE 64
__constant__ double c_far_w[6];        // 6-point rule weights (sum 1)

cudaError_t set_far_constants(const double bary[6][3], const double w[6]) {
  (void)bary;
  return cudaMemcpyToSymbol(c_far_w, w, sizeof(double) * 6);
}

// tile index -> (bi, bj) with bi <= bj, row-major over the upper triangle
__device__ __forceinline__ void tile_coords(int64_t t, int nb, int& bi, int& bj) {
  // rows have nb, nb-1, ... tiles; solve for bi
  double disc = (2.0 * nb + 1.0) * (2.0 * nb + 1.0) - 8.0 * (double)t;
  int r = (int)floor(((2.0 * nb + 1.0) - sqrt(disc)) * 0.5);
  if (r < 0) r = 0;
  auto start = [nb](int64_t row) { return row * (int64_t)nb - row * (row - 1) / 2; };
  while (r > 0 && start(r) > t) --r;
  while (r + 1 < nb && start(r + 1) <= t) ++r;
  bi = r;
  bj = (int)(r + (t - start(r)));
}

__global__ void __launch_bounds__(256) far_fp64_kernel(const double* __restrict__ qp,
                                                       const double* __restrict__ area,
                                                       const int32_t* __restrict__ tri, int nb,
                                                       int64_t nt, int64_t ldv,
                                                       float2* __restrict__ V) {
  __shared__ double s_q[FAR_TILE * 18];
  __shared__ double s_area[FAR_TILE];
  __shared__ int32_t s_tri[FAR_TILE * 3];
  __shared__ double s_out[FAR_TILE][FAR_TILE + 1];
  int bi, bj;
  tile_coords(blockIdx.x, nb, bi, bj);
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)bi * FAR_TILE, col0 = (int64_t)bj * FAR_TILE;
  for (int i = tid; i < FAR_TILE * 18; i += blockDim.x) s_q[i] = qp[col0 * 18 + i];
  for (int i = tid; i < FAR_TILE; i += blockDim.x) s_area[i] = area[col0 + i];
  for (int i = tid; i < FAR_TILE * 3; i += blockDim.x) s_tri[i] = tri[col0 * 3 + i];
  const int r = tid & 63;
  const int cgrp = tid >> 6;  // 4 groups of 16 columns
  const int64_t T = row0 + r;
  double x[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) x[k] = qp[T * 18 + k];
  const double aT = area[T];
  const int32_t t0 = tri[T * 3], t1 = tri[T * 3 + 1], t2 = tri[T * 3 + 2];
  __syncthreads();
  for (int cc = 0; cc < 16; ++cc) {
    const int c = cgrp * 16 + cc;
    const double* y = &s_q[c * 18];
    double acc = 0.0;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      double inner = 0.0;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        double dx = x[3 * p] - y[3 * q];
        double dy = x[3 * p + 1] - y[3 * q + 1];
        double dz = x[3 * p + 2] - y[3 * q + 2];
        double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        inner = fma(c_far_w[q], rsqrt(r2), inner);
      }
      acc = fma(c_far_w[p], inner, acc);
    }
    const int32_t u0 = s_tri[3 * c], u1 = s_tri[3 * c + 1], u2 = s_tri[3 * c + 2];
    bool touch = (t0 == u0) | (t0 == u1) | (t0 == u2) | (t1 == u0) | (t1 == u1) | (t1 == u2) |
                 (t2 == u0) | (t2 == u1) | (t2 == u2) | (t0 < 0) | (u0 < 0);
    double v = touch ? 0.0 : aT * s_area[c] * acc * (0.25 / M_PI);
    s_out[r][c] = v;
  }
  __syncthreads();
  // coalesced stores of the tile and of its transpose, as (hi, lo) floats
  for (int i = tid; i < FAR_TILE * FAR_TILE; i += blockDim.x) {
    int rr = i / FAR_TILE, c = i % FAR_TILE;
    int64_t R = row0 + rr, C = col0 + c;
    float h, l;
    split_df(s_out[rr][c], h, l);
    if (R < nt && C < nt) V[R * ldv + C] = make_float2(h, l);
  }
  if (bi != bj) {
    for (int i = tid; i < FAR_TILE * FAR_TILE; i += blockDim.x) {
      int c = i / FAR_TILE, rr = i % FAR_TILE;
      int64_t R = row0 + rr, C = col0 + c;
      float h, l;
      split_df(s_out[rr][c], h, l);
      if (R < nt && C < nt) V[C * ldv + R] = make_float2(h, l);
    }
  }
}

cudaError_t launch_far_fp64(const DevGeom& g, cudaStream_t s) {
  int nb = (int)(g.nt_pad / FAR_TILE);
  int64_t tiles = (int64_t)nb * (nb + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  far_fp64_kernel<<<(unsigned)tiles, 256, 0, s>>>(g.d_qp, g.d_area, g.d_tri, nb, g.nt, g.nt, g.d_V);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Near field
// ---------------------------------------------------------------------------
#define NEAR_MAXN 16
// Gauss-Legendre nodes and weights on [0,1] of the singular rules, FP64 and
// as float pairs; passed by value to the near-field kernels (so contexts that
// assemble concurrently with different orders do not share a table)
struct GLTable {
  double x[NEAR_MAXN], w[NEAR_MAXN];
  float2 xf[NEAR_MAXN], wf[NEAR_MAXN];
};

__device__ __forceinline__ double inv_norm3(double a, double b, double c) {
  return rsqrt(fma(c, c, fma(b, b, a * a)));
}

__device__ __forceinline__ double tri_area_d(const double* P) {
  double e1x = P[3] - P[0], e1y = P[4] - P[1], e1z = P[5] - P[2];
  double e2x = P[6] - P[0], e2y = P[7] - P[1], e2z = P[8] - P[2];
  double cx = e1y * e2z - e1z * e2y, cy = e1z * e2x - e1x * e2z, cz = e1x * e2y - e1y * e2x;
  return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

__global__ void __launch_bounds__(256) near_kernel(const __grid_constant__ GLTable gl,
                                                   const NearPair* __restrict__ pairs, int64_t npairs,
                                                   const double* __restrict__ xyz, int n, int64_t ldv,
                                                   float2* __restrict__ V, int64_t t0, int64_t t1) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= npairs) return;
  const NearPair pr = pairs[w];
  double P[9], Q[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      P[3 * i + k] = xyz[3 * (int64_t)pr.v[i] + k];
      Q[3 * i + k] = xyz[3 * (int64_t)pr.v[3 + i] + k];
    }
  const double aT = tri_area_d(P), aS = tri_area_d(Q);
  double sum = 0.0, pref;
  if (pr.cls == 3) {
    // identical: 1/|x-y| = 1/(xi |J w(eta)|); sectors s and s+3 coincide
    const double e1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
    const double e2[3] = {P[6] - P[3], P[7] - P[4], P[8] - P[5]};
    for (int idx = lane; idx < 3 * n; idx += 32) {
      int s = idx / n, j = idx % n;
      double et = gl.x[j];
      double a0, a1;  // J w = a0 e1 + a1 e2
      if (s == 0) { a0 = 1.0; a1 = et; }
      else if (s == 1) { a0 = 1.0 - et; a1 = 1.0; }
      else { a0 = -et; a1 = 1.0 - et; }
      sum += gl.w[j] * inv_norm3(a0 * e1[0] + a1 * e2[0], a0 * e1[1] + a1 * e2[1],
                                   a0 * e1[2] + a1 * e2[2]);
    }
    pref = aT * aT / (3.0 * M_PI);
  } else if (pr.cls == 2) {
    // edge: x - y = xi (-f_u e + f_v c - f_w d) on 4 cones
    const double e[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
    const double c[3] = {P[6] - P[3], P[7] - P[4], P[8] - P[5]};
    const double d[3] = {Q[6] - Q[3], Q[7] - Q[4], Q[8] - Q[5]};
    const int nn = n * n;
    for (int idx = lane; idx < 4 * nn; idx += 32) {
      int reg = idx / nn, rem = idx % nn, i1 = rem / n, i2 = rem % n;
      double sg = gl.x[i1], ta = gl.x[i2], wq = gl.w[i1] * gl.w[i2];
      double fu, fv, fw, J;
      if (reg == 0) { fu = sg; fv = 1.0 - sg; fw = ta; J = 1.0; }
      else if (reg == 1) { fu = sg * (1.0 - ta); fv = sg * ta; fw = 1.0; J = sg; }
      else if (reg == 2) { fu = -sg * (1.0 - ta); fv = 1.0; fw = sg * ta; J = sg; }
      else { fu = -sg; fv = ta; fw = 1.0 - sg; J = 1.0; }
      double gx = -fu * e[0] + fv * c[0] - fw * d[0];
      double gy = -fu * e[1] + fv * c[1] - fw * d[1];
      double gz = -fu * e[2] + fv * c[2] - fw * d[2];
      sum += wq * J * inv_norm3(gx, gy, gz);
    }
    pref = aT * aS / (6.0 * M_PI);
  } else {
    // vertex: 2 regions, x - y = xi g(e1,e2,e3)
    const double p1[3] = {P[3] - P[0], P[4] - P[1], P[5] - P[2]};
    const double p2[3] = {P[6] - P[3], P[7] - P[4], P[8] - P[5]};
    const double q1[3] = {Q[3] - Q[0], Q[4] - Q[1], Q[5] - Q[2]};
    const double q2[3] = {Q[6] - Q[3], Q[7] - Q[4], Q[8] - Q[5]};
    const int nnn = n * n * n;
    for (int idx = lane; idx < 2 * nnn; idx += 32) {
      int reg = idx / nnn, rem = idx % nnn;
      int i1 = rem / (n * n), i2 = (rem / n) % n, i3 = rem % n;
      double a1 = gl.x[i1], a2 = gl.x[i2], a3 = gl.x[i3];
      double wq = gl.w[i1] * gl.w[i2] * gl.w[i3] * a2;
      double s1, s2, t1, t2;
      if (reg == 0) { s1 = 1.0; s2 = a1; t1 = a2; t2 = a2 * a3; }
      else { t1 = 1.0; t2 = a1; s1 = a2; s2 = a2 * a3; }
      double gx = s1 * p1[0] + s2 * p2[0] - t1 * q1[0] - t2 * q2[0];
      double gy = s1 * p1[1] + s2 * p2[1] - t1 * q1[1] - t2 * q2[1];
      double gz = s1 * p1[2] + s2 * p2[2] - t1 * q1[2] - t2 * q2[2];
      sum += wq * inv_norm3(gx, gy, gz);
    }
    pref = aT * aS / (3.0 * M_PI);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if (lane == 0) {
    float h, l;
    split_df(pref * sum, h, l);
    // rows t0 .. t1-1 of V are held (all of them outside panel mode)
    if (pr.T >= t0 && pr.T < t1) V[(int64_t)(pr.T - t0) * ldv + pr.S] = make_float2(h, l);
    if (pr.S >= t0 && pr.S < t1) V[(int64_t)(pr.S - t0) * ldv + pr.T] = make_float2(h, l);
  }
}

// Same rules as near_kernel, evaluated in double-float on the FP32 pipe: per
// pair the edge vectors are formed in FP64 and split into float pairs; per
// evaluation the direction vector g, 1/|g| and the weighted sum use float pairs
// (Gauss-Legendre nodes and weights as (hi, lo) pairs in constant memory).

__device__ __forceinline__ void split3(const double* v, float2* o) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float h, l;
    split_df(v[k], h, l);
    o[k] = make_float2(h, l);
  }
}

// acc[k] += c * v[k]  (c a float pair, v a float-pair vector)
__device__ __forceinline__ void axpy3(float ch, float cl, const float2* v, float2* acc) {
#pragma unroll
  for (int k = 0; k < 3; ++k) df_fma_acc(ch, cl, v[k].x, v[k].y, acc[k].x, acc[k].y);
}

__global__ void __launch_bounds__(256) near_df_kernel(const __grid_constant__ GLTable gl,
                                                      const NearPair* __restrict__ pairs,
                                                      int64_t npairs, const double* __restrict__ xyz,
                                                      int n, int64_t ldv, float2* __restrict__ V,
                                                      int64_t t0, int64_t t1) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= npairs) return;
  const NearPair pr = pairs[w];
  double P[9], Q[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      P[3 * i + k] = xyz[3 * (int64_t)pr.v[i] + k];
      Q[3 * i + k] = xyz[3 * (int64_t)pr.v[3 + i] + k];
    }
  const double aT = tri_area_d(P), aS = tri_area_d(Q);
  double ev[4][3];
  // edge vectors (FP64 differences), split to float pairs
  for (int k = 0; k < 3; ++k) {
    ev[0][k] = P[3 + k] - P[k];      // identical: e1 | edge: e | vertex: p1
    ev[1][k] = P[6 + k] - P[3 + k];  // identical: e2 | edge: c | vertex: p2
    ev[2][k] = Q[6 + k] - Q[3 + k];  //                edge: d | vertex: q2
    ev[3][k] = Q[3 + k] - Q[k];      //                          vertex: q1
  }
  float2 v0[3], v1[3], v2[3], v3[3];
  split3(ev[0], v0);
  split3(ev[1], v1);
  split3(ev[2], v2);
  split3(ev[3], v3);
  float acch = 0.f, accl = 0.f;
  double pref;
  const float2 one = make_float2(1.f, 0.f);
  if (pr.cls == 3) {
    for (int idx = lane; idx < 3 * n; idx += 32) {
      const int sct = idx / n, j = idx % n;
      const float2 et = gl.xf[j];
      float2 om;  // 1 - eta
      df_add(1.f, 0.f, -et.x, -et.y, om.x, om.y);
      float2 a0, a1;
      if (sct == 0) { a0 = one; a1 = et; }
      else if (sct == 1) { a0 = om; a1 = one; }
      else { a0 = make_float2(-et.x, -et.y); a1 = om; }
      float2 g[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      axpy3(a0.x, a0.y, v0, g);
      axpy3(a1.x, a1.y, v1, g);
      float y, corr;
      df_rsqrt3(g[0].x, g[0].y, g[1].x, g[1].y, g[2].x, g[2].y, y, corr);
      const float2 wq = gl.wf[j];
      df_fma_acc(wq.x, wq.y, y, corr, acch, accl);
    }
    pref = aT * aT / (3.0 * M_PI);
  } else if (pr.cls == 2) {
    const int nn = n * n;
    for (int idx = lane; idx < 4 * nn; idx += 32) {
      const int reg = idx / nn, rem = idx % nn, i1 = rem / n, i2 = rem % n;
      const float2 sg = gl.xf[i1], ta = gl.xf[i2];
      float2 omt, oms, sgta, sgomt;
      df_add(1.f, 0.f, -ta.x, -ta.y, omt.x, omt.y);
      df_add(1.f, 0.f, -sg.x, -sg.y, oms.x, oms.y);
      df_mul(sg.x, sg.y, ta.x, ta.y, sgta.x, sgta.y);
      df_mul(sg.x, sg.y, omt.x, omt.y, sgomt.x, sgomt.y);
      float2 fu, fv, fw, J;
      if (reg == 0) { fu = sg; fv = oms; fw = ta; J = one; }
      else if (reg == 1) { fu = sgomt; fv = sgta; fw = one; J = sg; }
      else if (reg == 2) { fu = make_float2(-sgomt.x, -sgomt.y); fv = one; fw = sgta; J = sg; }
      else { fu = make_float2(-sg.x, -sg.y); fv = ta; fw = oms; J = one; }
      // g = -fu e + fv c - fw d
      float2 g[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      axpy3(-fu.x, -fu.y, v0, g);
      axpy3(fv.x, fv.y, v1, g);
      axpy3(-fw.x, -fw.y, v2, g);
      float y, corr;
      df_rsqrt3(g[0].x, g[0].y, g[1].x, g[1].y, g[2].x, g[2].y, y, corr);
      float2 wq, wJ;
      df_mul(gl.wf[i1].x, gl.wf[i1].y, gl.wf[i2].x, gl.wf[i2].y, wq.x, wq.y);
      df_mul(wq.x, wq.y, J.x, J.y, wJ.x, wJ.y);
      df_fma_acc(wJ.x, wJ.y, y, corr, acch, accl);
    }
    pref = aT * aS / (6.0 * M_PI);
  } else {
    const int nnn = n * n * n;
    for (int idx = lane; idx < 2 * nnn; idx += 32) {
      const int reg = idx / nnn, rem = idx % nnn;
      const int i1 = rem / (n * n), i2 = (rem / n) % n, i3 = rem % n;
      const float2 a1 = gl.xf[i1], a2 = gl.xf[i2], a3 = gl.xf[i3];
      float2 a23;
      df_mul(a2.x, a2.y, a3.x, a3.y, a23.x, a23.y);
      float2 s1, s2, t1, t2;
      if (reg == 0) { s1 = one; s2 = a1; t1 = a2; t2 = a23; }
      else { t1 = one; t2 = a1; s1 = a2; s2 = a23; }
      // g = s1 p1 + s2 p2 - t1 q1 - t2 q2
      float2 g[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      axpy3(s1.x, s1.y, v0, g);
      axpy3(s2.x, s2.y, v1, g);
      axpy3(-t1.x, -t1.y, v3, g);
      axpy3(-t2.x, -t2.y, v2, g);
      float y, corr;
      df_rsqrt3(g[0].x, g[0].y, g[1].x, g[1].y, g[2].x, g[2].y, y, corr);
      float2 w12, w123, wq;
      df_mul(gl.wf[i1].x, gl.wf[i1].y, gl.wf[i2].x, gl.wf[i2].y, w12.x, w12.y);
      df_mul(w12.x, w12.y, gl.wf[i3].x, gl.wf[i3].y, w123.x, w123.y);
      df_mul(w123.x, w123.y, a2.x, a2.y, wq.x, wq.y);
      df_fma_acc(wq.x, wq.y, y, corr, acch, accl);
    }
    pref = aT * aS / (3.0 * M_PI);
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
  if (lane == 0) {
    float h, l;
    split_df(pref * df_to_double(acch, accl), h, l);
    // rows t0 .. t1-1 of V are held (all of them outside panel mode)
    if (pr.T >= t0 && pr.T < t1) V[(int64_t)(pr.T - t0) * ldv + pr.S] = make_float2(h, l);
    if (pr.S >= t0 && pr.S < t1) V[(int64_t)(pr.S - t0) * ldv + pr.T] = make_float2(h, l);
  }
}

cudaError_t launch_near(const DevGeom& g, int n, const double* gl_x, const double* gl_w,
                        int fp64, cudaStream_t s, int64_t t0, int64_t t1) {
  if (t1 < 0) t1 = g.nt;
  if (n < 2 || n > NEAR_MAXN) return cudaErrorInvalidValue;
  GLTable gl{};
  for (int j = 0; j < n; ++j) {
    gl.x[j] = gl_x[j];
    gl.w[j] = gl_w[j];
    float xh = (float)gl_x[j], wh = (float)gl_w[j];
    gl.xf[j] = make_float2(xh, (float)(gl_x[j] - (double)xh));
    gl.wf[j] = make_float2(wh, (float)(gl_w[j] - (double)wh));
  }
  if (g.n_near == 0) return cudaSuccess;
  int64_t blocks = (g.n_near + 7) / 8;
  if (fp64)
    near_kernel<<<(unsigned)blocks, 256, 0, s>>>(gl, g.d_near, g.n_near, g.d_xyz, n, g.nt, g.d_V, t0, t1);
  else
    near_df_kernel<<<(unsigned)blocks, 256, 0, s>>>(gl, g.d_near, g.n_near, g.d_xyz, n, g.nt, g.d_V, t0, t1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Contraction W = sum S^T V S (gather form, upper triangle then mirrored)
// ---------------------------------------------------------------------------
#define CT 32
#define CT_CAP 512      // curl entries of a tile's 32 rows (or columns) kept in shared memory
#define CT_BATCH 4      // V gathers in flight per thread
// W[nu,nu'] = sum_{k in J(nu)} sum_{m in J(nu')} V[T_k,T_m] (s_k . s_m), in
// double-float on the FP32 pipe: V and the curl vectors are (hi, lo) float
// pairs; products are formed exactly with FMA and summed with two-sums.
// Upper-triangle 32x32 tiles; the curl lists of the tile's rows and columns
// (contiguous, since lists are stored by dof) are staged in shared memory, and
// the V gathers of one row entry against a column list are issued together.
// Diagonal tiles mirror their upper half so W is exactly symmetric.
// One W entry: sum over the row's curl entries [ka,kz) and the column's
// [ma,mz) (lists in shared memory when STAGED, else in global memory).
template <bool STAGED, bool PANEL = false>
__device__ __forceinline__ void contract_entry(const float2* __restrict__ V, int64_t ldv, int ka,
                                               int kz, int ma, int mz, const int32_t* rtri,
                                               const float2* rvec, const int32_t* ctri,
                                               const float2* cvec, float& acch, float& accl,
                                               int64_t t0 = 0, int64_t t1 = 0) {
  for (int k = ka; k < kz; ++k) {
    if (PANEL && (rtri[k] < t0 || rtri[k] >= t1)) continue;   // row of V not in this panel
    const float2* vrow = V + (int64_t)(rtri[k] - t0) * ldv;
    const float2 sk[3] = {rvec[3 * k], rvec[3 * k + 1], rvec[3 * k + 2]};
    int m = ma;
    for (; m + CT_BATCH <= mz; m += CT_BATCH) {
      float2 v[CT_BATCH];
#pragma unroll
      for (int u = 0; u < CT_BATCH; ++u) v[u] = vrow[ctri[m + u]];
#pragma unroll
      for (int u = 0; u < CT_BATCH; ++u) {
        float dh, dl;
        df_dot3(sk, cvec + 3 * (m + u), dh, dl);
        df_fma_acc(dh, dl, v[u].x, v[u].y, acch, accl);
      }
    }
    for (; m < mz; ++m) {
      const float2 v = vrow[ctri[m]];
      float dh, dl;
      df_dot3(sk, cvec + 3 * m, dh, dl);
      df_fma_acc(dh, dl, v.x, v.y, acch, accl);
    }
  }
}

__global__ void __launch_bounds__(256) contract_kernel(const float2* __restrict__ V, int64_t ldv,
                                                       const int64_t* __restrict__ jptr,
                                                       const int32_t* __restrict__ jtri,
                                                       const float2* __restrict__ jvec, int64_t N,
                                                       int nbt, float* __restrict__ Wh,
                                                       float* __restrict__ Wl, int64_t ldw) {
  __shared__ float2 s_out[CT][CT + 1];
  __shared__ int32_t s_rtri[CT_CAP], s_ctri[CT_CAP];
  __shared__ float2 s_rvec[3 * CT_CAP], s_cvec[3 * CT_CAP];
  __shared__ int32_t s_rptr[CT + 1], s_cptr[CT + 1];
  int bi, bj;
  tile_coords(blockIdx.x, nbt, bi, bj);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t r0 = (int64_t)bi * CT, c0 = (int64_t)bj * CT;
  const int64_t rl = (N - r0 < CT) ? N - r0 : CT, cl = (N - c0 < CT) ? N - c0 : CT;
  const int64_t rbase = jptr[r0], cbase = jptr[c0];
  const int64_t rcount = jptr[r0 + rl] - rbase, ccount = jptr[c0 + cl] - cbase;
  const bool staged = rcount <= CT_CAP && ccount <= CT_CAP;
  if (threadIdx.x <= CT) {
    const int i = threadIdx.x;
    s_rptr[i] = (int32_t)(jptr[r0 + (i < rl ? i : rl)] - rbase);
    s_cptr[i] = (int32_t)(jptr[c0 + (i < cl ? i : cl)] - cbase);
  }
  if (staged) {
    for (int64_t e = threadIdx.x; e < rcount; e += blockDim.x) {
      s_rtri[e] = jtri[rbase + e];
      s_rvec[3 * e] = jvec[3 * (rbase + e)];
      s_rvec[3 * e + 1] = jvec[3 * (rbase + e) + 1];
      s_rvec[3 * e + 2] = jvec[3 * (rbase + e) + 2];
    }
    for (int64_t e = threadIdx.x; e < ccount; e += blockDim.x) {
      s_ctri[e] = jtri[cbase + e];
      s_cvec[3 * e] = jvec[3 * (cbase + e)];
      s_cvec[3 * e + 1] = jvec[3 * (cbase + e) + 1];
      s_cvec[3 * e + 2] = jvec[3 * (cbase + e) + 2];
    }
  }
  __syncthreads();
  for (int rr = ty; rr < CT; rr += 8) {
    float acch = 0.f, accl = 0.f;
    if (rr < rl && tx < cl) {
      if (staged)
        contract_entry<true>(V, ldv, s_rptr[rr], s_rptr[rr + 1], s_cptr[tx], s_cptr[tx + 1], s_rtri,
                             s_rvec, s_ctri, s_cvec, acch, accl);
      else
        contract_entry<false>(V, ldv, s_rptr[rr], s_rptr[rr + 1], s_cptr[tx], s_cptr[tx + 1],
                              jtri + rbase, jvec + 3 * rbase, jtri + cbase, jvec + 3 * cbase, acch,
                              accl);
    }
    float h, l;
    two_sum(acch, accl, h, l);
    s_out[rr][tx] = make_float2(h, l);
  }
  __syncthreads();
  for (int rr = ty; rr < CT; rr += 8) {
    int64_t row = r0 + rr, c = c0 + tx;
    float2 v = (bi == bj && tx < rr) ? s_out[tx][rr] : s_out[rr][tx];
    if (row < N && c < N) {
      Wh[row * ldw + c] = v.x;
      Wl[row * ldw + c] = v.y;
    }
  }
  if (bi != bj) {
    for (int cc = ty; cc < CT; cc += 8) {
      int64_t R = c0 + cc, C = r0 + tx;
      if (R < N && C < N) {
        const float2 v = s_out[tx][cc];
        Wh[R * ldw + C] = v.x;
        Wl[R * ldw + C] = v.y;
      }
    }
  }
}

cudaError_t launch_contract(const DevGeom& g, cudaStream_t s) {
  int nbt = (int)((g.ndof + CT - 1) / CT);
  int64_t tiles = (int64_t)nbt * (nbt + 1) / 2;
  if (tiles == 0) return cudaSuccess;
  contract_kernel<<<(unsigned)tiles, 256, 0, s>>>(g.d_V, g.nt, g.d_jptr, g.d_jtri, g.d_jvecf, g.ndof,
                                                  nbt, g.d_Wh, g.wlo(), g.ldw);
  return cudaGetLastError();
}

// Panel mode: V holds the rows t0 .. t1-1 only.  W[nu, nu'] += the part of
// sum_{k in J(nu)} sum_{m in J(nu')} V[T_k, T_m] s_k . s_m with T_k in the
// panel, for the row tiles rt0 .. rt0+nrt-1 (the dofs the panel touches) and
// every column tile; W starts at zero and the panels add up (double-float).
__global__ void __launch_bounds__(256) contract_panel_kernel(const float2* __restrict__ V, int64_t ldv,
                                                             int64_t t0, int64_t t1,
                                                             const int64_t* __restrict__ jptr,
                                                             const int32_t* __restrict__ jtri,
                                                             const float2* __restrict__ jvec, int64_t N,
                                                             int nbt, int rt0, float* __restrict__ Wh,
                                                             float* __restrict__ Wl, int64_t ldw) {
  __shared__ int32_t s_rtri[CT_CAP], s_ctri[CT_CAP];
  __shared__ float2 s_rvec[3 * CT_CAP], s_cvec[3 * CT_CAP];
  __shared__ int32_t s_rptr[CT + 1], s_cptr[CT + 1];
  const int bi = rt0 + (int)(blockIdx.x / nbt), bj = (int)(blockIdx.x % nbt);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t r0 = (int64_t)bi * CT, c0 = (int64_t)bj * CT;
  const int64_t rl = (N - r0 < CT) ? N - r0 : CT, cl = (N - c0 < CT) ? N - c0 : CT;
  if (rl <= 0 || cl <= 0) return;
  const int64_t rbase = jptr[r0], cbase = jptr[c0];
  const int64_t rcount = jptr[r0 + rl] - rbase, ccount = jptr[c0 + cl] - cbase;
  const bool staged = rcount <= CT_CAP && ccount <= CT_CAP;
  if (threadIdx.x <= CT) {
    const int i = threadIdx.x;
    s_rptr[i] = (int32_t)(jptr[r0 + (i < rl ? i : rl)] - rbase);
    s_cptr[i] = (int32_t)(jptr[c0 + (i < cl ? i : cl)] - cbase);
  }
  if (staged) {
    for (int64_t e = threadIdx.x; e < rcount; e += blockDim.x) {
      s_rtri[e] = jtri[rbase + e];
      s_rvec[3 * e] = jvec[3 * (rbase + e)];
      s_rvec[3 * e + 1] = jvec[3 * (rbase + e) + 1];
      s_rvec[3 * e + 2] = jvec[3 * (rbase + e) + 2];
    }
    for (int64_t e = threadIdx.x; e < ccount; e += blockDim.x) {
      s_ctri[e] = jtri[cbase + e];
      s_cvec[3 * e] = jvec[3 * (cbase + e)];
      s_cvec[3 * e + 1] = jvec[3 * (cbase + e) + 1];
      s_cvec[3 * e + 2] = jvec[3 * (cbase + e) + 2];
    }
  }
  __syncthreads();
  for (int rr = ty; rr < CT; rr += 8) {
    if (rr >= rl || tx >= cl) continue;
    float acch = 0.f, accl = 0.f;
    if (staged)
      contract_entry<true, true>(V, ldv, s_rptr[rr], s_rptr[rr + 1], s_cptr[tx], s_cptr[tx + 1], s_rtri, s_rvec,
                                 s_ctri, s_cvec, acch, accl, t0, t1);
    else
      contract_entry<false, true>(V, ldv, s_rptr[rr], s_rptr[rr + 1], s_cptr[tx], s_cptr[tx + 1], jtri + rbase,
                                  jvec + 3 * rbase, jtri + cbase, jvec + 3 * cbase, acch, accl, t0, t1);
    if (acch == 0.f && accl == 0.f) continue;
    const int64_t o = (r0 + rr) * ldw + c0 + tx;
    float h, l;
    df_add(Wh[o], Wl[o], acch, accl, h, l);
    two_sum(h, l, h, l);
    Wh[o] = h;
    Wl[o] = l;
  }
}

cudaError_t launch_contract_panel(const DevGeom& g, int64_t t0, int64_t t1, int rt0, int nrt, cudaStream_t s) {
  const int nbt = (int)((g.ndof + CT - 1) / CT);
  const int64_t blocks = (int64_t)nrt * nbt;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  contract_panel_kernel<<<(unsigned)blocks, 256, 0, s>>>(g.d_V, g.nt, t0, t1, g.d_jptr, g.d_jtri, g.d_jvecf,
                                                         g.ndof, nbt, rt0, g.d_Wh, g.wlo(), g.ldw);
  return cudaGetLastError();
}

// rows row0 .. row0+nrows-1 of W as dense FP64 rows of length N
__global__ void w_to_double_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl,
                                   int64_t ldw, int64_t N, int64_t row0, int64_t nrows,
                                   double* __restrict__ out) {
  const int64_t n = nrows * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / N, c = i - r * N;
    const int64_t o = (row0 + r) * ldw + c;
    out[i] = df_to_double(Wh[o], Wl[o]);
  }
}

cudaError_t copy_rows_to_double(const DevGeom& g, int64_t row0, int64_t nrows, double* out,
                                cudaStream_t s) {
  const int64_t n = nrows * g.ndof;
  if (n == 0) return cudaSuccess;
  int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 64);
  w_to_double_kernel<<<(unsigned)blocks, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, g.ndof, row0, nrows, out);
  return cudaGetLastError();
}

// diag(W) in FP64
__global__ void diag_kernel(const float* __restrict__ Wh, const float* __restrict__ Wl, int64_t ldw, int64_t N,
                            double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = df_to_double(Wh[i * ldw + i], Wl[i * ldw + i]);
}

cudaError_t copy_diagonal(const DevGeom& g, double* out, cudaStream_t s) {
  if (g.ndof == 0) return cudaSuccess;
  diag_kernel<<<(unsigned)((g.ndof + 255) / 256), 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, g.ndof, out);
  return cudaGetLastError();
}

// W += rho Q Q^T for a screen with closed cells (Q: N x nc, an orthonormal
// basis of the cells' indicators); the correction is summed in FP64 and added
// to the float pair
__global__ void augment_kernel(float* __restrict__ Wh, float* __restrict__ Wl, int64_t ldw, int64_t N,
                               const double* __restrict__ Z, int nc, double rho) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e - (e / N) * N;
    double corr = 0.0;
    for (int k = 0; k < nc; ++k) corr = fma(Z[i * nc + k], Z[j * nc + k], corr);
    if (corr == 0.0) continue;
    const int64_t o = i * ldw + j;
    float h, l;
    split_df(df_to_double(Wh[o], Wl[o]) + rho * corr, h, l);
    Wh[o] = h;
    Wl[o] = l;
  }
}

cudaError_t launch_augment(const DevGeom& g, double rho, cudaStream_t s) {
  if (g.ndof == 0 || g.ncells == 0) return cudaSuccess;
  const int64_t n2 = g.ndof * g.ndof;
  const int64_t blocks = std::min<int64_t>((n2 + 255) / 256, 152 * 64);
  augment_kernel<<<(unsigned)blocks, 256, 0, s>>>(g.d_Wh, g.wlo(), g.ldw, g.ndof, g.d_cellZ, g.ncells, rho);
  return cudaGetLastError();
}

__global__ void rhs_kernel(const int64_t* __restrict__ jptr, const double* __restrict__ jrhs,
                           int64_t N, double gx, double gy, double gz, double* __restrict__ L) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc = 0.0;
  for (int64_t k = jptr[i]; k < jptr[i + 1]; ++k)
    acc += jrhs[3 * k] * gx + jrhs[3 * k + 1] * gy + jrhs[3 * k + 2] * gz;
  L[i] = acc;
}

cudaError_t launch_rhs(const DevGeom& g, const double gv[3], double* out, cudaStream_t s) {
  if (g.ndof == 0) return cudaSuccess;
  rhs_kernel<<<(unsigned)((g.ndof + 255) / 256), 256, 0, s>>>(g.d_jptr, g.d_jrhs, g.ndof, gv[0],
                                                               gv[1], gv[2], out);
  return cudaGetLastError();
}

}  // namespace msbem
