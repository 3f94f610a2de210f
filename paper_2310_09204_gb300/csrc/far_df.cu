// Far-field pair integrals  V_{TT'} = |T||T'|/(4 pi) sum_p w_p sum_q w_q / |x_p - y_q|
// (6-point degree-4 rule on each triangle, pairs sharing no vertex) in
// double-float arithmetic on the FP32 pipe.
//
// GB300 executes FP64 FMAs at about 1/70 of its FP32 rate, so this kernel keeps
// FP64 out of the 36-evaluation inner loop:
//   * each quadrature point is stored as centroid (FP64) + offset a_p = x_p - c
//     held as an unevaluated float pair (hi + lo, 48-bit significand); the
//     offsets are small (|a_p| < h), so their absolute error is ~2^-49 h;
//   * per pair the centroid difference D = c_T - c_T' is formed once in FP64
//     (exact to 2^-53 |D|) and split into a float pair by integer bit
//     operations, so no FP64<->FP32 conversion instruction is issued;
//   * per evaluation d = (a_p + D) - b_q is formed with error-free two-sums
//     (kept as unnormalised pairs),
//     r^2 with FMA-exact squares, 1/r from the FP32 reciprocal square root
//     followed by one second-order correction computed in double-float, and
//     the weighted sums are accumulated as float pairs.
// Relative error per pair is a few 1e-15 of |V|, far below the 1e-12 parity
// bar against the FP64 oracle.
#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define DF_TILE 64
__constant__ float c_wdf[12];   // rule weights as (hi, lo) pairs

// a + b as an unnormalised pair (s, e): s + e = a + b to ~2^-48 relative and
// |e| <= ulp(s) + |al + bl|; the consumers (df_rsqrt3, the next addition) only
// need the sum, not a canonical split, so the renormalisation is left out
__device__ __forceinline__ void df_add_raw(float ah, float al, float bh, float bl, float& s, float& e) {
  two_sum(ah, bh, s, e);
  e += al + bl;
}

// PANEL: rows of tiles tb0 .. (V holds triangle rows tb0*64 ..), every column
// tile, no mirrored write; otherwise the upper triangle of tiles, mirrored.
template <bool PANEL>
__global__ void __launch_bounds__(256) far_df_kernel(const double* __restrict__ cen,
                                                     const float* __restrict__ qoff,
                                                     const double* __restrict__ area,
                                                     const int32_t* __restrict__ tri, int nb,
                                                     int64_t nt, int64_t ldv,
                                                     float2* __restrict__ V, int tb0) {
  __shared__ float s_off[DF_TILE * 36];
  __shared__ double s_cen[DF_TILE * 3];
  __shared__ double s_area[DF_TILE];
  __shared__ int32_t s_tri[DF_TILE * 3];
  __shared__ float2 s_out[DF_TILE][DF_TILE + 1];
  // upper-triangle tile coordinates
  int bi, bj;
  if (PANEL) {
    bi = tb0 + (int)(blockIdx.x / nb);
    bj = (int)(blockIdx.x % nb);
  } else {
    const int64_t t = blockIdx.x;
    double disc = (2.0 * nb + 1.0) * (2.0 * nb + 1.0) - 8.0 * (double)t;
    int r = (int)floor(((2.0 * nb + 1.0) - sqrt(disc)) * 0.5);
    if (r < 0) r = 0;
    auto start = [nb](int64_t row) { return row * (int64_t)nb - row * (row - 1) / 2; };
    while (r > 0 && start(r) > t) --r;
    while (r + 1 < nb && start(r + 1) <= t) ++r;
    bi = r;
    bj = (int)(r + (t - start(r)));
  }
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)bi * DF_TILE, col0 = (int64_t)bj * DF_TILE;
  for (int i = tid; i < DF_TILE * 36; i += blockDim.x) s_off[i] = qoff[col0 * 36 + i];
  for (int i = tid; i < DF_TILE * 3; i += blockDim.x) {
    s_cen[i] = cen[col0 * 3 + i];
    s_tri[i] = tri[col0 * 3 + i];
  }
  for (int i = tid; i < DF_TILE; i += blockDim.x) s_area[i] = area[col0 + i];
  const int r = tid & 63;
  const int cgrp = tid >> 6;
  const int64_t T = row0 + r;
  float a[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) a[k] = qoff[T * 36 + k];
  const double cx = cen[T * 3], cy = cen[T * 3 + 1], cz = cen[T * 3 + 2];
  const double aT = area[T];
  const int32_t t0 = tri[T * 3], t1 = tri[T * 3 + 1], t2 = tri[T * 3 + 2];
  __syncthreads();
  for (int cc = 0; cc < 16; ++cc) {
    const int c = cgrp * 16 + cc;
    const int32_t u0 = s_tri[3 * c], u1 = s_tri[3 * c + 1], u2 = s_tri[3 * c + 2];
    const bool touch = (t0 == u0) | (t0 == u1) | (t0 == u2) | (t1 == u0) | (t1 == u1) |
                       (t1 == u2) | (t2 == u0) | (t2 == u1) | (t2 == u2) | (t0 < 0) | (u0 < 0);
    float2 v = make_float2(0.f, 0.f);
    if (!touch) {
      float Dxh, Dxl, Dyh, Dyl, Dzh, Dzl;
      split_df(cx - s_cen[3 * c], Dxh, Dxl);
      split_df(cy - s_cen[3 * c + 1], Dyh, Dyl);
      split_df(cz - s_cen[3 * c + 2], Dzh, Dzl);
      const float* b = &s_off[c * 36];
      float bq[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) bq[k] = b[k];
      float acch = 0.0f, accl = 0.0f;
#pragma unroll 1
      for (int p = 0; p < 6; ++p) {
        float uxh, uxl, uyh, uyl, uzh, uzl;   // u = a_p + D
        df_add_raw(a[6 * p + 0], a[6 * p + 1], Dxh, Dxl, uxh, uxl);
        df_add_raw(a[6 * p + 2], a[6 * p + 3], Dyh, Dyl, uyh, uyl);
        df_add_raw(a[6 * p + 4], a[6 * p + 5], Dzh, Dzl, uzh, uzl);
        float ih = 0.0f, il = 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          float dxh, dxl, dyh, dyl, dzh, dzl;  // d = u - b_q
          df_add_raw(uxh, uxl, -bq[6 * q + 0], -bq[6 * q + 1], dxh, dxl);
          df_add_raw(uyh, uyl, -bq[6 * q + 2], -bq[6 * q + 3], dyh, dyl);
          df_add_raw(uzh, uzl, -bq[6 * q + 4], -bq[6 * q + 5], dzh, dzl);
          float y, corr;
          df_rsqrt3(dxh, dxl, dyh, dyl, dzh, dzl, y, corr);
          // inner += w_q * (y + corr)
          const float wh = c_wdf[2 * q], wl = c_wdf[2 * q + 1];
          float ph = wh * y;
          float pe = fmaf(wh, y, -ph);
          pe = fmaf(wh, corr, pe);
          pe = fmaf(wl, y, pe);
          float s, e;
          two_sum(ih, ph, s, e);
          ih = s;
          il += e + pe;
        }
        // outer += w_p * inner
        const float wh = c_wdf[2 * p], wl = c_wdf[2 * p + 1];
        float ph = wh * ih;
        float pe = fmaf(wh, ih, -ph);
        pe = fmaf(wh, il, pe);
        pe = fmaf(wl, ih, pe);
        float s, e;
        two_sum(acch, ph, s, e);
        acch = s;
        accl += e + pe;
      }
      float vh, vl;
      split_df((widen(acch) + widen(accl)) * (aT * s_area[c]) * (0.25 / M_PI), vh, vl);
      v = make_float2(vh, vl);
    }
    s_out[r][c] = v;
  }
  __syncthreads();
  for (int i = tid; i < DF_TILE * DF_TILE; i += blockDim.x) {
    int rr = i / DF_TILE, c = i % DF_TILE;
    int64_t R = row0 + rr, C = col0 + c;
    if (R < nt && C < nt) V[(R - (int64_t)tb0 * DF_TILE) * ldv + C] = s_out[rr][c];
  }
  if (!PANEL && bi != bj) {
    for (int i = tid; i < DF_TILE * DF_TILE; i += blockDim.x) {
      int c = i / DF_TILE, rr = i % DF_TILE;
      int64_t R = row0 + rr, C = col0 + c;
      if (R < nt && C < nt) V[C * ldv + R] = s_out[rr][c];
    }
  }
}

cudaError_t set_far_df_constants(const double w[6]) {
  float h[12];
  for (int q = 0; q < 6; ++q) {
    float hi = (float)w[q];
    h[2 * q] = hi;
    h[2 * q + 1] = (float)(w[q] - (double)hi);
  }
  return cudaMemcpyToSymbol(c_wdf, h, sizeof(h));
}

cudaError_t launch_far_df(const DevGeom& g, cudaStream_t s) {
  int nb = (int)(g.nt_pad / DF_TILE);
  int64_t tiles = (int64_t)nb * (nb + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  far_df_kernel<false><<<(unsigned)tiles, 256, 0, s>>>(g.d_cen, g.d_qoff, g.d_area, g.d_tri, nb, g.nt, g.nt,
                                                       g.d_V, 0);
  return cudaGetLastError();
}

// rows [tb0*64, (tb0+ntb)*64) of V into a panel buffer of ntb*64 rows
cudaError_t launch_far_df_panel(const DevGeom& g, int tb0, int ntb, cudaStream_t s) {
  int nb = (int)(g.nt_pad / DF_TILE);
  int64_t tiles = (int64_t)ntb * nb;
  if (tiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  far_df_kernel<true><<<(unsigned)tiles, 256, 0, s>>>(g.d_cen, g.d_qoff, g.d_area, g.d_tri, nb, g.nt, g.nt,
                                                      g.d_V, tb0);
  return cudaGetLastError();
}

}  // namespace msbem
