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
//   * r^2 with FMA-exact squares, 1/r from the FP32 reciprocal square root
//     followed by one second-order correction computed in double-float.
//
// Two evaluation paths, chosen per pair by the distance of the centroids:
//   * close pairs (|D| < 4 (rho_T + rho_T'), rho = largest point offset of a
//     triangle): d = (a_p + D) - b_q formed with error-free two-sums, weights
//     applied per evaluation; relative error a few 1e-15 of |V|;
//   * separated pairs (the rest, where every |d| >= 3|D|/4): every point
//     offset and D are re-split onto the pair's own power-of-two grid
//     g = 2^(e-23), 2^e > |D| + rho_T + rho_T', so that the hi parts are
//     multiples of g below 2^24 g and d_hi = (D_hi + a_hi) - b_hi is exact in
//     FP32; d_lo carries the rest with an absolute error of a few 2^-24 g,
//     i.e. a relative error in |d| below ~2^-43 (2^e <= 2.5 |D| <= 3.4 |d|).
//     The evaluations are summed unweighted per orbit class of the rule (the
//     two orbits of three points with weights w_a, w_b: classes aa, ab + ba,
//     bb) and weighted once per pair.
// The column triangles' data of a tile (offsets, centroids, areas, vertex ids)
// is staged into shared memory by bulk asynchronous copies (TMA) completing on
// an mbarrier; the wait is bounded and a copy that never lands sets the error
// flag instead of hanging.
#include "df.cuh"
#include "msbem_internal.h"

namespace msbem {

#define DF_TILE 64
__constant__ float c_wdf[12];   // rule weights as (hi, lo) pairs
__constant__ float c_wcls[6];   // class weights w_a^2, w_a w_b, w_b^2 as (hi, lo) pairs

// a + b as an unnormalised pair (s, e): s + e = a + b to ~2^-48 relative and
// |e| <= ulp(s) + |al + bl|; the consumers (df_rsqrt3, the next addition) only
// need the sum, not a canonical split, so the renormalisation is left out
__device__ __forceinline__ void df_add_raw(float ah, float al, float bh, float bl, float& s, float& e) {
  two_sum(ah, bh, s, e);
  e += al + bl;
}

// (h, l) re-split onto the grid g (a power of two, ig = 1/g): H a multiple of
// g, h - H exact (Sterbenz: H = 0, or H and h within a factor of two)
__device__ __forceinline__ void grid_split(float h, float l, float g, float ig, float& H, float& L) {
  H = rintf(h * ig) * g;
  L = (h - H) + l;
}

// acc += y for positive y and acc (Fast2Sum on the larger / smaller term)
__device__ __forceinline__ void pos_acc(float& acch, float& accl, float y) {
  const float s = acch + y;
  const float big = fmaxf(acch, y), small = fminf(acch, y);
  accl += small - (s - big);
  acch = s;
}

__device__ __forceinline__ uint32_t fd_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t fd_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for phase 0 of the barrier; false after ~2 s or 2^24 polls
__device__ __noinline__ bool fd_wait(uint64_t* bar) {
  const uint64_t t0 = fd_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0,1,0,p;\n}\n"
        : "=r"(ok) : "r"(fd_smem(bar)) : "memory");
    if (ok) return true;
    if (fd_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void fd_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(fd_smem(dst)), "l"(src), "r"(bytes), "r"(fd_smem(bar)) : "memory");
}

// One row point p of a separated pair: its six evaluations against the
// column points, summed unweighted into the accumulators of the classes
// (row orbit, column orbit a) and (row orbit, column orbit b).
__device__ __forceinline__ void far_row(float Uxh, float Uxl, float Uyh, float Uyl, float Uzh, float Uzl,
                                        const float* bq, float& ah, float& al, float& ac, float& bh, float& bl,
                                        float& bc) {
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float dxh = Uxh - bq[6 * q + 0], dxl = Uxl - bq[6 * q + 1];   // hi: exact on the pair's grid
    const float dyh = Uyh - bq[6 * q + 2], dyl = Uyl - bq[6 * q + 3];
    const float dzh = Uzh - bq[6 * q + 4], dzl = Uzl - bq[6 * q + 5];
    float y, corr;
    df_rsqrt3(dxh, dxl, dyh, dyl, dzh, dzl, y, corr);
    if (q < 3) {
      pos_acc(ah, al, y);
      ac += corr;
    } else {
      pos_acc(bh, bl, y);
      bc += corr;
    }
  }
}

// PANEL: rows of tiles tb0 .. (V holds triangle rows tb0*64 ..), every column
// tile, no mirrored write; otherwise the upper triangle of tiles, mirrored.
template <bool PANEL>
__global__ void __launch_bounds__(256, 3) far_df_kernel(const double* __restrict__ cen,
                                                     const float* __restrict__ qoff,
                                                     const double* __restrict__ area,
                                                     const float2* __restrict__ cendf,
                                                     const float2* __restrict__ areadf,
                                                     const int32_t* __restrict__ tri, int nb,
                                                     int64_t nt, int64_t ldv,
                                                     float2* __restrict__ V, int tb0, int* __restrict__ err) {
  __shared__ __align__(128) float s_off[DF_TILE * 36];
  __shared__ __align__(16) double s_cen[DF_TILE * 3];
  __shared__ __align__(16) double s_area[DF_TILE];
  __shared__ __align__(16) int32_t s_tri[DF_TILE * 3];
  __shared__ __align__(16) float2 s_cdf[DF_TILE * 3];
  __shared__ __align__(16) float2 s_adf[DF_TILE];
  __shared__ float s_rho[DF_TILE];
  __shared__ float2 s_out[DF_TILE][DF_TILE + 1];
  __shared__ __align__(8) uint64_t s_bar;
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
  constexpr uint32_t B_OFF = DF_TILE * 36 * 4, B_CEN = DF_TILE * 3 * 8, B_AREA = DF_TILE * 8,
                     B_TRI = DF_TILE * 3 * 4, B_CDF = DF_TILE * 3 * 8, B_ADF = DF_TILE * 8;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fd_smem(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    // the column tile: offsets, centroids, areas and vertex ids (arrays padded
    // to whole tiles; every source offset is a multiple of 256 bytes)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fd_smem(&s_bar)),
                 "r"(B_OFF + B_CEN + B_AREA + B_TRI + B_CDF + B_ADF) : "memory");
    fd_bulk(s_off, qoff + col0 * 36, B_OFF, &s_bar);
    fd_bulk(s_cen, cen + col0 * 3, B_CEN, &s_bar);
    fd_bulk(s_area, area + col0, B_AREA, &s_bar);
    fd_bulk(s_tri, tri + col0 * 3, B_TRI, &s_bar);
    fd_bulk(s_cdf, cendf + col0 * 3, B_CDF, &s_bar);
    fd_bulk(s_adf, areadf + col0, B_ADF, &s_bar);
  }
  // the row triangle of this thread, from global memory meanwhile
  const int r = tid & 63;
  const int cgrp = tid >> 6;
  const int64_t T = row0 + r;
  float a[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) a[k] = qoff[T * 36 + k];
  const double cx = cen[T * 3], cy = cen[T * 3 + 1], cz = cen[T * 3 + 2];
  const double aT = area[T];
  const float2 cTx = cendf[T * 3], cTy = cendf[T * 3 + 1], cTz = cendf[T * 3 + 2];
  const float2 aTdf = areadf[T];
  const int32_t t0 = tri[T * 3], t1 = tri[T * 3 + 1], t2 = tri[T * 3 + 2];
  float rhoT = 0.f;
#pragma unroll
  for (int p = 0; p < 6; ++p)
    rhoT = fmaxf(rhoT, sqrtf(fmaf(a[6 * p], a[6 * p], fmaf(a[6 * p + 2], a[6 * p + 2], a[6 * p + 4] * a[6 * p + 4]))));
  rhoT *= 1.0001f;
  const bool landed = fd_wait(&s_bar);
  if (__syncthreads_or(!landed)) {
    // a copy never completed: let the copies land (bounded) before the shared
    // memory is given back, report, and write nothing
    if (tid == 0) {
      fd_wait(&s_bar);
      atomicExch(err, 1);
    }
    return;
  }
  if (tid < DF_TILE) {
    float m = 0.f;
    const float* b = &s_off[tid * 36];
#pragma unroll
    for (int p = 0; p < 6; ++p)
      m = fmaxf(m, sqrtf(fmaf(b[6 * p], b[6 * p], fmaf(b[6 * p + 2], b[6 * p + 2], b[6 * p + 4] * b[6 * p + 4]))));
    s_rho[tid] = m * 1.0001f;
  }
  __syncthreads();
  for (int cc = 0; cc < 16; ++cc) {
    const int c = cgrp * 16 + cc;
    const int32_t u0 = s_tri[3 * c], u1 = s_tri[3 * c + 1], u2 = s_tri[3 * c + 2];
    const bool touch = (t0 == u0) | (t0 == u1) | (t0 == u2) | (t1 == u0) | (t1 == u1) |
                       (t1 == u2) | (t2 == u0) | (t2 == u1) | (t2 == u2) | (t0 < 0) | (u0 < 0);
    float2 v = make_float2(0.f, 0.f);
    if (!touch) {
      // D = c_T - c_T' from the float-pair centroids (absolute error ~2^-48 of
      // the coordinates; the close pairs below take it from the FP64 ones)
      float Dxh, Dxl, Dyh, Dyl, Dzh, Dzl;
      df_add_raw(cTx.x, cTx.y, -s_cdf[3 * c].x, -s_cdf[3 * c].y, Dxh, Dxl);
      df_add_raw(cTy.x, cTy.y, -s_cdf[3 * c + 1].x, -s_cdf[3 * c + 1].y, Dyh, Dyl);
      df_add_raw(cTz.x, cTz.y, -s_cdf[3 * c + 2].x, -s_cdf[3 * c + 2].y, Dzh, Dzl);
      const float* b = &s_off[c * 36];
      float bq[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) bq[k] = b[k];
      const float rsum = rhoT + s_rho[c];
      const float m2 = fmaf(Dxh, Dxh, fmaf(Dyh, Dyh, Dzh * Dzh));
      float acch = 0.0f, accl = 0.0f;
      if (m2 >= 16.0f * rsum * rsum) {
        // separated: the pair's grid g = 2^(k-23) with 2^k > |D| + rho_T + rho_T'
        const float bound = fmaf(sqrtf(m2), 1.0001f, rsum);
        const int k = (int)((__float_as_uint(bound) >> 23) & 0xff) - 126;
        const float g = __uint_as_float((uint32_t)(k - 23 + 127) << 23);
        const float ig = __uint_as_float((uint32_t)(23 - k + 127) << 23);
        float DHx, DLx, DHy, DLy, DHz, DLz;
        grid_split(Dxh, Dxl, g, ig, DHx, DLx);
        grid_split(Dyh, Dyl, g, ig, DHy, DLy);
        grid_split(Dzh, Dzl, g, ig, DHz, DLz);
#pragma unroll
        for (int q = 0; q < 18; ++q) {
          float H, L;
          grid_split(bq[2 * q], bq[2 * q + 1], g, ig, H, L);
          bq[2 * q] = H;
          bq[2 * q + 1] = L;
        }
        // class sums (hi, lo, FP32 sum of the corrections): aa, ab + ba, bb
        float sah = 0.f, sal = 0.f, sac = 0.f, smh = 0.f, sml = 0.f, smc = 0.f, sbh = 0.f, sbl = 0.f,
              sbc = 0.f;
#pragma unroll 1
        for (int p = 0; p < 3; ++p) {   // row orbit a
          float AHx, ALx, AHy, ALy, AHz, ALz;
          grid_split(a[6 * p + 0], a[6 * p + 1], g, ig, AHx, ALx);
          grid_split(a[6 * p + 2], a[6 * p + 3], g, ig, AHy, ALy);
          grid_split(a[6 * p + 4], a[6 * p + 5], g, ig, AHz, ALz);
          far_row(DHx + AHx, DLx + ALx, DHy + AHy, DLy + ALy, DHz + AHz, DLz + ALz, bq, sah, sal, sac, smh, sml,
                  smc);
        }
#pragma unroll 1
        for (int p = 3; p < 6; ++p) {   // row orbit b
          float AHx, ALx, AHy, ALy, AHz, ALz;
          grid_split(a[6 * p + 0], a[6 * p + 1], g, ig, AHx, ALx);
          grid_split(a[6 * p + 2], a[6 * p + 3], g, ig, AHy, ALy);
          grid_split(a[6 * p + 4], a[6 * p + 5], g, ig, AHz, ALz);
          far_row(DHx + AHx, DLx + ALx, DHy + AHy, DLy + ALy, DHz + AHz, DLz + ALz, bq, smh, sml, smc, sbh, sbl,
                  sbc);
        }
        // weighted once: w_a^2 S_aa + w_a w_b S_ab + w_b^2 S_bb (double-float)
        df_fma_acc(c_wcls[0], c_wcls[1], sah, sal + sac, acch, accl);
        df_fma_acc(c_wcls[2], c_wcls[3], smh, sml + smc, acch, accl);
        df_fma_acc(c_wcls[4], c_wcls[5], sbh, sbl + sbc, acch, accl);
        // V = S |T| |T'| / (4 pi) in double-float
        constexpr double kq = 0.25 / M_PI;
        constexpr float kqh = (float)kq;
        constexpr float kql = (float)(kq - (double)kqh);
        float sh, sl, vh, vl;
        df_mul(aTdf.x, aTdf.y, s_adf[c].x, s_adf[c].y, sh, sl);
        df_mul(sh, sl, kqh, kql, sh, sl);
        df_mul(acch, accl, sh, sl, vh, vl);
        v = make_float2(vh, vl);
      } else {
        // close: D from the FP64 centroids (exact to 2^-53 |D|), exact
        // differences, weights per evaluation
        split_df(cx - s_cen[3 * c], Dxh, Dxl);
        split_df(cy - s_cen[3 * c + 1], Dyh, Dyl);
        split_df(cz - s_cen[3 * c + 2], Dzh, Dzl);
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
  cudaError_t e = cudaMemcpyToSymbol(c_wdf, h, sizeof(h));
  if (e != cudaSuccess) return e;
  // class weights (the rule's two orbits: points 0-2 weight w[0], 3-5 weight w[3])
  const double cls[3] = {w[0] * w[0], w[0] * w[3], w[3] * w[3]};
  float k[6];
  for (int i = 0; i < 3; ++i) {
    float hi = (float)cls[i];
    k[2 * i] = hi;
    k[2 * i + 1] = (float)(cls[i] - (double)hi);
  }
  return cudaMemcpyToSymbol(c_wcls, k, sizeof(k));
}

cudaError_t launch_far_df(const DevGeom& g, int* err, cudaStream_t s) {
  int nb = (int)(g.nt_pad / DF_TILE);
  int64_t tiles = (int64_t)nb * (nb + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  far_df_kernel<false><<<(unsigned)tiles, 256, 0, s>>>(g.d_cen, g.d_qoff, g.d_area, g.d_cendf, g.d_areadf,
                                                       g.d_tri, nb, g.nt, g.nt, g.d_V, 0, err);
  return cudaGetLastError();
}

// rows [tb0*64, (tb0+ntb)*64) of V into a panel buffer of ntb*64 rows
cudaError_t launch_far_df_panel(const DevGeom& g, int tb0, int ntb, int* err, cudaStream_t s) {
  int nb = (int)(g.nt_pad / DF_TILE);
  int64_t tiles = (int64_t)ntb * nb;
  if (tiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  far_df_kernel<true><<<(unsigned)tiles, 256, 0, s>>>(g.d_cen, g.d_qoff, g.d_area, g.d_cendf, g.d_areadf,
                                                      g.d_tri, nb, g.nt, g.nt, g.d_V, tb0, err);
  return cudaGetLastError();
}

}  // namespace msbem
