// Double-float ("df") helpers: a value is the unevaluated sum hi + lo of two
// floats (48-bit significand).  GB300 runs FP32 FMAs about 70x faster than
// FP64 FMAs, so the hot loops that need FP64-level accuracy use these.
// Error-free transformations: Knuth's two-sum and the FMA exact product.
#pragma once

#include <cuda_runtime.h>

namespace msbem {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Float nearest to x (ties away from zero), by integer operations only:
// adding half of the 29 dropped significand bits to the bit pattern rounds,
// and a carry into the exponent is exactly the round-up across a binade.
// Magnitudes below the normal float range give 0.
__device__ __forceinline__ float round_to_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) + (1ull << 28);
  const unsigned sign = (unsigned)(b >> 63);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  const unsigned mant = (unsigned)((b >> 29) & 0x7fffff);
  const unsigned bits = (ex > 0 && ex < 255) ? ((sign << 31) | ((unsigned)ex << 23) | mant) : (sign << 31);
  return __uint_as_float(bits);
}

// Exact widening of a (normal or zero) float to double by integer operations.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const int ex = (int)((u >> 23) & 0xff);
  const unsigned long long mant = (unsigned long long)(u & 0x7fffff) << 29;
  const unsigned long long bits =
      ex ? (sign | ((unsigned long long)(ex - 127 + 1023) << 52) | mant) : sign;
  return __longlong_as_double((long long)bits);
}

// x -> hi + lo with |x - hi - lo| <= 2^-49 |x| (one FP64 add; x - hi is exact)
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = round_to_float(x);
  lo = round_to_float(x - widen(hi));
}

__device__ __forceinline__ double df_to_double(float hi, float lo) { return widen(hi) + widen(lo); }

// (rh, rl) = a + b, normalised
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  rh = s + e;
  rl = e - (rh - s);
}

// acc += a * b   (acc kept as an unnormalised pair; 13 FP32 ops)
__device__ __forceinline__ void df_fma_acc(float ah, float al, float bh, float bl, float& acch,
                                           float& accl) {
  float ph = ah * bh;
  float pe = fmaf(ah, bh, -ph);
  pe = fmaf(al, bl, pe);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  float s, e;
  two_sum(acch, ph, s, e);
  acch = s;
  accl += e + pe;
}

// dot product of two double-float 3-vectors, as an unnormalised pair
// (lo*lo terms, below 2^-48 relative, are dropped; 28 FP32 ops)
__device__ __forceinline__ void df_dot3(const float2* a, const float2* b, float& dh, float& dl) {
  const float p0 = a[0].x * b[0].x, p1 = a[1].x * b[1].x, p2 = a[2].x * b[2].x;
  const float e0 = fmaf(a[0].x, b[0].x, -p0), e1 = fmaf(a[1].x, b[1].x, -p1),
              e2 = fmaf(a[2].x, b[2].x, -p2);
  float s, t1, t2;
  two_sum(p0, p1, s, t1);
  two_sum(s, p2, s, t2);
  float err = ((e0 + e1) + (e2 + t1)) + t2;
  err = fmaf(a[0].x, b[0].y, err);
  err = fmaf(a[0].y, b[0].x, err);
  err = fmaf(a[1].x, b[1].y, err);
  err = fmaf(a[1].y, b[1].x, err);
  err = fmaf(a[2].x, b[2].y, err);
  err = fmaf(a[2].y, b[2].x, err);
  dh = s;
  dl = err;
}

// inverse distance of the double-float vector d: returns (y, corr) with
// 1/|d| = y + corr to ~2^-46 relative
__device__ __forceinline__ void df_rsqrt3(float dxh, float dxl, float dyh, float dyl, float dzh,
                                          float dzl, float& y, float& corr) {
  // r^2 = sum dh^2 + 2 dh dl (+ dl^2, below 2^-48 relative)
  float px = dxh * dxh, py = dyh * dyh, pz = dzh * dzh;
  float ex = fmaf(dxh, dxh, -px), ey = fmaf(dyh, dyh, -py), ez = fmaf(dzh, dzh, -pz);
  float s, e1, e2;
  two_sum(px, py, s, e1);
  two_sum(s, pz, s, e2);
  float cr = dxh * dxl;
  cr = fmaf(dyh, dyl, cr);
  cr = fmaf(dzh, dzl, cr);
  float low = fmaf(2.0f, cr, ((e1 + e2) + (ex + ey)) + ez);
  // y0 ~ 1/sqrt(s); e = 1 - r^2 y0^2 evaluated in double-float
  float y0 = rsqrtf(s);
  float y2h = y0 * y0;
  float y2l = fmaf(y0, y0, -y2h);
  float th = s * y2h;
  float tl = fmaf(s, y2h, -th);
  tl = fmaf(s, y2l, tl);
  tl = fmaf(low, y2h, tl);
  float ee = (1.0f - th) - tl;
  // 1/sqrt(r^2) = y0 (1 - ee)^(-1/2) = y0 (1 + ee/2 + 3 ee^2/8 + ...)
  y = y0;
  corr = y0 * ee * fmaf(0.375f, ee, 0.5f);
}

// (rh, rl) = a * b  (exact product of the high parts plus cross terms)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
  const float ph = ah * bh;
  float pe = fmaf(ah, bh, -ph);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  rh = ph + pe;
  rl = pe - (rh - ph);
}

// Warp reduction of LEN sums per lane at once ("transposed" butterfly): at the
// step of lane mask m, the lanes with that bit set keep the upper half of their
// values and the others the lower half, each adding its partner's half, so
// LEN values cost LEN - 1 shuffles instead of 5 LEN.  Every value is summed
// over the same lane pairing as a plain xor butterfly, so the result of a sum
// does not depend on how many others are reduced with it.  On return (LEN = V
// at the start) lane L holds the sums of indices L * V/32 + j when V >= 32,
// else index L >> log2(32/V).
template <int LEN, int MASK, bool DF>
__device__ __forceinline__ void warp_xreduce(float* h, float* l, int lane) {
  if constexpr (MASK > 0) {
    if constexpr (LEN >= 2) {
      constexpr int HALF = LEN / 2;
      const bool up = (lane & MASK) != 0;
#pragma unroll
      for (int i = 0; i < HALF; ++i) {
        const float sh = up ? h[i] : h[HALF + i];
        const float kh = up ? h[HALF + i] : h[i];
        const float rh = __shfl_xor_sync(0xffffffffu, sh, MASK);
        if constexpr (DF) {
          const float sl = up ? l[i] : l[HALF + i];
          const float kl = up ? l[HALF + i] : l[i];
          const float rl = __shfl_xor_sync(0xffffffffu, sl, MASK);
          float s, e;
          two_sum(kh, rh, s, e);
          h[i] = s;
          l[i] = (kl + rl) + e;
        } else {
          h[i] = kh + rh;
        }
      }
      warp_xreduce<HALF, MASK / 2, DF>(h, l, lane);
    } else {
      const float rh = __shfl_xor_sync(0xffffffffu, h[0], MASK);
      if constexpr (DF) {
        const float rl = __shfl_xor_sync(0xffffffffu, l[0], MASK);
        float s, e;
        two_sum(h[0], rh, s, e);
        h[0] = s;
        l[0] = (l[0] + rl) + e;
      } else {
        h[0] += rh;
      }
      warp_xreduce<1, MASK / 2, DF>(h, l, lane);
    }
  }
}

}  // namespace msbem
