// rbc_stencil.cuh -- the leapfrog update of Eq. 1 for four consecutive nodes,
// in packed fp32x2 arithmetic (sm_100 family FADD2/FMUL2/FFMA2: two lanes of
// fp32 per instruction, each correctly rounded, so the results equal those of
// the scalar sequence).
//
//   out = (2 p - p_old) + a * sum_k c_k s_k,
//   s_k = sum over the axes of [(p_{-k} - p) + (p_{+k} - p)]   (k = 1..4)
//
// The weights c1..c4 are those of rbc_internal.cuh; summing differences from
// the centre makes the fp32 rounding relative to the second differences
// instead of |p|, because c0 = -2 (c1 + c2 + c3 + c4) cancels exactly.
#pragma once

#include "rbc_internal.cuh"

namespace rbc {

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 half2of(const float4 &v, int j) { return j ? hi2(v) : lo2(v); }
__device__ __forceinline__ float2 neg2(const float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 sum_diff2(const float2 m, const float2 p, const float2 np) {
  return __fadd2_rn(__fadd2_rn(m, np), __fadd2_rn(p, np));
}

// w[0..11]: x window x0-4 .. x0+7 (centre at w[4..7]); zq[0..8]: z window
// (zq[4] = centre); ym[k-1] / yp[k-1]: y neighbours at distance k (3-D only).
template <bool kThreeD>
__device__ __forceinline__ float4 leap4p(const float *w, const float4 *zq, const float4 *ym, const float4 *yp,
                                         const float4 po, const float4 av) {
  float2 out[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 p = make_float2(w[4 + 2 * j], w[5 + 2 * j]);
    const float2 np = neg2(p);
    float2 s[5];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
      const float2 xm = make_float2(w[4 + 2 * j - k], w[5 + 2 * j - k]);
      const float2 xp = make_float2(w[4 + 2 * j + k], w[5 + 2 * j + k]);
      float2 t = sum_diff2(xm, xp, np);
      t = __fadd2_rn(t, sum_diff2(half2of(zq[4 - k], j), half2of(zq[4 + k], j), np));
      if (kThreeD) t = __fadd2_rn(t, sum_diff2(half2of(ym[k - 1], j), half2of(yp[k - 1], j), np));
      s[k] = t;
    }
    float2 lap = __fmul2_rn(make_float2(kC4, kC4), s[4]);
    lap = __ffma2_rn(make_float2(kC3, kC3), s[3], lap);
    lap = __ffma2_rn(make_float2(kC2, kC2), s[2], lap);
    lap = __ffma2_rn(make_float2(kC1, kC1), s[1], lap);
    const float2 base = __fadd2_rn(__fadd2_rn(p, p), neg2(half2of(po, j)));
    out[j] = __ffma2_rn(half2of(av, j), lap, base);
  }
  return make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
}

// Same update split as out = base + inc, inc = a * lap (the discrete second
// time difference p^{n+1} - 2 p^n + p^{n-1} without the point terms), for
// callers that need the increment itself (the FWI gradient).
__device__ __forceinline__ float4 leap4p_inc(const float *w, const float4 *zq, const float4 po, const float4 av,
                                             float4 *inc) {
  float2 out[2], dd[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 p = make_float2(w[4 + 2 * j], w[5 + 2 * j]);
    const float2 np = neg2(p);
    float2 s[5];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
      const float2 xm = make_float2(w[4 + 2 * j - k], w[5 + 2 * j - k]);
      const float2 xp = make_float2(w[4 + 2 * j + k], w[5 + 2 * j + k]);
      float2 t = sum_diff2(xm, xp, np);
      t = __fadd2_rn(t, sum_diff2(half2of(zq[4 - k], j), half2of(zq[4 + k], j), np));
      s[k] = t;
    }
    float2 lap = __fmul2_rn(make_float2(kC4, kC4), s[4]);
    lap = __ffma2_rn(make_float2(kC3, kC3), s[3], lap);
    lap = __ffma2_rn(make_float2(kC2, kC2), s[2], lap);
    lap = __ffma2_rn(make_float2(kC1, kC1), s[1], lap);
    const float2 base = __fadd2_rn(__fadd2_rn(p, p), neg2(half2of(po, j)));
    dd[j] = __fmul2_rn(half2of(av, j), lap);
    out[j] = __fadd2_rn(base, dd[j]);
  }
  *inc = make_float4(dd[0].x, dd[0].y, dd[1].x, dd[1].y);
  return make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
}

} // namespace rbc
