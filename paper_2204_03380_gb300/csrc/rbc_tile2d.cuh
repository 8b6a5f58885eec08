// rbc_tile2d.cuh -- per-warp device code of the 2-D stencil kernels, shared by
// the single-shot kernels (rbc_kernels.cu) and the batched multi-shot kernels
// (rbc_batch.cu).  A lane owns a float4 of x; a warp marches RZ rows of a
// 128-column tile with an (RZ + 8)-deep register queue; x neighbours come from
// the adjacent lanes by shuffles (lanes 0/31 load the 4-float halo).
#pragma once

#include "rbc_internal.cuh"
#include "rbc_stencil.cuh"

namespace rbc {

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float cmp(const float4 &v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 shfl_up4(float4 v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_up_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_up_sync(0xffffffffu, v.w, 1);
  return v;
}
__device__ __forceinline__ float4 shfl_dn4(float4 v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  v.z = __shfl_down_sync(0xffffffffu, v.z, 1);
  v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
  return v;
}

// Leapfrog update of 4 consecutive nodes from the x window (lf, c, rt) and
// the z window zq[0..8] (zq[4] == c); see rbc_stencil.cuh.
__device__ __forceinline__ float4 leap4_2d(const float4 lf, const float4 c, const float4 rt, const float4 *zq,
                                           const float4 po, const float4 av) {
  const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w, rt.x, rt.y, rt.z, rt.w};
  return leap4p<false>(w, zq, nullptr, nullptr, po, av);
}

// Subtract a point term from component (src - o) of v when the source node
// falls in the float4 starting at offset o.
__device__ __forceinline__ void point_sub(float4 &v, int d, float term) {
  if (d == 0) v.x -= term;
  else if (d == 1) v.y -= term;
  else if (d == 2) v.z -= term;
  else if (d == 3) v.w -= term;
}

__device__ __forceinline__ float4 masked_prod(const float4 u, const float4 v, int x0, int lo, int hi) {
  float4 r;
  r.x = (x0 + 0 >= lo && x0 + 0 < hi) ? u.x * v.x : 0.f;
  r.y = (x0 + 1 >= lo && x0 + 1 < hi) ? u.y * v.y : 0.f;
  r.z = (x0 + 2 >= lo && x0 + 2 < hi) ? u.z * v.z : 0.f;
  r.w = (x0 + 3 >= lo && x0 + 3 < hi) ? u.w * v.w : 0.f;
  return r;
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Forward leapfrog (Eq. 1) of RZ rows starting at zb for the float4 at x0;
// the point source is subtracted where it falls.
template <int RZ>
__device__ __forceinline__ void fwd2d_rows(const Lay &L, const float *__restrict__ a, const float *__restrict__ cur,
                                           float *__restrict__ nxt, int lane, int x0, int zb, int src, float fsrc) {
  const bool xok = x0 < L.NX4;
  const int col = L.origin + x0;
  float4 q[RZ + 8];
#pragma unroll
  for (int j = 0; j < RZ + 8; ++j) {
    const int z = zb - kHaloR + j;
    q[j] = (xok && z < L.NZ + kHaloR) ? ldg4(cur + col + z * L.pitch) : zero4();
  }
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int z = zb + j;
    if (z >= L.NZ) break;
    const int o = col + z * L.pitch;
    const float4 c = q[j + 4];
    float4 lf = shfl_up4(c), rt = shfl_dn4(c);
    if (lane == 0) lf = ldg4(cur + o - 4);
    if (lane == 31) rt = ldg4(cur + o + 4);
    if (xok) {
      const float4 av = ldg4(a + o);
      const float4 po = ld4(nxt + o);
      float4 r = leap4_2d(lf, c, rt, &q[j], po, av);
      const int d = src - o;
      if ((unsigned)d < 4u) point_sub(r, d, cmp(av, d) * fsrc);
      st4(nxt + o, r);
    }
  }
}

// One field of the reverse pass: advance (cur, nxt) and return the centre
// values of `cur` for the imaging condition.
template <int RZ, bool kInc>
__device__ __forceinline__ void rev_field2d(const Lay &L, const float *__restrict__ a,
                                            const float *__restrict__ cur, float *__restrict__ nxt,
                                            bool update, int lane, int x0, int zb, bool xok,
                                            int src, float fsrc, float4 *cen, float4 *inc) {
  const int col = L.origin + x0;
  if (!update) {
#pragma unroll
    for (int j = 0; j < RZ; ++j) {
      const int z = zb + j;
      cen[j] = (xok && z < L.NZ) ? ldg4(cur + col + z * L.pitch) : zero4();
    }
    return;
  }
  float4 q[RZ + 8];
#pragma unroll
  for (int j = 0; j < RZ + 8; ++j) {
    const int z = zb - kHaloR + j;
    q[j] = (xok && z < L.NZ + kHaloR) ? ldg4(cur + col + z * L.pitch) : zero4();
  }
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int z = zb + j;
    cen[j] = q[j + 4];
    if (z >= L.NZ) break;
    const int o = col + z * L.pitch;
    const float4 c = q[j + 4];
    float4 lf = shfl_up4(c), rt = shfl_dn4(c);
    if (lane == 0) lf = ldg4(cur + o - 4);
    if (lane == 31) rt = ldg4(cur + o + 4);
    if (xok) {
      const float4 av = ldg4(a + o);
      const float4 po = ld4(nxt + o);
      float4 r;
      if (kInc) {
        // the increment p^{n+1} - 2 p^n + p^{n-1} (point term included)
        const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w, rt.x, rt.y, rt.z, rt.w};
        r = leap4p_inc(w, &q[j], po, av, &inc[j]);
        const int d = src - o;
        if ((unsigned)d < 4u) {
          point_sub(r, d, cmp(av, d) * fsrc);
          point_sub(inc[j], d, cmp(av, d) * fsrc);
        }
      } else {
        r = leap4_2d(lf, c, rt, &q[j], po, av);
        const int d = src - o;
        if ((unsigned)d < 4u) point_sub(r, d, cmp(av, d) * fsrc);
      }
      st4(nxt + o, r);
    }
  }
}

// ---- shared-memory tiles (single-shot and batched reverse kernels) ----
// A block of NW warps covers 128 columns x T = NW * RZ rows.  The current
// level(s) over the tile and its 4-node halo (T + 8 rows x 136 columns) are
// staged in shared memory by 16-byte cp.async copies of the whole block (each
// row crosses L2 once per tile instead of (RZ + 8) / RZ times through a
// per-warp register queue, and no register holds a copy in flight), while
// every lane loads its own a and p^{n-1} float4s into registers; one barrier,
// then each warp updates its RZ rows with x and z neighbours from shared
// memory.  Rows beyond the zero halo below the grid are zero-filled.
__device__ __forceinline__ void cp_async16z(float *dst, const float *src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

constexpr int kStRow = kTileX + 2 * kHaloR;  // staged floats per row: x0 - 4 .. x0 + 131

// Stage rows Z0 - 4 .. Z0 + T + 3 of `f` (columns X0 - 4 .. X0 + 131) into `s`.
template <int T>
__device__ __forceinline__ void stage_rows(const Lay &L, const float *__restrict__ f, float *s, int X0, int Z0,
                                           int tid, int nthr) {
  constexpr int kCh = kStRow / 4;  // 16-byte chunks per row
  for (int i = tid; i < (T + 8) * kCh; i += nthr) {
    const int r = i / kCh, c = i - r * kCh;
    const int z = Z0 - kHaloR + r;
    const bool ok = z < L.NZ + kHaloR;  // rows -4 .. NZ + 3 exist (zero halo); z >= -4 always
    const float *src = f + (ok ? L.origin + z * L.pitch + X0 - kHaloR + 4 * c : 0);
    cp_async16z(s + r * kStRow + 4 * c, src, ok);
  }
}

// The leapfrog of Eq. 1 for the float4 of lane `lane` in staged row rr
// (rr = 4 + local row) of `s`.
__device__ __forceinline__ float4 leap_staged(const float *s, int rr, int lane, const float4 po, const float4 av,
                                              float4 *cen) {
  const float *row = s + rr * kStRow + 4 * lane;
  const float4 lf = *reinterpret_cast<const float4 *>(row);
  const float4 c = *reinterpret_cast<const float4 *>(row + 4);
  const float4 rt = *reinterpret_cast<const float4 *>(row + 8);
  float4 zq[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) zq[k] = *reinterpret_cast<const float4 *>(row + (k - 4) * kStRow + 4);
  *cen = c;
  return leap4_2d(lf, c, rt, zq, po, av);
}

__device__ __forceinline__ float4 staged_c(const float *s, int rr, int lane) {
  return *reinterpret_cast<const float4 *>(s + rr * kStRow + 4 * lane + 4);
}

// The tile's own rows of one pitched buffer (T rows x 128 columns) into `s`
// (rows beyond the zero halo below the grid are zero-filled).
template <int T>
__device__ __forceinline__ void stage_own(const Lay &L, const float *__restrict__ f, float *s, int X0, int Z0,
                                          int tid, int nthr) {
  constexpr int kCh = kTileX / 4;
  for (int i = tid; i < T * kCh; i += nthr) {
    const int r = i / kCh, c = i - r * kCh;
    const int z = Z0 + r;
    const bool ok = z < L.NZ + kHaloR;
    cp_async16z(s + r * kTileX + 4 * c, f + (ok ? L.origin + z * L.pitch + X0 + 4 * c : 0), ok);
  }
}

} // namespace rbc
