// rbc_kernels.cu -- sm_103a kernels of librbc.
//
// Hot path (Algorithm 3 of arXiv:2204.03380, per time step):
//   k_fwd2d / k_fwd3d : leapfrog step of Eq. 1 + fused point-source injection
//                       + fused receiver sampling (Algorithm 1).
//   k_rev2d / k_rev3d : one pass over the grid that advances the
//                       reconstruction p^R (Eq. 6, source re-subtracted) and the
//                       receiver wavefield pbar (Eq. 2, record injected) by one
//                       level back in time and accumulates the two integrals of
//                       the imaging condition (Eq. 3) -- a is read once for
//                       both updates.
// All are HBM/L2 streaming kernels (about 2 flop/byte): no tensor cores.
// Every lane owns a float4 (4 consecutive x) so a warp covers a 128-float,
// 512-byte row segment with fully coalesced 16-byte accesses; in 2-D the x
// neighbours come from the adjacent lanes by warp shuffles (lanes 0/31 fetch
// the 4-float halo) and the z neighbours from a register queue marching down
// z.  The 3-D kernels (TMA-fed plane rings) are in rbc_kernels3d.cu.
#include <cstdio>
#include <cstdlib>

#include "rbc_tile2d.cuh"

namespace rbc {

// Record the current level at every receiver (Algorithm 1 "record
// seismogram"): grid-strided so any block may sample any receiver.
__device__ __forceinline__ void sample_receivers(const StepArgs &A, int nblocks, int bid) {
  const int nrec = A.info->nrec;
  const int nthr = blockDim.x * blockDim.y;
  const int tid = bid * nthr + threadIdx.y * blockDim.x + threadIdx.x;
  for (int r = tid; r < nrec; r += nblocks * nthr)
    A.seis_t[(long long)A.n * nrec + r] = A.cur[A.rec_off[r]];
}

// Add the record at this block's receivers to the freshly written pbar_{n-1}
// (Eq. 2 source term).  Runs after the block's stores; the fence + barrier
// make those stores visible to the atomics of other threads of the block.
__device__ __forceinline__ void inject_receivers(const RevArgs &A, int bid) {
  const int beg = A.tile_ptr[bid], end = A.tile_ptr[bid + 1];
  if (end > beg) __threadfence();
  __syncthreads();
  if (end <= beg) return;
  const int nrec = A.info->nrec;
  const float sc = A.info->rec_scale;
  const int nthr = blockDim.x * blockDim.y;
  for (int k = beg + threadIdx.y * blockDim.x + threadIdx.x; k < end; k += nthr) {
    const int r = A.tile_rec[k];
    const int o = A.rec_off[r];
    atomicAdd(A.bn + o, sc * A.a[o] * A.seis_t[(long long)A.n * nrec + r]);
  }
}

// ------------------------------------------------------------------ 2-D ----
// Block: 32 x k2dWarpsF (forward) or 32 x k2dWarpsR (reverse) threads; tile
// 128 (x) x warps*RZ (z); each warp marches RZ rows with an (RZ + 8)-deep
// register queue.
template <int RZ>
__global__ void __launch_bounds__(32 * k2dWarpsF) k_fwd2d(const StepArgs A) {
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int x0 = blockIdx.x * kTileX + lane * 4;
  const int zb = (blockIdx.y * k2dWarpsF + w) * RZ;
  griddep_wait();
  if (A.sample) sample_receivers(A, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
  if (zb < L.NZ)  // warp-uniform; no block barrier in this kernel
    fwd2d_rows<RZ>(L, A.a, A.cur, A.nxt, lane, x0, zb, A.info->src_off, A.wav[A.n] * A.info->src_fwd);
  griddep_launch();
}

template <int RZ, bool kGrad>
__global__ void __launch_bounds__(32 * k2dWarpsR) k_rev2d(const RevArgs A) {
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int x0 = blockIdx.x * kTileX + lane * 4;
  const int zb = (blockIdx.y * k2dWarpsR + w) * RZ;
  const bool xok = x0 < L.NX4;
  const bool active = zb < L.NZ;  // warp-uniform
  griddep_wait();
  if (active) {
    float4 cr[RZ], cb[RZ], inc[RZ];
    const int src = A.info->src_off;
    const float fsrc = A.do_r ? A.wav[A.n_src] * A.info->src_rev : 0.f;  // f[nt] does not exist
    // Eq. 6: reconstruction (exact inverse of the forward step)
    rev_field2d<RZ, kGrad>(L, A.a, A.rc, A.rn, A.do_r != 0, lane, x0, zb, xok, src, fsrc, cr, inc);
    // Eq. 2 (or the FWI adjoint): receiver wavefield; the record is added below, after the store
    rev_field2d<RZ, false>(L, A.a, A.bc, A.bn, A.do_b != 0, lane, x0, zb, xok, -1, 0.f, cb, inc);
    if (kGrad) {
      // FWI: num += mu^m (p^m - 2 p^{m-1} + p^{m-2}) on the interior
      if (A.do_r && xok && x0 + 3 >= A.ix0 && x0 < A.ix1) {
#pragma unroll
        for (int j = 0; j < RZ; ++j) {
          const int z = zb + j;
          if (z >= A.iz0 && z < A.iz1) {
            const int o = L.origin + x0 + z * L.pitch;
            st4(A.num + o, add4(ld4(A.num + o), masked_prod(cb[j], inc[j], x0, A.ix0, A.ix1)));
          }
        }
      }
    } else if (xok && x0 + 3 >= A.ix0 && x0 < A.ix1) {
      // Eq. 3: the two time integrals, interior only
#pragma unroll
      for (int j = 0; j < RZ; ++j) {
        const int z = zb + j;
        if (z >= A.iz0 && z < A.iz1) {
          const int o = L.origin + x0 + z * L.pitch;
          st4(A.num + o, add4(ld4(A.num + o), masked_prod(cr[j], cb[j], x0, A.ix0, A.ix1)));
          st4(A.den + o, add4(ld4(A.den + o), masked_prod(cr[j], cr[j], x0, A.ix0, A.ix1)));
        }
      }
    }
  }
  if (A.do_b) inject_receivers(A, blockIdx.y * gridDim.x + blockIdx.x);
  griddep_launch();
}

// ---------------------------------------------- 2-D, shared-memory tiles ----
// (staging helpers in rbc_tile2d.cuh)
template <int RZ, int NW, int MB>
__global__ void __launch_bounds__(32 * NW, MB) k_fwd2d_tile(const StepArgs A) {
  constexpr int T = NW * RZ;
  __shared__ __align__(16) float s_p[(T + 8) * kStRow];
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int X0 = blockIdx.x * kTileX, Z0 = blockIdx.y * T;
  const int x0 = X0 + lane * 4, zb = Z0 + w * RZ;
  const bool xok = x0 < L.NX4;
  griddep_wait();
  if (A.sample) sample_receivers(A, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
  stage_rows<T>(L, A.cur, s_p, X0, Z0, tid, 32 * NW);
  asm volatile("cp.async.commit_group;" ::: "memory");
  float4 av[RZ], po[RZ];
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int o = L.origin + x0 + (zb + j) * L.pitch;
    const bool ok = xok && zb + j < L.NZ;
    av[j] = ok ? ldg4(A.a + o) : zero4();
    po[j] = ok ? ld4(A.nxt + o) : zero4();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int src = A.info->src_off;
  const float fsrc = A.wav[A.n] * A.info->src_fwd;
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int z = zb + j;
    if (xok && z < L.NZ) {
      const int o = L.origin + x0 + z * L.pitch;
      float4 c;
      float4 r = leap_staged(s_p, w * RZ + j + kHaloR, lane, po[j], av[j], &c);
      const int d = src - o;
      if ((unsigned)d < 4u) point_sub(r, d, cmp(av[j], d) * fsrc);
      st4(A.nxt + o, r);
    }
  }
  griddep_launch();
}

template <int RZ, int NW, int MB, bool kGrad>
__global__ void __launch_bounds__(32 * NW, MB) k_rev2d_tile(const RevArgs A) {
  constexpr int T = NW * RZ;
  __shared__ __align__(16) float s_r[(T + 8) * kStRow], s_b[(T + 8) * kStRow];
  __shared__ __align__(16) float s_num[T * kTileX], s_den[kGrad ? 4 : T * kTileX];
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int X0 = blockIdx.x * kTileX, Z0 = blockIdx.y * T;
  const int x0 = X0 + lane * 4, zb = Z0 + w * RZ;
  const bool xok = x0 < L.NX4;
  griddep_wait();
  stage_rows<T>(L, A.rc, s_r, X0, Z0, tid, 32 * NW);
  stage_rows<T>(L, A.bc, s_b, X0, Z0, tid, 32 * NW);
  // the imaging accumulators' rows: read-modify-written below, so their loads
  // fly with the fields' instead of stalling the update loop
  const bool img_tile = Z0 < A.iz1 && Z0 + T > A.iz0 && X0 < A.ix1 && X0 + kTileX > A.ix0;
  if (img_tile) {
    stage_own<T>(L, A.num, s_num, X0, Z0, tid, 32 * NW);
    if (!kGrad) stage_own<T>(L, A.den, s_den, X0, Z0, tid, 32 * NW);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  float4 av[RZ], pr[RZ], pb[RZ];
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int o = L.origin + x0 + (zb + j) * L.pitch;
    const bool ok = xok && zb + j < L.NZ;
    av[j] = ok ? ldg4(A.a + o) : zero4();
    pr[j] = ok && A.do_r ? ld4(A.rn + o) : zero4();
    pb[j] = ok && A.do_b ? ld4(A.bn + o) : zero4();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int src = A.info->src_off;
  const float fsrc = A.do_r ? A.wav[A.n_src] * A.info->src_rev : 0.f;  // f[nt] does not exist
  const bool img = xok && x0 + 3 >= A.ix0 && x0 < A.ix1;
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int z = zb + j, rr = w * RZ + j + kHaloR;
    if (!(xok && z < L.NZ)) continue;
    const int o = L.origin + x0 + z * L.pitch;
    const int d = src - o;
    float4 cr = staged_c(s_r, rr, lane), cb = staged_c(s_b, rr, lane), inc = zero4();
    if (A.do_r) {
      // Eq. 6: reconstruction (exact inverse of the forward step)
      float4 r;
      if (kGrad) {
        const float *row = s_r + rr * kStRow + 4 * lane;
        const float4 lf = *reinterpret_cast<const float4 *>(row), rt = *reinterpret_cast<const float4 *>(row + 8);
        float4 zq[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) zq[k] = *reinterpret_cast<const float4 *>(row + (k - 4) * kStRow + 4);
        const float w12[12] = {lf.x, lf.y, lf.z, lf.w, cr.x, cr.y, cr.z, cr.w, rt.x, rt.y, rt.z, rt.w};
        r = leap4p_inc(w12, zq, pr[j], av[j], &inc);
        if ((unsigned)d < 4u) point_sub(inc, d, cmp(av[j], d) * fsrc);
      } else {
        r = leap_staged(s_r, rr, lane, pr[j], av[j], &cr);
      }
      if ((unsigned)d < 4u) point_sub(r, d, cmp(av[j], d) * fsrc);
      st4(A.rn + o, r);
    }
    if (A.do_b) {
      // Eq. 2 (or the FWI adjoint): the record is added below, after the stores
      st4(A.bn + o, leap_staged(s_b, rr, lane, pb[j], av[j], &cb));
    }
    if (img && z >= A.iz0 && z < A.iz1) {
      const int so = (w * RZ + j) * kTileX + 4 * lane;
      if (kGrad) {
        // FWI: num += mu^m (p^m - 2 p^{m-1} + p^{m-2}) on the interior
        if (A.do_r) st4(A.num + o, add4(ld4(s_num + so), masked_prod(cb, inc, x0, A.ix0, A.ix1)));
      } else {
        // Eq. 3: the two time integrals, interior only
        st4(A.num + o, add4(ld4(s_num + so), masked_prod(cr, cb, x0, A.ix0, A.ix1)));
        st4(A.den + o, add4(ld4(s_den + so), masked_prod(cr, cr, x0, A.ix0, A.ix1)));
      }
    }
  }
  if (A.do_b) inject_receivers(A, blockIdx.y * gridDim.x + blockIdx.x);
  griddep_launch();
}

// ------------------------------------------ 2-D, two levels per launch ----
// Temporal blocking of the forward step: one launch advances (p^{n-1}, p^n)
// to (p^{n+1}, p^{n+2}).  A block of 4 warps owns a tile of 128 columns x 8
// rows.  It stages p^n over the tile and an 8-node apron (24 x 144 floats),
// p^{n-1} and a over a 4-node apron (16 x 136 each), computes p^{n+1} over the
// 4-node apron into shared memory (the source term with f[n]), then p^{n+2}
// over the tile (f[n+1]), and writes both levels of its tile.  Level m lives
// in buffer m mod 4 of a four-buffer rotation, so no launch writes a buffer
// that a neighbouring block still reads.  The receivers of the tile (the
// reverse kernel's per-tile lists, same 128 x 8 tiling) record levels n and
// n + 1 from shared memory.
constexpr int kT2 = 8;                          // rows per tile
constexpr int kP2W = kTileX + 4 * kHaloR;        // 144: p^n row, x0 - 8 .. x0 + 135
constexpr int kQ2W = kTileX + 2 * kHaloR;        // 136: apron rows, x0 - 4 .. x0 + 131

// Rows z0 .. z0 + rows - 1, columns x0 .. x0 + 4 chunks - 1 of `f` into `s`
// (row stride `stride` floats); rows outside -4 .. NZ + 3 are zero-filled.
__device__ __forceinline__ void stage_box(const Lay &L, const float *__restrict__ f, float *s, int x0, int z0,
                                          int rows, int chunks, int stride, int tid, int nthr) {
  for (int i = tid; i < rows * chunks; i += nthr) {
    const int r = i / chunks, c = i - r * chunks;
    const int z = z0 + r;
    const bool ok = z >= -kHaloR && z < L.NZ + kHaloR;
    cp_async16z(s + r * stride + 4 * c, f + (ok ? L.origin + z * L.pitch + x0 + 4 * c : 0), ok);
  }
}

__global__ void __launch_bounds__(128, 5) k_fwd2d_2lev(const StepArgs A, const float *__restrict__ prev,
                                                       float *__restrict__ out1, float *__restrict__ out2,
                                                       const int *__restrict__ tile_ptr,
                                                       const int *__restrict__ tile_rec) {
  __shared__ __align__(16) float s_c[(kT2 + 16) * kP2W];  // p^n
  __shared__ __align__(16) float s_p[(kT2 + 8) * kQ2W];   // p^{n-1}
  __shared__ __align__(16) float s_a[(kT2 + 8) * kQ2W];   // a
  __shared__ __align__(16) float s_q[(kT2 + 8) * kQ2W];   // p^{n+1}
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int X0 = blockIdx.x * kTileX, Z0 = blockIdx.y * kT2;
  griddep_wait();
  stage_box(L, A.cur, s_c, X0 - 2 * kHaloR, Z0 - 2 * kHaloR, kT2 + 16, kP2W / 4, kP2W, tid, 128);
  stage_box(L, prev, s_p, X0 - kHaloR, Z0 - kHaloR, kT2 + 8, kQ2W / 4, kQ2W, tid, 128);
  stage_box(L, A.a, s_a, X0 - kHaloR, Z0 - kHaloR, kT2 + 8, kQ2W / 4, kQ2W, tid, 128);
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int src = A.info->src_off;
  const float f0 = A.wav[A.n] * A.info->src_fwd, f1 = A.wav[A.n + 1] * A.info->src_fwd;
  // p^{n+1} over the apron: rows Z0 - 4 .. Z0 + 11, columns X0 - 4 .. X0 + 131
  // (34 float4 per row: lane k and, for lanes 0 and 1, float4 32 + lane);
  // outside the grid every staged value is zero, so the update is zero there
  for (int r = w * 4; r < w * 4 + 4; ++r) {
    const int z = Z0 - kHaloR + r;
    for (int c4 = lane; c4 < kQ2W / 4; c4 += 32) {
      const float *row = s_c + (r + kHaloR) * kP2W + 4 * c4;  // p^n at x = X0 - 8 + 4 c4 ..
      const float4 lf = *reinterpret_cast<const float4 *>(row), c = *reinterpret_cast<const float4 *>(row + 4),
                   rt = *reinterpret_cast<const float4 *>(row + 8);
      float4 zq[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) zq[k] = *reinterpret_cast<const float4 *>(row + (k - 4) * kP2W + 4);
      const float4 av = *reinterpret_cast<const float4 *>(s_a + r * kQ2W + 4 * c4);
      const float4 po = *reinterpret_cast<const float4 *>(s_p + r * kQ2W + 4 * c4);
      float4 v = leap4_2d(lf, c, rt, zq, po, av);
      const int d = src - (L.origin + z * L.pitch + X0 - kHaloR + 4 * c4);
      if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * f0);
      *reinterpret_cast<float4 *>(s_q + r * kQ2W + 4 * c4) = v;
    }
  }
  __syncthreads();
  // p^{n+2} over the tile; both levels of the tile to their buffers
  const int x0 = X0 + lane * 4;
  const bool xok = x0 < L.NX4;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int rl = w * 2 + j, z = Z0 + rl;
    if (!(xok && z < L.NZ)) continue;
    const float *row = s_q + (rl + kHaloR) * kQ2W + 4 * lane;  // p^{n+1} at x = x0 - 4 ..
    const float4 lf = *reinterpret_cast<const float4 *>(row), c = *reinterpret_cast<const float4 *>(row + 4),
                 rt = *reinterpret_cast<const float4 *>(row + 8);
    float4 zq[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) zq[k] = *reinterpret_cast<const float4 *>(row + (k - 4) * kQ2W + 4);
    const float4 av = *reinterpret_cast<const float4 *>(s_a + (rl + kHaloR) * kQ2W + 4 * lane + 4);
    const float4 po = *reinterpret_cast<const float4 *>(s_c + (rl + 2 * kHaloR) * kP2W + 4 * lane + 8);
    float4 v = leap4_2d(lf, c, rt, zq, po, av);
    const int o = L.origin + z * L.pitch + x0;
    const int d = src - o;
    if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * f1);
    st4(out1 + o, c);
    st4(out2 + o, v);
  }
  // record levels n and n + 1 at this tile's receivers
  if (A.sample) {
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    const int nrec = A.info->nrec;
    for (int k = tile_ptr[bid] + tid; k < tile_ptr[bid + 1]; k += 128) {
      const int r = tile_rec[k];
      const int off = A.rec_off[r] - L.origin;
      const int z = off / L.pitch, x = off - z * L.pitch;
      A.seis_t[(long long)A.n * nrec + r] = s_c[(z - Z0 + 2 * kHaloR) * kP2W + x - X0 + 2 * kHaloR];
      A.seis_t[(long long)(A.n + 1) * nrec + r] = s_q[(z - Z0 + kHaloR) * kQ2W + x - X0 + kHaloR];
    }
  }
  griddep_launch();
}

bool launch_fwd2_2d(const StepArgs &A, const float *prev, float *out1, float *out2, const int *tile_ptr,
                    const int *tile_rec, cudaStream_t s) {
  const Lay &L = A.L;
  if (L.ndim != 2) return false;
  const dim3 grid((L.NX + kTileX - 1) / kTileX, (L.NZ + kT2 - 1) / kT2);
  launch_pdl(k_fwd2d_2lev, grid, dim3(32, 4), 0, s, A, prev, out1, out2, tile_ptr, tile_rec);
  return true;
}

int fwd2_tile_rows() { return kT2; }

// ------------------------------------------------------------ launchers ----
static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// 2-D kernel shapes: 0 = register-queue kernels (k_fwd2d 4 warps x 2 rows,
// k_rev2d 8 warps x 2 rows); 1 = shared-memory tiles of 4 warps x 2 rows,
// 7 resident blocks per SM asked of the compiler (k_fwd2d_tile /
// k_rev2d_tile).  Measured on the survey grid (2421 x 871, warm L2, per
// launch): forward 5.78 us (shape 0) vs 6.32 us (1); reverse 15.25 us (0) vs
// 13.54 us (1); other tile shapes (2 x 8, 4 x 4, 1 x 8, no register cap) lost
// to both.  Default: forward 0, reverse 1; RBC_TILE2D="fwd,rev" overrides it
// (read once per process).
struct Shape2d { int fwd, rev; };
static Shape2d shape2d() {
  static Shape2d sh = [] {
    Shape2d v{0, 1};
    const char *e = getenv("RBC_TILE2D");
    if (e) {
      int f = -1, r = -1;
      if (sscanf(e, "%d,%d", &f, &r) == 2 && f >= 0 && f <= 1 && r >= 0 && r <= 1) v = Shape2d{f, r};
    }
    return v;
  }();
  return sh;
}
static int tile_rows_2d(int k, bool fwd) {
  if (k == 1) return 8;
  return fwd ? k2dWarpsF * k2dRowsF : k2dWarpsR * k2dRowsR;
}

bool launch_fwd(const StepArgs &A, cudaStream_t s) {
  const Lay &L = A.L;
  if (L.ndim == 3) return launch_fwd3d(A, s);
  const int k = shape2d().fwd;
  dim3 grid(cdiv(L.NX, kTileX), cdiv(L.NZ, tile_rows_2d(k, true)));
  if (k == 1)
    launch_pdl(k_fwd2d_tile<2, 4, 7>, grid, dim3(32, 4), 0, s, A);
  else
    launch_pdl(k_fwd2d<k2dRowsF>, grid, dim3(32, k2dWarpsF), 0, s, A);
  return true;
}

void rev_tiling(const Lay &L, int zc, int *gx, int *gy, int *gz, int *t) {
  if (L.ndim == 2) {
    *t = tile_rows_2d(shape2d().rev, false);
    *gx = cdiv(L.NX, kTileX);
    *gy = cdiv(L.NZ, *t);
    *gz = 1;
  } else {
    *gx = cdiv(L.NX, kTileX);
    *gy = cdiv(L.NY, tile_rows_3d());
    *gz = cdiv(L.NZ, zc);
    *t = tile_rows_3d();
  }
}

bool launch_rev(const RevArgs &A, cudaStream_t s) {
  if (A.L.ndim == 3) return launch_rev3d(A, s);
  int gx, gy, gz, t;
  rev_tiling(A.L, A.zc, &gx, &gy, &gz, &t);
  const dim3 grid(gx, gy);
  const bool g = A.mode == 1;
  if (shape2d().rev == 1)
    launch_pdl(g ? k_rev2d_tile<2, 4, 7, true> : k_rev2d_tile<2, 4, 7, false>, grid, dim3(32, 4), 0, s, A);
  else
    launch_pdl(g ? k_rev2d<k2dRowsR, true> : k_rev2d<k2dRowsR, false>, grid, dim3(32, k2dWarpsR), 0, s, A);
  return true;
}

// ----------------------------------------------------------- auxiliaries ----
__global__ void k_copy_in(const Lay L, const float *__restrict__ dense, float *__restrict__ pitched) {
  const long long n = (long long)L.NX * L.NY * L.NZ;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.NX);
    const long long r = i / L.NX;
    const int y = (int)(r % L.NY);
    const int z = (int)(r / L.NY);
    pitched[lay_off(L, x, y, z)] = dense[i];
  }
}

__global__ void k_copy_out(const Lay L, const float *__restrict__ pitched, float *__restrict__ dense) {
  const long long n = (long long)L.NX * L.NY * L.NZ;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.NX);
    const long long r = i / L.NX;
    const int y = (int)(r % L.NY);
    const int z = (int)(r / L.NY);
    dense[i] = pitched[lay_off(L, x, y, z)];
  }
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  return (int)(b < 1 ? 1 : b);
}

void launch_copy_in(const Lay &L, const float *dense, float *pitched, cudaStream_t s) {
  const long long n = (long long)L.NX * L.NY * L.NZ;
  k_copy_in<<<grid_for(n, 256), 256, 0, s>>>(L, dense, pitched);
}

void launch_copy_out(const Lay &L, const float *pitched, float *dense, cudaStream_t s) {
  const long long n = (long long)L.NX * L.NY * L.NZ;
  k_copy_out<<<grid_for(n, 256), 256, 0, s>>>(L, pitched, dense);
}

// out[c][r] = in[r][c] for an rows x cols matrix (32 x 32 shared tiles).
__global__ void k_transpose(const float *__restrict__ in, float *__restrict__ out, int rows, int cols) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[k][threadIdx.x] = in[(long long)r * cols + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(long long)c * rows + r] = t[threadIdx.x][k];
  }
}

void launch_transpose(const float *in, float *out, int rows, int cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32));
  k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
}

__global__ void k_accum_interior(const Lay L, const float *__restrict__ pitched, float *__restrict__ dense,
                                 int nb, int top, int nx, int ny, int nz, int overwrite) {
  const long long n = (long long)nx * ny * nz;
  const int yo = (L.ndim == 3) ? nb : 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    const float v = pitched[lay_off(L, x + nb, y + yo, z + top)];
    dense[i] = overwrite ? v : dense[i] + v;
  }
}

void launch_accum_interior(const Lay &L, const float *pitched, float *dense, int nb, int top, int nx, int ny,
                           int nz, int overwrite, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  k_accum_interior<<<grid_for(n, 256), 256, 0, s>>>(L, pitched, dense, nb, top, nx, ny, nz, overwrite);
}

// Maximum of non-negative values as ordered uint bits (atomicMax).
__global__ void k_max(const float *__restrict__ x, long long n, unsigned int *out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(out, __float_as_uint(m));
  }
}

void launch_max(const float *x, long long n, unsigned int *out_bits, cudaStream_t s) {
  k_max<<<grid_for(n, 256), 256, 0, s>>>(x, n, out_bits);
}

__global__ void k_image_stack(const float *__restrict__ num, const float *__restrict__ den,
                              const unsigned int *__restrict__ maxbits, float eps_rel, int nx, int ny,
                              int nz, int off_x, int off_y, int sx, int sy, float *__restrict__ image) {
  const long long n = (long long)nx * ny * nz;
  const float e = eps_rel * __uint_as_float(*maxbits);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    image[((long long)z * sy + y + off_y) * sx + x + off_x] += num[i] / (den[i] + e);
  }
}

void launch_image_stack(const float *num, const float *den, const unsigned int *maxbits, float eps_rel,
                        int nx, int ny, int nz, int off_x, int off_y, int sx, int sy, float *image,
                        cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  k_image_stack<<<grid_for(n, 256), 256, 0, s>>>(num, den, maxbits, eps_rel, nx, ny, nz, off_x, off_y,
                                                 sx, sy, image);
}

// ------------------------------------------------------------------ FWI ----
// resid[r][n] = seis_t[n][r] - dobs[r][n]; misfit += 1/2 sum resid^2 (fp64).
__global__ void k_fwi_residual(const float *__restrict__ seis_t, const float *__restrict__ dobs,
                               float *__restrict__ resid, double *misfit, int nrec, int nt) {
  const long long n = (long long)nrec * (nt + 1);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / (nt + 1)), t = (int)(i % (nt + 1));
    const float d = seis_t[(long long)t * nrec + r] - dobs[i];
    resid[i] = d;
    acc += 0.5 * (double)d * (double)d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(misfit, acc);
}

void launch_fwi_residual(const float *seis_t, const float *dobs, float *resid, double *misfit, int nrec, int nt,
                         cudaStream_t s) {
  const long long n = (long long)nrec * (nt + 1);
  k_fwi_residual<<<grid_for(n, 256), 256, 0, s>>>(seis_t, dobs, resid, misfit, nrec, nt);
}

// Adjoint record, time-major with nt + 2 rows: row m = scale * resid[.][m-1]
// for m = 1..nt+1, row 0 = 0 (the reverse kernel injects row m when it forms
// level m - 1 of the adjoint field).
__global__ void k_fwi_adjoint_source(const float *__restrict__ resid, float *__restrict__ seis_t, int nrec, int nt,
                                     float scale) {
  const long long n = (long long)nrec * (nt + 2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / nrec), r = (int)(i % nrec);
    seis_t[i] = m == 0 ? 0.f : scale * resid[(long long)r * (nt + 1) + m - 1];
  }
}

void launch_fwi_adjoint_source(const float *resid, float *seis_t, int nrec, int nt, float scale, cudaStream_t s) {
  const long long n = (long long)nrec * (nt + 2);
  k_fwi_adjoint_source<<<grid_for(n, 256), 256, 0, s>>>(resid, seis_t, nrec, nt, scale);
}

// dJ/dv = dJ/da * da/dv with dJ/da = -num / a^2 (num = sum mu p_tt, mu = a
// lambda) and da/dv = 2 a / v, v = sqrt(a) h / dt:  grad += -2 num dt / (a^1.5 h).
__global__ void k_fwi_finalize(const Lay L, const float *__restrict__ num, const float *__restrict__ a,
                               float *__restrict__ grad, int nb, int nx, int nz, double dt, double h) {
  const long long n = (long long)nx * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), z = (int)(i / nx);
    const int o = lay_off(L, x + nb, 0, z + nb);
    const double av = a[o];
    atomicAdd(grad + i, (float)(-2.0 * (double)num[o] * dt / (av * sqrt(av) * h)));
  }
}

void launch_fwi_finalize(const Lay &L, const float *num, const float *a, float *grad, int nb, int nx, int nz,
                         double dt, double h, cudaStream_t s) {
  const long long n = (long long)nx * nz;
  k_fwi_finalize<<<grid_for(n, 256), 256, 0, s>>>(L, num, a, grad, nb, nx, nz, dt, h);
}

// ----------------------------------------------------- random boundary ----
// splitmix64 (Steele, Lea & Flood 2014) as a counter generator: draw j of
// stream `seed` is the finaliser applied to seed + j * golden-gamma.
__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t j) {
  uint64_t z = seed + j * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(uint64_t seed, uint64_t j) {
  return (double)(sm64(seed, j) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ int pad_distance(int q, int nb, int n) {
  return q < nb ? nb - q : (q >= nb + n ? q - (nb + n - 1) : 0);
}

// Section 4.3: random velocities in an nb-cell pad, blended towards the
// nearest interior value with a coefficient between the Gaussian (Eq. 5) and
// linear (Eq. 4) tapers; a = (v dt / h)^2.
__global__ void k_rbc_build(int ndim, int nx, int ny, int nz, int nb, int top, const float *__restrict__ v_int,
                            double v_lo, double v_hi, double v_max, uint64_t seed, int mode, double dt,
                            double h, float *__restrict__ v_pad, float *__restrict__ a) {
  const int NX = nx + 2 * nb, NZ = nz + nb + top;
  const int NY = (ndim == 3) ? ny + 2 * nb : 1;
  const int nyi = (ndim == 3) ? ny : 1;
  const long long n = (long long)NX * NY * NZ;
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < n;
       L += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(L % NX);
    const long long r = L / NX;
    const int y = (int)(r % NY);
    const int z = (int)(r / NY);
    if (top != nb && z < top) {  // free surface: the zero-pressure rows (a = 0 keeps p = 0)
      if (v_pad) v_pad[L] = 0.f;
      a[L] = 0.f;
      continue;
    }
    int i = max(pad_distance(x, nb, nx), pad_distance(z, top, nz));
    if (ndim == 3) i = max(i, pad_distance(y, nb, ny));
    const int ex = min(max(x - nb, 0), nx - 1), ez = min(max(z - top, 0), nz - 1);
    const int ey = (ndim == 3) ? min(max(y - nb, 0), ny - 1) : 0;
    double v = (double)v_int[((long long)ez * nyi + ey) * nx + ex];
    if (i > 0) {
      const double g = (double)(nb - i) / (double)(nb - 1);
      const double uu = (double)(i - 1) / (double)(nb - 1);
      const double hh = exp(-120.0 * uu * uu);
      const double lo = hh < g ? hh : g, up = hh < g ? g : hh;
      const double c = lo + (up - lo) * u01(seed, 2ULL * (uint64_t)L + 1ULL);
      const double vr = v_lo + (v_hi - v_lo) * u01(seed, 2ULL * (uint64_t)L + 2ULL);
      if (mode == 0) {
        v = c * v + (1.0 - c) * vr;
      } else {
        v = c * vr;
        if (v < v_lo) v = v_lo;
      }
      if (v > v_max) v = v_max;
    }
    if (v_pad) v_pad[L] = (float)v;
    const double cc = v * dt / h;
    a[L] = (float)(cc * cc);
  }
}

void launch_rbc_build(int ndim, int nx, int ny, int nz, int nb, int top, const float *v_int, double v_lo,
                      double v_hi, double v_max, uint64_t seed, int mode, double dt, double h,
                      float *v_pad, float *a, cudaStream_t s) {
  const long long n = (long long)(nx + 2 * nb) * (ndim == 3 ? ny + 2 * nb : 1) * (nz + nb + top);
  k_rbc_build<<<grid_for(n, 256), 256, 0, s>>>(ndim, nx, ny, nz, nb, top, v_int, v_lo, v_hi, v_max, seed,
                                               mode, dt, h, v_pad, a);
}

// -------------------------------------- RTM with wavefield storage ----
// Algorithm 2 keeps the source wavefield every k steps (Eq. 7); the kept
// level is the interior box as a dense [nz][ny][nx] slot.  Threads run along
// x of one interior row (coalesced on both sides), blocks stride over rows.
__global__ void k_store_level(const Lay L, const float *__restrict__ p, float *__restrict__ slot, int nb, int top,
                              int nx, int ny, int nz) {
  griddep_wait();
  const int yo = (L.ndim == 3) ? nb : 0;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < nx)
    for (int r = blockIdx.y; r < ny * nz; r += gridDim.y) {
      const int y = r % ny, z = r / ny;
      slot[(long long)r * nx + x] = p[lay_off(L, x + nb, y + yo, z + top)];
    }
  griddep_launch();
}

// Eq. 3 integrals at a kept level n: num += p^n pbar_n, den += (p^n)^2, with
// p^n read back from its slot (num/den in the pitched layout).
__global__ void k_store_image(const Lay L, const float *__restrict__ slot, const float *__restrict__ pb,
                              float *__restrict__ num, float *__restrict__ den, int nb, int top, int nx, int ny,
                              int nz) {
  griddep_wait();
  const int yo = (L.ndim == 3) ? nb : 0;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < nx)
    for (int r = blockIdx.y; r < ny * nz; r += gridDim.y) {
      const int y = r % ny, z = r / ny;
      const int o = lay_off(L, x + nb, y + yo, z + top);
      const float v = slot[(long long)r * nx + x];
      num[o] += v * pb[o];
      den[o] += v * v;
    }
  griddep_launch();
}

// Eq. 2 source term after a receiver-wavefield step: pbar_{n-1} at the
// receivers += a_r s[r][n] h^(2-d) (atomics: receivers may share a node).
__global__ void k_rec_inject(const float *__restrict__ a, float *__restrict__ bn, const int *__restrict__ rec_off,
                             const ShotInfo *info, const float *__restrict__ seis_t, int n) {
  griddep_wait();
  const int nrec = info->nrec;
  const float sc = info->rec_scale;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
    const int o = rec_off[r];
    atomicAdd(bn + o, sc * a[o] * seis_t[(long long)n * nrec + r]);
  }
  griddep_launch();
}

static dim3 interior_grid(int nx, int rows) {
  return dim3(cdiv(nx, 128), (unsigned)min(rows, 4 * 152 * 16 / max(1, cdiv(nx, 128))));
}

void launch_store_level(const Lay &L, const float *p, float *slot, int nb, int top, int nx, int ny, int nz,
                        cudaStream_t s) {
  launch_pdl(k_store_level, interior_grid(nx, ny * nz), dim3(128), 0, s, L, p, slot, nb, top, nx, ny, nz);
}

void launch_store_image(const Lay &L, const float *slot, const float *pb, float *num, float *den, int nb, int top,
                        int nx, int ny, int nz, cudaStream_t s) {
  launch_pdl(k_store_image, interior_grid(nx, ny * nz), dim3(128), 0, s, L, slot, pb, num, den, nb, top, nx, ny,
             nz);
}

void launch_rec_inject(const float *a, float *bn, const int *rec_off, const ShotInfo *info, const float *seis_t,
                       int n, int nrec_cap, cudaStream_t s) {
  launch_pdl(k_rec_inject, dim3(cdiv(max(nrec_cap, 1), 256)), dim3(256), 0, s, a, bn, rec_off, info, seis_t, n);
}

} // namespace rbc
