// rbc_kernels3d.cu -- 3-D stencil kernels of librbc for sm_103a, fed by TMA.
//
// Each block owns a 128 (x) x TY (y) column tile and marches down a chunk of
// z planes.  One elected thread streams the x-y planes the block needs through
// shared-memory rings with cp.async.bulk.tensor (TMA, no multicast) and
// mbarrier completion:
//   * the P ring holds planes of the current field(s) with a 4-node halo in x
//     and y ((TY + 8) x 136 floats); a plane stays from the iteration that
//     pushes it onto the z queue (z + 4) to the one that uses it as the centre
//     plane (z), so the ring is at least 5 deep plus the prefetch distance;
//   * the T ring holds the block's own tiles of the plane being updated
//     (a and the level overwritten in place), TY x 128 floats each.
// Threads own a float4 in x; x neighbours come from the halo row in shared
// memory, y neighbours from the rows above/below, z neighbours from a 9-deep
// register queue.  Every mbarrier wait is bounded (about a second of clock);
// a block whose wait gives up records the fact in the context's error word,
// lets every in-flight copy land (again bounded) and leaves the plane loop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rbc_internal.cuh"
#include "rbc_stencil.cuh"

namespace rbc {

namespace {

constexpr int kTY = 8;        // y rows per reverse tile (one warp per field each)
#ifndef RBC_FWD3D_ROWS
#define RBC_FWD3D_ROWS 16
#endif
constexpr int kTYf = RBC_FWD3D_ROWS;  // y rows per forward tile (one warp each)
constexpr int kRP = 8;        // forward P ring: 5 live planes + 3 in flight
constexpr int kRT = 5;        // forward T ring: 1 live plane + 4 in flight
constexpr int kRPr = 8;       // reverse P ring (two fields): 5 live + 3 in flight
constexpr int kRTr = 4;       // reverse T ring (a, p^R, pbar, num, den): 1 live + 3 in flight
constexpr int kHaloW = 136;   // 128 + 2 x 4 halo floats
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

constexpr int kPStage = (kTY + 8) * kHaloW;  // floats per field per P stage
constexpr int kTTile = kTY * 128;            // floats per tile

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sa(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on one phase of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void tma3(float *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          sa(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
      : "memory");
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float cmp(const float4 &v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Leapfrog update of 4 consecutive nodes (see rbc_stencil.cuh).  xr: this
// thread's halo row in shared memory at the centre plane (float4 at xr =
// x0-4..x0-1, xr+4 = centre, xr+8 = right); rows +-k sit at +-k*kHaloW;
// zq[0..8]: z queue.
__device__ __forceinline__ float4 leap4_3d(const float *xr, const float4 *zq, const float4 po, const float4 av) {
  const float4 lf = lds4(xr), c = lds4(xr + 4), rt = lds4(xr + 8);
  float4 ym[4], yp[4];
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    ym[k - 1] = lds4(xr + 4 - k * kHaloW);
    yp[k - 1] = lds4(xr + 4 + k * kHaloW);
  }
  const float w[12] = {lf.x, lf.y, lf.z, lf.w, c.x, c.y, c.z, c.w, rt.x, rt.y, rt.z, rt.w};
  return leap4p<true>(w, zq, ym, yp, po, av);
}

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

__device__ __forceinline__ void flag_error(int *err, int code) {
  if (err) atomicOr_system(err, code);
}

// Warp-specialised pipeline: warps 0..kTY-1 (and kTY..2kTY-1 in the reverse
// kernel) consume, the last warp produces.  Each ring stage has a "full"
// barrier (one arrival + the TMA byte count) and an "empty" barrier (one
// arrival per consumer warp when it is done with the stage), so consumer warps
// never meet at a block-wide barrier inside the plane loop and the producer
// refills a stage as soon as every consumer has released it.

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another thread of the block has
// flagged an abort; sets the flag itself when its own time runs out.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, uint32_t parity, volatile int *abort_blk) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_blk) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_blk = 1;
      return false;
    }
  }
  return true;
}

// Persistent blocks: the grid has one block per resident slot and every block
// walks a strided list of tiles (128 x kTY columns x one z chunk).  Per tile
// the P sequence is the planes zb-4 .. ze+3 (the first four only feed the z
// queue) and the T sequence the planes zb .. ze-1; sequence numbers keep
// counting across tiles, so the producer streams the next tile's planes while
// the consumers finish the current one.  A P ring of at least 8 stages holds a
// tile's first 8 planes at once.

struct Tile3 {
  int bx, by, zb, ze;
};

__device__ __forceinline__ Tile3 tile_of(int t, int gx, int gy, int zc, int NZ) {
  Tile3 T;
  T.bx = t % gx;
  const int u = t / gx;
  T.by = u % gy;
  T.zb = (u / gy) * zc;
  T.ze = min(T.zb + zc, NZ);
  return T;
}

// ------------------------------------------------------------- forward ----
template <int TY>
constexpr size_t fwd_smem() {
  return sizeof(float) * (kRP * (TY + 8) * kHaloW + kRT * 2 * TY * 128) + 16 * (kRP + kRT) + 16;
}
static_assert(kRP >= 8, "the P ring must hold a tile's first 8 planes");

// TY rows per tile (one consumer warp each) plus one producer warp.
template <int TY>
__global__ void __launch_bounds__(32 * (TY + 1)) k_fwd3d_tma(const __grid_constant__ CUtensorMap tm_cur,
                                                               const __grid_constant__ CUtensorMap tm_a,
                                                               const __grid_constant__ CUtensorMap tm_old,
                                                               const StepArgs A) {
  constexpr int kPStage = (TY + 8) * kHaloW;
  constexpr int kTTile = TY * 128;
  extern __shared__ __align__(128) float smem[];
  float *sp = smem;                         // [kRP][TY + 8][136]
  float *st = sp + kRP * kPStage;           // [kRT][2][TY][128]  (a, old)
  uint64_t *fullP = reinterpret_cast<uint64_t *>(st + kRT * 2 * kTTile);
  uint64_t *emptyP = fullP + kRP;
  uint64_t *fullT = emptyP + kRP;
  uint64_t *emptyT = fullT + kRT;
  volatile int *abort_blk = reinterpret_cast<volatile int *>(emptyT + kRT);
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int nthr = blockDim.x * blockDim.y;
  const int gx = (L.NX + kTileX - 1) / kTileX, gy = (L.NY + TY - 1) / TY;
  const int ntiles = gx * gy * ((L.NZ + A.zc - 1) / A.zc);
  if (A.sample) {
    const int nrec = A.info->nrec;
    for (int r = blockIdx.x * nthr + tid; r < nrec; r += gridDim.x * nthr)
      A.seis_t[(long long)A.n * nrec + r] = A.cur[A.rec_off[r]];
  }
  if (tid == 0) {
    *abort_blk = 0;
    for (int s = 0; s < kRP; ++s) mbar_init(&fullP[s], 1), mbar_init(&emptyP[s], TY);
    for (int s = 0; s < kRT; ++s) mbar_init(&fullT[s], 1), mbar_init(&emptyT[s], TY);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (w == TY) {
    // ---- producer (one lane): P planes and T tiles in the order they are consumed
    if (lane == 0) {
      const uint32_t pbytes = sizeof(float) * kPStage, tbytes = sizeof(float) * 2 * kTTile;
      int gp = 0, gt = 0;  // sequence numbers
      bool ok = true;
      // failure-detection test hook: block 0 of the first step never issues
      // P plane 8, so its consumers' bounded wait runs out
      const int withhold = (A.info->fault == 1 && A.n == 0 && blockIdx.x == 0) ? 8 : -1;
      auto issueP = [&](int plane, int hx, int hy) {
        if (gp == withhold) {
          ++gp;
          return;
        }
        const int s = gp % kRP, f = gp / kRP;
        if (f > 0) ok = mbar_wait_ab(&emptyP[s], (f - 1) & 1, abort_blk);
        if (!ok) return;
        mbar_expect_tx(&fullP[s], pbytes);
        tma3(sp + s * kPStage, &tm_cur, hx, hy, plane + kHaloR, &fullP[s]);
        ++gp;
      };
      auto issueT = [&](int plane, int tx, int ty) {
        const int s = gt % kRT, f = gt / kRT;
        if (f > 0) ok = mbar_wait_ab(&emptyT[s], (f - 1) & 1, abort_blk);
        if (!ok) return;
        mbar_expect_tx(&fullT[s], tbytes);
        tma3(st + s * 2 * kTTile, &tm_a, tx, ty, plane + kHaloR, &fullT[s]);
        tma3(st + s * 2 * kTTile + kTTile, &tm_old, tx, ty, plane + kHaloR, &fullT[s]);
        ++gt;
      };
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        const Tile3 T = tile_of(t, gx, gy, A.zc, L.NZ);
        const int hx = T.bx * kTileX + kHaloX - 4, hy = T.by * TY;       // halo box (tensor coords)
        const int tx = T.bx * kTileX + kHaloX, ty = T.by * TY + kHaloR;  // tile box
        for (int i = 0; ok && i < 8; ++i) issueP(T.zb - 4 + i, hx, hy);
        for (int r = 0; ok && r < T.ze - T.zb; ++r) {
          issueP(T.zb + r + 4, hx, hy);
          if (ok) issueT(T.zb + r, tx, ty);
        }
      }
      if (*abort_blk) {
        flag_error(A.err, 1);
        // let every issued copy land before the block's shared memory is released
        for (int k = max(0, gp - kRP); k < gp; ++k)
          if (k != withhold) mbar_wait(&fullP[k % kRP], (k / kRP) & 1);
        for (int k = max(0, gt - kRT); k < gt; ++k) mbar_wait(&fullT[k % kRT], (k / kRT) & 1);
      }
    }
    return;
  }
  // ---- consumers: one row of the tile per warp, a float4 of x per lane
  const int src = A.info->src_off;
  const float fsrc = A.wav[A.n] * A.info->src_fwd;
  const int rowc = (w + 4) * kHaloW + lane * 4;
  int gp = 0, gt = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile3 T = tile_of(t, gx, gy, A.zc, L.NZ);
    const int x0 = T.bx * kTileX + lane * 4, y = T.by * TY + w;
    const bool xok = x0 < L.NX4, yok = y < L.NY;
    const int col = L.origin + y * L.pitch + x0;
    const int nplanes = T.ze - T.zb;
    float4 q[9];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ok = ok && mbar_wait_ab(&fullP[(gp + j) % kRP], ((gp + j) / kRP) & 1, abort_blk);
      q[j] = lds4(sp + ((gp + j) % kRP) * kPStage + rowc + 4);
    }
    ok = __all_sync(0xffffffffu, ok);  // keep the warp's decision uniform
    if (lane == 0)
      for (int j = 0; j < 4; ++j) mbar_arrive(&emptyP[(gp + j) % kRP]);
#pragma unroll 4  // the z queue's shifts become register renames within an unrolled group
    for (int r = 0; ok && r < nplanes; ++r) {
      const int z = T.zb + r;
      const int top = gp + r + 8, cen = gp + r + 4, tk = gt + r;
      ok = mbar_wait_ab(&fullP[top % kRP], (top / kRP) & 1, abort_blk) &&
           mbar_wait_ab(&fullT[tk % kRT], (tk / kRT) & 1, abort_blk);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      q[8] = lds4(sp + (top % kRP) * kPStage + rowc + 4);
      if (xok && yok) {
        const float *tt = st + (tk % kRT) * 2 * kTTile + w * 128 + lane * 4;
        const float4 av = lds4(tt), po = lds4(tt + kTTile);
        float4 v = leap4_3d(sp + (cen % kRP) * kPStage + rowc, q, po, av);
        const int o = col + z * L.plane;
        const int d = src - o;
        if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * fsrc);
        st4(A.nxt + o, v);
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&emptyP[cen % kRP]);
        mbar_arrive(&emptyT[tk % kRT]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
    if (!ok) break;
    __syncwarp();
    if (lane == 0)
      for (int j = nplanes + 4; j < nplanes + 8; ++j) mbar_arrive(&emptyP[(gp + j) % kRP]);
    gp += nplanes + 8;
    gt += nplanes;
  }
}

// ------------------------------------------------------------- reverse ----
// 2 x kTY consumer warps: warps 0..kTY-1 advance p^R and accumulate the
// imaging integrals (reading pbar at the centre plane from the pbar ring),
// warps kTY..2kTY-1 advance pbar and then add the record at the receivers of
// their own row of the tile; the last warp produces.  P stage: the p^R and
// pbar halo planes; T stage: a, p^R and pbar tiles overwritten in place, and
// the num/den tiles where the tile meets the image box.
constexpr size_t kRevSmem =
    sizeof(float) * (2 * kRPr * kPStage + kRTr * 5 * kTTile) + 16 * (kRPr + kRTr) + 16;
static_assert(kRPr >= 8, "the P ring must hold a tile's first 8 planes");

__global__ void __launch_bounds__(32 * (2 * kTY + 1)) k_rev3d_tma(const __grid_constant__ CUtensorMap tm_rc,
                                                                   const __grid_constant__ CUtensorMap tm_bc,
                                                                   const __grid_constant__ CUtensorMap tm_a,
                                                                   const __grid_constant__ CUtensorMap tm_rn,
                                                                   const __grid_constant__ CUtensorMap tm_bn,
                                                                   const __grid_constant__ CUtensorMap tm_num,
                                                                   const __grid_constant__ CUtensorMap tm_den,
                                                                   const RevArgs A) {
  extern __shared__ __align__(128) float smem[];
  float *spr = smem;                        // [kRPr][kTY + 8][136]  p^R
  float *spb = spr + kRPr * kPStage;        // [kRPr][kTY + 8][136]  pbar
  float *st = spb + kRPr * kPStage;         // [kRTr][5][kTY][128]  a, p^R old, pbar old, num, den
  uint64_t *fullP = reinterpret_cast<uint64_t *>(st + kRTr * 5 * kTTile);
  uint64_t *emptyP = fullP + kRPr;
  uint64_t *fullT = emptyP + kRPr;
  uint64_t *emptyT = fullT + kRTr;
  volatile int *abort_blk = reinterpret_cast<volatile int *>(emptyT + kRTr);
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int gx = (L.NX + kTileX - 1) / kTileX, gy = (L.NY + kTY - 1) / kTY;
  const int ntiles = gx * gy * ((L.NZ + A.zc - 1) / A.zc);
  const bool do_r = A.do_r != 0, do_b = A.do_b != 0;
  if (tid == 0) {
    *abort_blk = 0;
    for (int s = 0; s < kRPr; ++s) mbar_init(&fullP[s], 1), mbar_init(&emptyP[s], 2 * kTY);
    for (int s = 0; s < kRTr; ++s) mbar_init(&fullT[s], 1), mbar_init(&emptyT[s], 2 * kTY);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (w == 2 * kTY) {
    if (lane == 0) {
      const uint32_t pbytes = 2 * sizeof(float) * kPStage;
      int gp = 0, gt = 0;
      bool ok = true;
      auto issueP = [&](int plane, int hx, int hy) {
        const int s = gp % kRPr, f = gp / kRPr;
        if (f > 0) ok = mbar_wait_ab(&emptyP[s], (f - 1) & 1, abort_blk);
        if (!ok) return;
        mbar_expect_tx(&fullP[s], pbytes);
        tma3(spr + s * kPStage, &tm_rc, hx, hy, plane + kHaloR, &fullP[s]);
        tma3(spb + s * kPStage, &tm_bc, hx, hy, plane + kHaloR, &fullP[s]);
        ++gp;
      };
      auto issueT = [&](int plane, int tx, int ty, bool tile_img) {
        const int s = gt % kRTr, f = gt / kRTr;
        if (f > 0) ok = mbar_wait_ab(&emptyT[s], (f - 1) & 1, abort_blk);
        if (!ok) return;
        const bool img = tile_img && plane >= A.iz0 && plane < A.iz1;
        mbar_expect_tx(&fullT[s], (img ? 5u : 3u) * sizeof(float) * kTTile);
        float *t5 = st + s * 5 * kTTile;
        tma3(t5, &tm_a, tx, ty, plane + kHaloR, &fullT[s]);
        tma3(t5 + kTTile, &tm_rn, tx, ty, plane + kHaloR, &fullT[s]);
        tma3(t5 + 2 * kTTile, &tm_bn, tx, ty, plane + kHaloR, &fullT[s]);
        if (img) {
          tma3(t5 + 3 * kTTile, &tm_num, tx, ty, plane + kHaloR, &fullT[s]);
          tma3(t5 + 4 * kTTile, &tm_den, tx, ty, plane + kHaloR, &fullT[s]);
        }
        ++gt;
      };
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        const Tile3 T = tile_of(t, gx, gy, A.zc, L.NZ);
        const int hx = T.bx * kTileX + kHaloX - 4, hy = T.by * kTY;
        const int tx = T.bx * kTileX + kHaloX, ty = T.by * kTY + kHaloR;
        // num/den tiles are streamed only where the tile meets the image box
        const bool tile_img = (T.by * kTY < A.iy1) && (T.by * kTY + kTY > A.iy0) && (T.bx * kTileX < A.ix1) &&
                              (T.bx * kTileX + kTileX > A.ix0);
        for (int i = 0; ok && i < 8; ++i) issueP(T.zb - 4 + i, hx, hy);
        for (int r = 0; ok && r < T.ze - T.zb; ++r) {
          issueP(T.zb + r + 4, hx, hy);
          if (ok) issueT(T.zb + r, tx, ty, tile_img);
        }
      }
      if (*abort_blk) {
        flag_error(A.err, 1);
        for (int k = max(0, gp - kRPr); k < gp; ++k) mbar_wait(&fullP[k % kRPr], (k / kRPr) & 1);
        for (int k = max(0, gt - kRTr); k < gt; ++k) mbar_wait(&fullT[k % kRTr], (k / kRTr) & 1);
      }
    }
    return;
  }
  const bool is_r = w < kTY;                // p^R group, else pbar group
  const int row = is_r ? w : w - kTY;
  const bool upd = is_r ? do_r : do_b;
  float *nxt = is_r ? A.rn : A.bn;
  const float *sp = is_r ? spr : spb;
  const int tslot = is_r ? 1 : 2;
  const int src = is_r ? A.info->src_off : -1;
  const float fsrc = (is_r && do_r) ? A.wav[A.n_src] * A.info->src_rev : 0.f;  // f[nt] does not exist
  const int rowc = (row + 4) * kHaloW + lane * 4;
  int gp = 0, gt = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile3 T = tile_of(t, gx, gy, A.zc, L.NZ);
    const int x0 = T.bx * kTileX + lane * 4, y = T.by * kTY + row;
    const bool xok = x0 < L.NX4, yok = y < L.NY;
    const bool img_xy = is_r && xok && yok && y >= A.iy0 && y < A.iy1 && x0 + 3 >= A.ix0 && x0 < A.ix1;
    const int col = L.origin + y * L.pitch + x0;
    const int nplanes = T.ze - T.zb;
    float4 q[9];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ok = ok && mbar_wait_ab(&fullP[(gp + j) % kRPr], ((gp + j) / kRPr) & 1, abort_blk);
      q[j] = lds4(sp + ((gp + j) % kRPr) * kPStage + rowc + 4);
    }
    ok = __all_sync(0xffffffffu, ok);  // keep the warp's decision uniform
    if (lane == 0)
      for (int j = 0; j < 4; ++j) mbar_arrive(&emptyP[(gp + j) % kRPr]);
    for (int r = 0; ok && r < nplanes; ++r) {
      const int z = T.zb + r;
      const int top = gp + r + 8, cen = gp + r + 4, tk = gt + r;
      ok = mbar_wait_ab(&fullP[top % kRPr], (top / kRPr) & 1, abort_blk) &&
           mbar_wait_ab(&fullT[tk % kRTr], (tk / kRTr) & 1, abort_blk);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      q[8] = lds4(sp + (top % kRPr) * kPStage + rowc + 4);
      if (xok && yok) {
        const int o = col + z * L.plane;
        const float *tt = st + (tk % kRTr) * 5 * kTTile + row * 128 + lane * 4;
        const float4 av = lds4(tt);
        const int cs = (cen % kRPr) * kPStage + rowc;
        if (upd) {
          float4 v = leap4_3d(sp + cs, q, lds4(tt + tslot * kTTile), av);
          const int d = src - o;
          if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * fsrc);
          st4(nxt + o, v);
        }
        if (img_xy && z >= A.iz0 && z < A.iz1) {
          const float4 b = lds4(spb + cs + 4);  // pbar_n at this node
          st4(A.num + o, add4(lds4(tt + 3 * kTTile), masked_prod(q[4], b, x0, A.ix0, A.ix1)));
          st4(A.den + o, add4(lds4(tt + 4 * kTTile), masked_prod(q[4], q[4], x0, A.ix0, A.ix1)));
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&emptyP[cen % kRPr]);
        mbar_arrive(&emptyT[tk % kRTr]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
    if (!ok) break;
    __syncwarp();
    if (lane == 0)
      for (int j = nplanes + 4; j < nplanes + 8; ++j) mbar_arrive(&emptyP[(gp + j) % kRPr]);
    gp += nplanes + 8;
    gt += nplanes;
    // Eq. 2 source term at this warp's receivers (its row of the tile), after
    // the warp's own stores of pbar_{n-1}
    if (!is_r && do_b) {
      const int cell = t * kTY + row;
      const int beg = A.tile_ptr[cell], end = A.tile_ptr[cell + 1];
      if (end > beg) {
        __threadfence();
        __syncwarp();
        const int nrec = A.info->nrec;
        const float sc = A.info->rec_scale;
        for (int k = beg + lane; k < end; k += 32) {
          const int rr = A.tile_rec[k];
          const int o = A.rec_off[rr];
          atomicAdd(A.bn + o, sc * A.a[o] * A.seis_t[(long long)A.n * nrec + rr]);
        }
      }
    }
  }
}

// ----------------------------------------------------------- host side ----
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map over one pitched field buffer: dims (pitch, rows, NZ + 8).
bool make_map(CUtensorMap *m, const Lay &L, const float *buf, int box_x, int box_y) {
  auto fn = encode_fn();
  if (!fn) return false;
  const float *base = buf + 0;  // buffer start (tensor coordinate 0 = padded -32, -4, -4)
  cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)(L.NZ + 2 * kHaloR)};
  cuuint64_t strides[2] = {(cuuint64_t)L.pitch * sizeof(float), (cuuint64_t)L.plane * sizeof(float)};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// One block per resident slot (at most one per tile).
int persistent_grid(const Lay &L, int zc, int ty, const void *fn, int threads, size_t smem) {
  const int ntiles = cdiv(L.NX, kTileX) * cdiv(L.NY, ty) * cdiv(L.NZ, zc);
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  const int slots = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  return ntiles < slots ? ntiles : slots;
}

} // namespace

void *tmap_encode_fn() { return reinterpret_cast<void *>(encode_fn()); }

int tile_rows_3d() { return kTY; }

// z planes per tile of the 3-D kernels for this grid: with one persistent
// block per SM, the busiest block streams ceil(tiles / SMs) tiles of zc + 8
// planes each (8 halo planes per tile), so take the chunking that minimises
// that product (on 580 x 580 x 380: 95 planes forward, 190 reverse).
int zc_for_3d(const Lay &L, bool fwd) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const long long per = (long long)cdiv(L.NX, kTileX) * cdiv(L.NY, fwd ? RBC_FWD3D_ROWS : kTY);
  int best = k3dZC;
  long long best_cost = -1;
  for (int c = 1; c <= cdiv(L.NZ, 16); ++c) {
    const int zc = cdiv(L.NZ, c);
    const long long cost = ((per * c + sms - 1) / sms) * (zc + 8);
    if (best_cost < 0 || cost < best_cost) best_cost = cost, best = zc;
  }
  return best;
}

// The pitched buffers start at their allocation; tensor coordinates are the
// padded node plus (32, 4, 4).  Field pointers passed in StepArgs/RevArgs are
// buffer starts (the kernels add L.origin for plain loads and stores).
bool launch_fwd3d(const StepArgs &A, cudaStream_t s) {
  constexpr int TY = kTYf;
  constexpr size_t smem = fwd_smem<TY>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fwd3d_tma<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  CUtensorMap mc, ma, mo;
  if (!make_map(&mc, A.L, A.cur, kHaloW, TY + 8) || !make_map(&ma, A.L, A.a, kTileX, TY) ||
      !make_map(&mo, A.L, A.nxt, kTileX, TY))
    return false;
  k_fwd3d_tma<TY><<<persistent_grid(A.L, A.zc, TY, (const void *)k_fwd3d_tma<TY>, 32 * (TY + 1), smem),
                    dim3(32, TY + 1), smem, s>>>(mc, ma, mo, A);
  return true;
}

bool launch_rev3d(const RevArgs &A, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rev3d_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRevSmem);
    attr = true;
  }
  CUtensorMap mr, mb, ma, mrn, mbn, mnum, mden;
  if (!make_map(&mr, A.L, A.rc, kHaloW, kTY + 8) || !make_map(&mb, A.L, A.bc, kHaloW, kTY + 8) ||
      !make_map(&ma, A.L, A.a, kTileX, kTY) || !make_map(&mrn, A.L, A.rn, kTileX, kTY) ||
      !make_map(&mbn, A.L, A.bn, kTileX, kTY) || !make_map(&mnum, A.L, A.num, kTileX, kTY) ||
      !make_map(&mden, A.L, A.den, kTileX, kTY))
    return false;
  k_rev3d_tma<<<persistent_grid(A.L, A.zc, kTY, (const void *)k_rev3d_tma, 32 * (2 * kTY + 1), kRevSmem),
                dim3(32, 2 * kTY + 1), kRevSmem, s>>>(mr, mb, ma, mrn, mbn, mnum, mden, A);
  return true;
}

} // namespace rbc
