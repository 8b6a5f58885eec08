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

constexpr int kTY = 8;        // y rows per block (one warp each)
constexpr int kRP = 8;        // forward P ring: 5 live planes + 3 in flight
constexpr int kRT = 5;        // forward T ring: 1 live plane + 4 in flight
constexpr int kRPr = 7;       // reverse P ring (two fields): 5 live + 2 in flight
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
__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
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

// ------------------------------------------------------------- forward ----
// Shared memory: P ring (kRP stages of one halo plane), T ring (kRT stages of
// a and p^{n-1} tiles), barriers.
constexpr size_t kFwdSmem = sizeof(float) * (kRP * kPStage + kRT * 2 * kTTile) + 8 * (kRP + kRT) + 16;

__global__ void __launch_bounds__(32 * kTY) k_fwd3d_tma(const __grid_constant__ CUtensorMap tm_cur,
                                                         const __grid_constant__ CUtensorMap tm_a,
                                                         const __grid_constant__ CUtensorMap tm_old,
                                                         const StepArgs A) {
  extern __shared__ __align__(128) float smem[];
  float *sp = smem;                         // [kRP][kTY + 8][136]
  float *st = sp + kRP * kPStage;           // [kRT][2][kTY][128]  (a, old)
  uint64_t *barP = reinterpret_cast<uint64_t *>(st + kRT * 2 * kTTile);
  uint64_t *barT = barP + kRP;
  int &abort_blk = *reinterpret_cast<int *>(barT + kRT);
  int armP[kRP], armT[kRT];  // phases armed per stage (thread 0 only)
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int bx = blockIdx.x, by = blockIdx.y;
  const int x0 = bx * kTileX + lane * 4, y = by * kTY + w;
  const int zb = blockIdx.z * A.zc, ze = min(zb + A.zc, L.NZ);
  const bool xok = x0 < L.NX4, yok = y < L.NY;
  if (A.sample) {
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int bid = (blockIdx.z * gridDim.y + by) * gridDim.x + bx;
    const int nrec = A.info->nrec;
    for (int r = bid * blockDim.x * blockDim.y + tid; r < nrec; r += nb * blockDim.x * blockDim.y)
      A.seis_t[(long long)A.n * nrec + r] = A.cur[A.rec_off[r]];
  }
  // tensor-map coordinates: padded node (x, y, z) -> (x + 32, y + 4, z + 4)
  const int hx = bx * kTileX + kHaloX - 4, hy = by * kTY;        // halo box origin
  const int tx = bx * kTileX + kHaloX, ty = by * kTY + kHaloR;   // tile box origin
  const uint32_t pbytes = sizeof(float) * kPStage, tbytes = sizeof(float) * 2 * kTTile;
  for (int s = 0; s < kRP; ++s) armP[s] = 0;
  for (int s = 0; s < kRT; ++s) armT[s] = 0;
  if (tid == 0) {
    abort_blk = 0;
    for (int s = 0; s < kRP; ++s) mbar_init(&barP[s], 1);
    for (int s = 0; s < kRT; ++s) mbar_init(&barT[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int last_p = ze + 3;  // last plane pushed onto a queue
  if (tid == 0) {
    for (int r = 0; r < kRP && zb + r <= last_p; ++r) {
      mbar_expect_tx(&barP[r], pbytes);
        ++armP[r];
      tma3(sp + r * kPStage, &tm_cur, hx, hy, zb + r + kHaloR, &barP[r]);
    }
    for (int r = 0; r < kRT && zb + r < ze; ++r) {
      mbar_expect_tx(&barT[r], tbytes);
        ++armT[r];
      tma3(st + r * 2 * kTTile, &tm_a, tx, ty, zb + r + kHaloR, &barT[r]);
      tma3(st + r * 2 * kTTile + kTTile, &tm_old, tx, ty, zb + r + kHaloR, &barT[r]);
    }
  }
  // z queue: planes zb-4 .. zb-1 straight from global, zb .. zb+3 from the ring
  float4 q[9];
  const int col = L.origin + y * L.pitch + x0;
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = (xok && zb - 4 + j >= -kHaloR) ? ldg4(A.cur + col + (zb - 4 + j) * L.plane) : zero4();
  bool ok = true;
  const int rowc = (w + 4) * kHaloW + lane * 4;  // this thread's halo-row float offset
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (zb + j <= last_p) {
      ok = mbar_wait(&barP[j], 0) && ok;
      q[4 + j] = lds4(sp + j * kPStage + rowc + 4);
    } else {
      q[4 + j] = zero4();
    }
  }
  const int src = A.info->src_off;
  const float fsrc = A.wav[A.n] * A.info->src_fwd;
  for (int z = zb; z < ze; ++z) {
    const int r = z - zb;
    const int rp = (r + 4) % kRP;
    ok = mbar_wait(&barP[rp], ((r + 4) / kRP) & 1) && ok;
    q[8] = lds4(sp + rp * kPStage + rowc + 4);
    ok = mbar_wait(&barT[r % kRT], (r / kRT) & 1) && ok;
    if (xok && yok) {
      const float *tt = st + (r % kRT) * 2 * kTTile + w * 128 + lane * 4;
      const float4 av = lds4(tt), po = lds4(tt + kTTile);
      float4 v = leap4_3d(sp + (r % kRP) * kPStage + rowc, q, po, av);
      const int o = col + z * L.plane;
      const int d = src - o;
      if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * fsrc);
      st4(A.nxt + o, v);
    }
    if (!ok) abort_blk = 1;
    __syncthreads();
    if (abort_blk) break;
    if (tid == 0) {
      const int np = z + kRP;  // refill the stage of plane z
      if (np <= last_p) {
        const int s = r % kRP;
        mbar_expect_tx(&barP[s], pbytes);
        ++armP[s];
        tma3(sp + s * kPStage, &tm_cur, hx, hy, np + kHaloR, &barP[s]);
      }
      const int nt_ = z + kRT;
      if (nt_ < ze) {
        const int s = r % kRT;
        mbar_expect_tx(&barT[s], tbytes);
        ++armT[s];
        tma3(st + s * 2 * kTTile, &tm_a, tx, ty, nt_ + kHaloR, &barT[s]);
        tma3(st + s * 2 * kTTile + kTTile, &tm_old, tx, ty, nt_ + kHaloR, &barT[s]);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
  }
  if (abort_blk && tid == 0) {
    flag_error(A.err, 1);
    // let every copy already issued land before the block's shared memory is released
    for (int s = 0; s < kRP; ++s)
      if (armP[s]) mbar_wait(&barP[s], (armP[s] - 1) & 1);
    for (int s = 0; s < kRT; ++s)
      if (armT[s]) mbar_wait(&barT[s], (armT[s] - 1) & 1);
  }
}

// ------------------------------------------------------------- reverse ----
// Two fields: P rings for p^R and pbar halo planes; T ring for the a, p^R and
// pbar tiles overwritten in place and the num/den tiles (loaded only where the
// tile meets the image box).
constexpr size_t kRevSmem = sizeof(float) * (2 * kRPr * kPStage + kRTr * 5 * kTTile) + 8 * (kRPr + kRTr) + 16;

__global__ void __launch_bounds__(32 * kTY) k_rev3d_tma(const __grid_constant__ CUtensorMap tm_rc,
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
  uint64_t *barP = reinterpret_cast<uint64_t *>(st + kRTr * 5 * kTTile);
  uint64_t *barT = barP + kRPr;
  int &abort_blk = *reinterpret_cast<int *>(barT + kRTr);
  int armP[kRPr], armT[kRTr];
  const Lay &L = A.L;
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const int bx = blockIdx.x, by = blockIdx.y;
  const int x0 = bx * kTileX + lane * 4, y = by * kTY + w;
  const int zb = blockIdx.z * A.zc, ze = min(zb + A.zc, L.NZ);
  const bool xok = x0 < L.NX4, yok = y < L.NY;
  const bool do_r = A.do_r != 0, do_b = A.do_b != 0;
  const bool img_xy = xok && yok && y >= A.iy0 && y < A.iy1 && x0 + 3 >= A.ix0 && x0 < A.ix1;
  const int hx = bx * kTileX + kHaloX - 4, hy = by * kTY;
  const int tx = bx * kTileX + kHaloX, ty = by * kTY + kHaloR;
  const uint32_t pbytes = 2 * sizeof(float) * kPStage;
  // num/den tiles are streamed only for planes and tiles that meet the image box
  const bool tile_img = (by * kTY < A.iy1) && (by * kTY + kTY > A.iy0) && (bx * kTileX < A.ix1) &&
                        (bx * kTileX + kTileX > A.ix0);
  auto tbytes_of = [&](int plane) -> uint32_t {
    const bool img = tile_img && plane >= A.iz0 && plane < A.iz1;
    return (img ? 5u : 3u) * sizeof(float) * kTTile;
  };
  for (int s = 0; s < kRPr; ++s) armP[s] = 0;
  for (int s = 0; s < kRTr; ++s) armT[s] = 0;
  if (tid == 0) {
    abort_blk = 0;
    for (int s = 0; s < kRPr; ++s) mbar_init(&barP[s], 1);
    for (int s = 0; s < kRTr; ++s) mbar_init(&barT[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int last_p = ze + 3;
  if (tid == 0) {
    for (int r = 0; r < kRPr && zb + r <= last_p; ++r) {
      mbar_expect_tx(&barP[r], pbytes);
        ++armP[r];
      tma3(spr + r * kPStage, &tm_rc, hx, hy, zb + r + kHaloR, &barP[r]);
      tma3(spb + r * kPStage, &tm_bc, hx, hy, zb + r + kHaloR, &barP[r]);
    }
    for (int r = 0; r < kRTr && zb + r < ze; ++r) {
      const uint32_t tb = tbytes_of(zb + r);
      mbar_expect_tx(&barT[r], tb);
      ++armT[r];
      float *t = st + r * 5 * kTTile;
      tma3(t, &tm_a, tx, ty, zb + r + kHaloR, &barT[r]);
      tma3(t + kTTile, &tm_rn, tx, ty, zb + r + kHaloR, &barT[r]);
      tma3(t + 2 * kTTile, &tm_bn, tx, ty, zb + r + kHaloR, &barT[r]);
      if (tb > 3u * sizeof(float) * kTTile) {
        tma3(t + 3 * kTTile, &tm_num, tx, ty, zb + r + kHaloR, &barT[r]);
        tma3(t + 4 * kTTile, &tm_den, tx, ty, zb + r + kHaloR, &barT[r]);
      }
    }
  }
  float4 qr[9], qb[9];
  const int col = L.origin + y * L.pitch + x0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool in = xok && zb - 4 + j >= -kHaloR;
    qr[j] = in ? ldg4(A.rc + col + (zb - 4 + j) * L.plane) : zero4();
    qb[j] = in ? ldg4(A.bc + col + (zb - 4 + j) * L.plane) : zero4();
  }
  bool ok = true;
  const int rowc = (w + 4) * kHaloW + lane * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (zb + j <= last_p) {
      ok = mbar_wait(&barP[j], 0) && ok;
      qr[4 + j] = lds4(spr + j * kPStage + rowc + 4);
      qb[4 + j] = lds4(spb + j * kPStage + rowc + 4);
    } else {
      qr[4 + j] = zero4();
      qb[4 + j] = zero4();
    }
  }
  const int src = A.info->src_off;
  const float fsrc = do_r ? A.wav[A.n] * A.info->src_rev : 0.f;  // f[nt] does not exist
  for (int z = zb; z < ze; ++z) {
    const int r = z - zb;
    const int rp = (r + 4) % kRPr;
    ok = mbar_wait(&barP[rp], ((r + 4) / kRPr) & 1) && ok;
    qr[8] = lds4(spr + rp * kPStage + rowc + 4);
    qb[8] = lds4(spb + rp * kPStage + rowc + 4);
    ok = mbar_wait(&barT[r % kRTr], (r / kRTr) & 1) && ok;
    if (xok && yok) {
      const int o = col + z * L.plane;
      const float *tt = st + (r % kRTr) * 5 * kTTile + w * 128 + lane * 4;
      const float4 av = lds4(tt);
      const int sc = (r % kRPr) * kPStage + rowc;
      if (do_r) {
        float4 v = leap4_3d(spr + sc, qr, lds4(tt + kTTile), av);
        const int d = src - o;
        if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * fsrc);
        st4(A.rn + o, v);
      }
      if (do_b) st4(A.bn + o, leap4_3d(spb + sc, qb, lds4(tt + 2 * kTTile), av));
      if (img_xy && z >= A.iz0 && z < A.iz1) {
        st4(A.num + o, add4(lds4(tt + 3 * kTTile), masked_prod(qr[4], qb[4], x0, A.ix0, A.ix1)));
        st4(A.den + o, add4(lds4(tt + 4 * kTTile), masked_prod(qr[4], qr[4], x0, A.ix0, A.ix1)));
      }
    }
    if (!ok) abort_blk = 1;
    __syncthreads();
    if (abort_blk) break;
    if (tid == 0) {
      const int np = z + kRPr;
      if (np <= last_p) {
        const int s = r % kRPr;
        mbar_expect_tx(&barP[s], pbytes);
        ++armP[s];
        tma3(spr + s * kPStage, &tm_rc, hx, hy, np + kHaloR, &barP[s]);
        tma3(spb + s * kPStage, &tm_bc, hx, hy, np + kHaloR, &barP[s]);
      }
      const int nt_ = z + kRTr;
      if (nt_ < ze) {
        const int s = r % kRTr;
        float *t = st + s * 5 * kTTile;
        const uint32_t tb = tbytes_of(nt_);
        mbar_expect_tx(&barT[s], tb);
        ++armT[s];
        tma3(t, &tm_a, tx, ty, nt_ + kHaloR, &barT[s]);
        tma3(t + kTTile, &tm_rn, tx, ty, nt_ + kHaloR, &barT[s]);
        tma3(t + 2 * kTTile, &tm_bn, tx, ty, nt_ + kHaloR, &barT[s]);
        if (tb > 3u * sizeof(float) * kTTile) {
          tma3(t + 3 * kTTile, &tm_num, tx, ty, nt_ + kHaloR, &barT[s]);
          tma3(t + 4 * kTTile, &tm_den, tx, ty, nt_ + kHaloR, &barT[s]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      qr[k] = qr[k + 1];
      qb[k] = qb[k + 1];
    }
  }
  if (abort_blk && tid == 0) {
    flag_error(A.err, 1);
    for (int s = 0; s < kRPr; ++s)
      if (armP[s]) mbar_wait(&barP[s], (armP[s] - 1) & 1);
    for (int s = 0; s < kRTr; ++s)
      if (armT[s]) mbar_wait(&barT[s], (armT[s] - 1) & 1);
  }
  // receivers of this tile (Eq. 2 source term) after the block's stores
  if (do_b) {
    const int bid = (blockIdx.z * gridDim.y + by) * gridDim.x + bx;
    const int beg = A.tile_ptr[bid], end = A.tile_ptr[bid + 1];
    if (end > beg) {
      __threadfence();
      __syncthreads();
      const int nrec = A.info->nrec;
      const float sc = A.info->rec_scale;
      for (int k = beg + tid; k < end; k += blockDim.x * blockDim.y) {
        const int rr = A.tile_rec[k];
        const int o = A.rec_off[rr];
        atomicAdd(A.bn + o, sc * A.a[o] * A.seis_t[(long long)A.n * nrec + rr]);
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

} // namespace

int tile_rows_3d() { return kTY; }

// The pitched buffers start at their allocation; tensor coordinates are the
// padded node plus (32, 4, 4).  Field pointers passed in StepArgs/RevArgs are
// buffer starts (the kernels add L.origin for plain loads and stores).
bool launch_fwd3d(const StepArgs &A, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fwd3d_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    attr = true;
  }
  CUtensorMap mc, ma, mo;
  if (!make_map(&mc, A.L, A.cur, kHaloW, kTY + 8) || !make_map(&ma, A.L, A.a, kTileX, kTY) ||
      !make_map(&mo, A.L, A.nxt, kTileX, kTY))
    return false;
  dim3 grid(cdiv(A.L.NX, kTileX), cdiv(A.L.NY, kTY), cdiv(A.L.NZ, A.zc));
  k_fwd3d_tma<<<grid, dim3(32, kTY), kFwdSmem, s>>>(mc, ma, mo, A);
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
  dim3 grid(cdiv(A.L.NX, kTileX), cdiv(A.L.NY, kTY), cdiv(A.L.NZ, A.zc));
  k_rev3d_tma<<<grid, dim3(32, kTY), kRevSmem, s>>>(mr, mb, ma, mrn, mbn, mnum, mden, A);
  return true;
}

} // namespace rbc
