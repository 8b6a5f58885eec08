// rbc_batch.cu -- RTM of many 2-D shots with uneven apertures in one launch
// per time step (Algorithm 3's shot loop folded into the grid).
//
// Every shot keeps its own padded grid (its aperture window plus the random
// boundary) in the pitched, zero-haloed layout; all grids share nz, nb, h,
// dt and nt.  One kernel launch per time step walks a work list of (shot,
// tile) items with persistent blocks, so shots of any width share the
// machine without a tail per shot; the shot descriptors live in device
// memory.  The shots run in groups of consecutive shots whose fields fit in
// L2 (each group's whole forward loop, then its whole reverse loop, over the
// group's contiguous range of the work list), and every group's two loops
// are CUDA graphs replayed for every batch.  Rows per warp of the forward
// and reverse kernels are chosen at creation by timing the candidates on the
// first group.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/rbc.h"
#include "rbc_tile2d.cuh"

using namespace rbc;

namespace rbc {
int set_error(int code, const char *msg);  // rbc_abi.cu
void add_launches(long long n);            // rbc_abi.cu
}

namespace {

struct BShot {
  Lay L;
  float *a, *p0, *p1, *q0, *q1, *num, *den;
  int src_off;
  int nrec;
  const int *rec_off;   // receiver offsets in this shot's layout
  const int *tile_ptr;  // receivers of each reverse tile (CSR, local tiles)
  const int *tile_rec;
  const float *seis_t;  // [nt+1][nrec]
  int gx, gzf, gzr;     // x tiles, z tiles of the forward / reverse kernels
  int tbase_f, tbase_r; // first global work item of this shot
  int ix0, ix1, iz0, iz1;
  int off_x;            // survey column of this shot's interior x = 0
  unsigned int maxbits; // max(den) of the shot (image ratio)
};

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// warps per block of the tiled forward kernel (the single-shot forward kernel
// runs 4 as well; the reverse and streaming kernels run k2dWarps)
constexpr int kBWarpsF = 4;

// ---------------------------------------------------------------- kernels --
template <int RZ>
__global__ void __launch_bounds__(32 * kBWarpsF) k_fwd2d_batch(const BShot *__restrict__ shots,
                                                                const int *__restrict__ item_shot, int item0,
                                                                int item1, int n, const float *__restrict__ wav,
                                                                float src_scale) {
  const int lane = threadIdx.x, w = threadIdx.y;
  griddep_wait();
  const float f = wav[n] * src_scale;
  // the next item's shot index is fetched one item ahead
  int sh = item0 + (int)blockIdx.x < item1 ? __ldg(item_shot + item0 + blockIdx.x) : 0;
  for (int t = item0 + blockIdx.x; t < item1; t += gridDim.x) {
    const BShot &S = shots[sh];
    sh = t + (int)gridDim.x < item1 ? __ldg(item_shot + t + gridDim.x) : 0;
    const int loc = t - S.tbase_f;
    const int bx = loc % S.gx, bz = loc / S.gx;
    const int zb = (bz * kBWarpsF + w) * RZ;
    if (zb >= S.L.NZ) continue;  // warp-uniform
    const float *cur = (n & 1) ? S.p1 : S.p0;
    float *nxt = (n & 1) ? S.p0 : S.p1;
    fwd2d_rows<RZ>(S.L, S.a, cur, nxt, lane, bx * kTileX + lane * 4, zb, S.src_off, f);
  }
  griddep_launch();
}

template <int RZ>
__global__ void __launch_bounds__(32 * k2dWarps) k_rev2d_batch(const BShot *__restrict__ shots,
                                                                const int *__restrict__ item_shot, int item0,
                                                                int item1, int n, int nt, const float *__restrict__ wav,
                                                                float src_scale, float rec_scale) {
  const int lane = threadIdx.x, w = threadIdx.y;
  const bool do_r = n < nt && n > 0, do_b = n > 0;
  griddep_wait();
  const float fsrc = do_r ? wav[n] * src_scale : 0.f;  // f[nt] does not exist
  int sh = item0 + (int)blockIdx.x < item1 ? __ldg(item_shot + item0 + blockIdx.x) : 0;
  for (int t = item0 + blockIdx.x; t < item1; t += gridDim.x) {
    const BShot &S = shots[sh];
    sh = t + (int)gridDim.x < item1 ? __ldg(item_shot + t + gridDim.x) : 0;
    const Lay &L = S.L;
    const int loc = t - S.tbase_r;
    const int bx = loc % S.gx, bz = loc / S.gx;
    const int x0 = bx * kTileX + lane * 4;
    const int zb = (bz * k2dWarps + w) * RZ;
    const bool xok = x0 < L.NX4;
    // p^R_n in p[n & 1], pbar_n in q[n & 1]
    const float *rc = (n & 1) ? S.p1 : S.p0;
    float *rn = (n & 1) ? S.p0 : S.p1;
    const float *bc = (n & 1) ? S.q1 : S.q0;
    float *bn = (n & 1) ? S.q0 : S.q1;
    if (zb < L.NZ) {  // warp-uniform
      float4 cr[RZ], cb[RZ], inc[RZ];
      rev_field2d<RZ, false>(L, S.a, rc, rn, do_r, lane, x0, zb, xok, S.src_off, fsrc, cr, inc);
      rev_field2d<RZ, false>(L, S.a, bc, bn, do_b, lane, x0, zb, xok, -1, 0.f, cb, inc);
      if (xok && x0 + 3 >= S.ix0 && x0 < S.ix1) {
#pragma unroll
        for (int j = 0; j < RZ; ++j) {
          const int z = zb + j;
          if (z >= S.iz0 && z < S.iz1) {
            const int o = L.origin + x0 + z * L.pitch;
            st4(S.num + o, add4(ld4(S.num + o), masked_prod(cr[j], cb[j], x0, S.ix0, S.ix1)));
            st4(S.den + o, add4(ld4(S.den + o), masked_prod(cr[j], cr[j], x0, S.ix0, S.ix1)));
          }
        }
      }
    }
    // Eq. 2 source term at this tile's receivers, after the block's stores
    if (do_b) {
      const int beg = S.tile_ptr[loc], end = S.tile_ptr[loc + 1];
      if (end > beg) {
        __threadfence();
        __syncthreads();
        for (int k = beg + w * 32 + lane; k < end; k += 32 * k2dWarps) {
          const int r = S.tile_rec[k];
          const int o = S.rec_off[r];
          atomicAdd(bn + o, rec_scale * S.a[o] * S.seis_t[(long long)n * S.nrec + r]);
        }
        __syncthreads();
      }
    }
  }
  griddep_launch();
}

// Tiled form of the fused reverse step: one block of 4 warps per work item of
// 128 columns x 16 rows (4 per warp), non-persistent (a grid of the items of
// up to kBGMax consecutive shots), with the current levels of both fields
// over the item and its halo and the item's imaging accumulators staged in
// shared memory by cp.async before a single barrier, as in the single-shot
// k_rev2d_tile.  What a block needs before it can stage (the shots' layouts,
// field pointers, tile counts and image boxes, which stay fixed for the life
// of the batch) is a kernel parameter: the item's shot is found from the
// shots' first items, with no dependent loads from global memory; the
// per-call part (source offset, receivers, records) is read from the shot
// descriptors in global memory, the source offset before the wait for the
// previous step.
constexpr int kBTileW = 4, kBTileRZ = 4, kBTileT = kBTileW * kBTileRZ;
constexpr int kBGMax = 16;  // shots per launch of the tiled reverse
struct BRevShot {
  Lay L;
  float *a, *p0, *p1, *q0, *q1, *num, *den;
  int gx, ix0, ix1, iz0, iz1;
};
struct BRevGroup {
  int nshot, shot0;           // shots shot0 .. shot0 + nshot - 1 of the batch
  int tbase[kBGMax + 1];      // first item of each shot in this launch, then the item count
  BRevShot s[kBGMax];
};
__global__ void __launch_bounds__(32 * kBTileW, 5) k_rev2d_batch_tile(const __grid_constant__ BRevGroup G,
                                                                      const BShot *__restrict__ shots, int n, int nt,
                                                                      const float *__restrict__ wav, float src_scale,
                                                                      float rec_scale) {
  constexpr int T = kBTileT, RZ = kBTileRZ;
  __shared__ __align__(16) float s_r[(T + 8) * kStRow], s_b[(T + 8) * kStRow];
  __shared__ __align__(16) float s_num[T * kTileX], s_den[T * kTileX];
  const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
  const bool do_r = n < nt && n > 0, do_b = n > 0;
  const int t = blockIdx.x;
  int si = 0;
  while (si + 1 < G.nshot && t >= G.tbase[si + 1]) ++si;
  const BRevShot &S = G.s[si];
  const BShot &D = shots[G.shot0 + si];
  const int src = D.src_off;  // in flight during the wait
  const Lay &L = S.L;
  const int loc = t - G.tbase[si];
  const int X0 = (loc % S.gx) * kTileX, Z0 = (loc / S.gx) * T;
  const int x0 = X0 + lane * 4, zb = Z0 + w * RZ;
  const bool xok = x0 < L.NX4;
  // p^R_n in p[n & 1], pbar_n in q[n & 1]
  const float *rc = (n & 1) ? S.p1 : S.p0;
  float *rn = (n & 1) ? S.p0 : S.p1;
  const float *bc = (n & 1) ? S.q1 : S.q0;
  float *bn = (n & 1) ? S.q0 : S.q1;
  const bool img_tile = Z0 < S.iz1 && Z0 + T > S.iz0 && X0 < S.ix1 && X0 + kTileX > S.ix0;
  griddep_wait();
  stage_rows<T>(L, rc, s_r, X0, Z0, tid, 32 * kBTileW);
  stage_rows<T>(L, bc, s_b, X0, Z0, tid, 32 * kBTileW);
  if (img_tile) {
    stage_own<T>(L, S.num, s_num, X0, Z0, tid, 32 * kBTileW);
    stage_own<T>(L, S.den, s_den, X0, Z0, tid, 32 * kBTileW);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  float4 av[RZ], pr[RZ], pb[RZ];
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int o = L.origin + x0 + (zb + j) * L.pitch;
    const bool ok = xok && zb + j < L.NZ;
    av[j] = ok ? ldg4(S.a + o) : zero4();
    pr[j] = ok && do_r ? ld4(rn + o) : zero4();
    pb[j] = ok && do_b ? ld4(bn + o) : zero4();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const float fsrc = do_r ? wav[n] * src_scale : 0.f;  // f[nt] does not exist
  const bool img = xok && x0 + 3 >= S.ix0 && x0 < S.ix1;
#pragma unroll
  for (int j = 0; j < RZ; ++j) {
    const int z = zb + j, rr = w * RZ + j + kHaloR;
    if (!(xok && z < L.NZ)) continue;
    const int o = L.origin + x0 + z * L.pitch;
    float4 cr = staged_c(s_r, rr, lane), cb = staged_c(s_b, rr, lane);
    if (do_r) {
      // Eq. 6: reconstruction (exact inverse of the forward step)
      float4 r = leap_staged(s_r, rr, lane, pr[j], av[j], &cr);
      const int d = src - o;
      if ((unsigned)d < 4u) point_sub(r, d, cmp(av[j], d) * fsrc);
      st4(rn + o, r);
    }
    // Eq. 2: the record is added below, after the block's stores
    if (do_b) st4(bn + o, leap_staged(s_b, rr, lane, pb[j], av[j], &cb));
    if (img && z >= S.iz0 && z < S.iz1) {
      const int so = (w * RZ + j) * kTileX + 4 * lane;
      st4(S.num + o, add4(ld4(s_num + so), masked_prod(cr, cb, x0, S.ix0, S.ix1)));
      st4(S.den + o, add4(ld4(s_den + so), masked_prod(cr, cr, x0, S.ix0, S.ix1)));
    }
  }
  // Eq. 2 source term at this item's receivers, after the block's stores
  if (do_b) {
    const int beg = D.tile_ptr[loc], end = D.tile_ptr[loc + 1];
    if (end > beg) {
      __threadfence();
      __syncthreads();
      for (int k = beg + tid; k < end; k += 32 * kBTileW) {
        const int r = D.tile_rec[k];
        const int o = D.rec_off[r];
        atomicAdd(bn + o, rec_scale * S.a[o] * D.seis_t[(long long)n * D.nrec + r]);
      }
    }
  }
  griddep_launch();
}

// Streaming form of the forward step for DRAM-bound batches: every warp owns
// a 128-column strip of kSZ rows of one shot and keeps its own rings in
// shared memory -- kSR rows of p^n (with the 4-column halo, 544 bytes each)
// and kSA rows of a and p^{n-1} -- filled by bulk asynchronous copies
// (cp.async.bulk, completion counted on one mbarrier per ring slot) up to
// kSR rows ahead of the row being computed.  Loads are in flight while the
// warp computes, where the register-queue kernels wait on them; the x and z
// neighbours come from the ring.  Every wait is bounded.
constexpr int kSZ = 64, kSR = 12, kSA = 4;
constexpr int kSRow = kTileX + 8;                             // 136 floats: x0-4 .. x0+131
constexpr int kSWarp = kSR * kSRow + 2 * kSA * kTileX;        // floats per warp
constexpr size_t kStreamSmem = sizeof(float) * kSWarp * k2dWarps + sizeof(uint64_t) * (kSR + kSA) * k2dWarps;
constexpr long long kSWait = 2000000000LL;                    // about a second

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool s_try(uint64_t *b, uint32_t par) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(s_addr(b)), "r"(par) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool s_wait(uint64_t *b, uint32_t par) {
  if (s_try(b, par)) return true;
  const long long t0 = clock64();
  while (!s_try(b, par))
    if (clock64() - t0 > kSWait) return false;
  return true;
}
__device__ __forceinline__ void s_copy(float *dst, const float *src, uint32_t bytes, uint64_t *b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s_addr(dst)), "l"(src), "r"(bytes), "r"(s_addr(b))
               : "memory");
}
__device__ __forceinline__ void s_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(32 * k2dWarps) k_fwd2d_stream(const BShot *__restrict__ shots,
                                                                 const int *__restrict__ item_shot, int item0,
                                                                 int item1, int n, const float *__restrict__ wav,
                                                                 float src_scale, int *err) {
  extern __shared__ __align__(128) float sm_s[];
  const int lane = threadIdx.x, w = threadIdx.y;
  float *rc = sm_s + w * kSWarp;       // [kSR][kSRow]  p^n
  float *ra = rc + kSR * kSRow;        // [kSA][128]    a
  float *rp = ra + kSA * kTileX;       // [kSA][128]    p^{n-1}
  uint64_t *bc = reinterpret_cast<uint64_t *>(sm_s + k2dWarps * kSWarp) + w * (kSR + kSA);
  uint64_t *ba = bc + kSR;
  if (lane == 0) {
    for (int i = 0; i < kSR + kSA; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bc + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  griddep_wait();
  const float f = wav[n] * src_scale;
  int gc = 0, ga = 0;  // copies issued so far into the p^n / (a, p^{n-1}) rings
  bool ok = true;
  for (int t = item0 + blockIdx.x * k2dWarps + w; ok && t < item1; t += gridDim.x * k2dWarps) {
    const BShot &S = shots[item_shot[t]];
    const Lay &L = S.L;
    const int loc = t - S.tbase_f;
    const int x0 = (loc % S.gx) * kTileX, zb = (loc / S.gx) * kSZ;
    const int nrow = min(kSZ, L.NZ - zb);
    const float *cur = (n & 1) ? S.p1 : S.p0;
    float *nxt = (n & 1) ? S.p0 : S.p1;
    const int c0 = gc, a0 = ga;
    // p^n rows zb-4 .. zb+nrow+3 (task index i = row - zb + 4); a, p^{n-1} rows zb .. zb+nrow-1
    auto issue_c = [&](int i) {
      const int q = c0 + i;
      uint64_t *b = bc + q % kSR;
      s_expect(b, kSRow * 4);
      s_copy(rc + (q % kSR) * kSRow, cur + L.origin + (zb - 4 + i) * L.pitch + x0 - 4, kSRow * 4, b);
    };
    auto issue_a = [&](int i) {
      const int q = a0 + i;
      uint64_t *b = ba + q % kSA;
      const int o = L.origin + (zb + i) * L.pitch + x0;
      s_expect(b, 2 * kTileX * 4);
      s_copy(ra + (q % kSA) * kTileX, S.a + o, kTileX * 4, b);
      s_copy(rp + (q % kSA) * kTileX, nxt + o, kTileX * 4, b);
    };
    if (lane == 0) {
      for (int i = 0; i < min(kSR, nrow + 8); ++i) issue_c(i);
      for (int i = 0; i < min(kSA, nrow); ++i) issue_a(i);
    }
    int waited_c = 0, waited_a = 0;  // rows of this task already seen complete
    const int xl = x0 + lane * 4;
    int r = 0;
    for (; r < nrow; ++r) {
      while (ok && waited_c <= r + 8) {
        const int q = c0 + waited_c;
        ok = s_wait(bc + q % kSR, (uint32_t)(q / kSR) & 1u);
        if (ok) ++waited_c;
      }
      if (ok) {
        const int q = a0 + r;
        ok = s_wait(ba + q % kSA, (uint32_t)(q / kSA) & 1u);
        if (ok) waited_a = r + 1;
      }
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      const int z = zb + r;
      const float *crow = rc + ((c0 + r + 4) % kSR) * kSRow + lane * 4;
      const float4 lf = *reinterpret_cast<const float4 *>(crow), c = *reinterpret_cast<const float4 *>(crow + 4),
                   rt = *reinterpret_cast<const float4 *>(crow + 8);
      float4 zq[9];
#pragma unroll
      for (int k = 0; k < 9; ++k)
        zq[k] = *reinterpret_cast<const float4 *>(rc + ((c0 + r + k) % kSR) * kSRow + lane * 4 + 4);
      const int qa = (a0 + r) % kSA;
      const float4 av = *reinterpret_cast<const float4 *>(ra + qa * kTileX + lane * 4);
      const float4 po = *reinterpret_cast<const float4 *>(rp + qa * kTileX + lane * 4);
      if (xl < L.NX4) {
        const int o = L.origin + z * L.pitch + xl;
        float4 v = leap4_2d(lf, c, rt, zq, po, av);
        const int d = S.src_off - o;
        if ((unsigned)d < 4u) point_sub(v, d, cmp(av, d) * f);
        st4(nxt + o, v);
      }
      __syncwarp();  // every lane is done with p^n row r and (a, p^{n-1}) row r: their slots refill
      if (lane == 0) {
        if (r + kSR < nrow + 8) issue_c(r + kSR);
        if (r + kSA < nrow) issue_a(r + kSA);
      }
    }
    if (!ok) {
      // let this task's copies in flight land before the block's shared memory goes away:
      // rows below min(r + ring, end) were issued, rows below waited_* were seen complete
      if (lane == 0) {
        atomicOr(err, 1);
        for (int i = waited_c; i < min(r + kSR, nrow + 8); ++i) {
          const int q = c0 + i;
          s_wait(bc + q % kSR, (uint32_t)(q / kSR) & 1u);
        }
        for (int i = waited_a; i < min(r + kSA, nrow); ++i) {
          const int q = a0 + i;
          s_wait(ba + q % kSA, (uint32_t)(q / kSA) & 1u);
        }
      }
      break;
    }
    gc = c0 + nrow + 8;
    ga = a0 + nrow;
  }
  griddep_launch();
}

// Streaming form of the fused reverse step (Eqs. 6, 2 and 3): the same
// per-warp task and rings as k_fwd2d_stream, with two window rings (p^R_n,
// pbar_n) and one ring of the rows read once (a, p^R_{n+1}, pbar_{n+1}, and
// num / den where the row meets the image).  The task's receivers are added
// to pbar_{n-1} after its last row is stored.
constexpr int kSRr = 12, kSAr = 3;
constexpr int kSWarpR = 2 * kSRr * kSRow + kSAr * 5 * kTileX;
constexpr size_t kStreamSmemR =
    sizeof(float) * kSWarpR * k2dWarps + sizeof(uint64_t) * (2 * kSRr + kSAr) * k2dWarps;

__global__ void __launch_bounds__(32 * k2dWarps) k_rev2d_stream(const BShot *__restrict__ shots,
                                                                 const int *__restrict__ item_shot, int item0,
                                                                 int item1, int n, int nt, const float *__restrict__ wav,
                                                                 float src_scale, float rec_scale, int *err) {
  extern __shared__ __align__(128) float sm_r[];
  const int lane = threadIdx.x, w = threadIdx.y;
  float *wr = sm_r + w * kSWarpR;          // [kSRr][kSRow] p^R_n
  float *wb = wr + kSRr * kSRow;           // [kSRr][kSRow] pbar_n
  float *rr = wb + kSRr * kSRow;           // [kSAr][5][128] a, p^R_{n+1}, pbar_{n+1}, num, den
  uint64_t *bw = reinterpret_cast<uint64_t *>(sm_r + k2dWarps * kSWarpR) + w * (2 * kSRr + kSAr);
  uint64_t *br = bw + 2 * kSRr;  // bw[kSRr]: the window slots' barriers (both rings)
  if (lane == 0) {
    for (int i = 0; i < 2 * kSRr + kSAr; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bw + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  griddep_wait();
  const bool do_r = n < nt && n > 0, do_b = n > 0;
  const float fsrc = do_r ? wav[n] * src_scale : 0.f;  // f[nt] does not exist
  int gc = 0, ga = 0;
  bool ok = true;
  for (int t = item0 + blockIdx.x * k2dWarps + w; ok && t < item1; t += gridDim.x * k2dWarps) {
    const BShot &S = shots[item_shot[t]];
    const Lay &L = S.L;
    const int loc = t - S.tbase_r;
    const int x0 = (loc % S.gx) * kTileX, zb = (loc / S.gx) * kSZ;
    const int nrow = min(kSZ, L.NZ - zb);
    const float *rc = (n & 1) ? S.p1 : S.p0;
    float *rn = (n & 1) ? S.p0 : S.p1;
    const float *bc = (n & 1) ? S.q1 : S.q0;
    float *bn = (n & 1) ? S.q0 : S.q1;
    const bool strip_img = x0 < S.ix1 && x0 + kTileX > S.ix0;
    const int c0 = gc, a0 = ga;
    auto issue_w = [&](int i) {
      const int q = c0 + i;
      const int o = L.origin + (zb - 4 + i) * L.pitch + x0 - 4;
      s_expect(bw + q % kSRr, 2 * kSRow * 4);
      s_copy(wr + (q % kSRr) * kSRow, rc + o, kSRow * 4, bw + q % kSRr);
      s_copy(wb + (q % kSRr) * kSRow, bc + o, kSRow * 4, bw + q % kSRr);
    };
    auto issue_r = [&](int i) {
      const int q = a0 + i, z = zb + i;
      const int o = L.origin + z * L.pitch + x0;
      float *d = rr + (q % kSAr) * 5 * kTileX;
      const bool img = strip_img && z >= S.iz0 && z < S.iz1;
      s_expect(br + q % kSAr, (img ? 5 : 3) * kTileX * 4);
      s_copy(d, S.a + o, kTileX * 4, br + q % kSAr);
      s_copy(d + kTileX, rn + o, kTileX * 4, br + q % kSAr);
      s_copy(d + 2 * kTileX, bn + o, kTileX * 4, br + q % kSAr);
      if (img) {
        s_copy(d + 3 * kTileX, S.num + o, kTileX * 4, br + q % kSAr);
        s_copy(d + 4 * kTileX, S.den + o, kTileX * 4, br + q % kSAr);
      }
    };
    if (lane == 0) {
      for (int i = 0; i < min(kSRr, nrow + 8); ++i) issue_w(i);
      for (int i = 0; i < min(kSAr, nrow); ++i) issue_r(i);
    }
    int waited_w = 0, waited_r = 0;
    const int xl = x0 + lane * 4;
    const bool xok = xl < L.NX4;
    int r = 0;
    for (; r < nrow; ++r) {
      while (ok && waited_w <= r + 8) {
        const int q = c0 + waited_w;
        ok = s_wait(bw + q % kSRr, (uint32_t)(q / kSRr) & 1u);
        if (ok) ++waited_w;
      }
      if (ok) {
        const int q = a0 + r;
        ok = s_wait(br + q % kSAr, (uint32_t)(q / kSAr) & 1u);
        if (ok) waited_r = r + 1;
      }
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      const int z = zb + r;
      const int o = L.origin + z * L.pitch + xl;
      const float *d = rr + ((a0 + r) % kSAr) * 5 * kTileX + lane * 4;
      const float4 av = *reinterpret_cast<const float4 *>(d);
      float4 cen[2];
#pragma unroll
      for (int f = 0; f < 2; ++f) {  // f = 0: p^R (Eq. 6), f = 1: pbar (Eq. 2)
        const float *ring = f ? wb : wr;
        const float *crow = ring + ((c0 + r + 4) % kSRr) * kSRow + lane * 4;
        const float4 lf = *reinterpret_cast<const float4 *>(crow), c = *reinterpret_cast<const float4 *>(crow + 4),
                     rt = *reinterpret_cast<const float4 *>(crow + 8);
        cen[f] = c;
        if ((f ? do_b : do_r) && xok) {
          float4 zq[9];
#pragma unroll
          for (int k = 0; k < 9; ++k)
            zq[k] = *reinterpret_cast<const float4 *>(ring + ((c0 + r + k) % kSRr) * kSRow + lane * 4 + 4);
          const float4 po = *reinterpret_cast<const float4 *>(d + (1 + f) * kTileX);
          float4 v = leap4_2d(lf, c, rt, zq, po, av);
          if (!f) {
            const int dd = S.src_off - o;
            if ((unsigned)dd < 4u) point_sub(v, dd, cmp(av, dd) * fsrc);
          }
          st4((f ? bn : rn) + o, v);
        }
      }
      if (strip_img && z >= S.iz0 && z < S.iz1 && xok && xl + 3 >= S.ix0 && xl < S.ix1) {
        st4(S.num + o, add4(*reinterpret_cast<const float4 *>(d + 3 * kTileX),
                            masked_prod(cen[0], cen[1], xl, S.ix0, S.ix1)));
        st4(S.den + o, add4(*reinterpret_cast<const float4 *>(d + 4 * kTileX),
                            masked_prod(cen[0], cen[0], xl, S.ix0, S.ix1)));
      }
      __syncwarp();  // the slots of row r are free
      if (lane == 0) {
        if (r + kSRr < nrow + 8) issue_w(r + kSRr);
        if (r + kSAr < nrow) issue_r(r + kSAr);
      }
    }
    if (!ok) {
      if (lane == 0) {
        atomicOr(err, 1);
        for (int i = waited_w; i < min(r + kSRr, nrow + 8); ++i) {
          const int q = c0 + i;
          s_wait(bw + q % kSRr, (uint32_t)(q / kSRr) & 1u);
        }
        for (int i = waited_r; i < min(r + kSAr, nrow); ++i) {
          const int q = a0 + i;
          s_wait(br + q % kSAr, (uint32_t)(q / kSAr) & 1u);
        }
      }
      break;
    }
    // Eq. 2 source term at the task's receivers, after all of its pbar_{n-1} stores
    if (do_b) {
      const int beg = S.tile_ptr[loc], end = S.tile_ptr[loc + 1];
      if (end > beg) {
        __syncwarp();
        for (int k = beg + lane; k < end; k += 32) {
          const int rec = S.tile_rec[k];
          const int oo = S.rec_off[rec];
          atomicAdd(bn + oo, rec_scale * S.a[oo] * S.seis_t[(long long)n * S.nrec + rec]);
        }
      }
    }
    gc = c0 + nrow + 8;
    ga = a0 + nrow;
  }
  griddep_launch();
}

// Per-shot max(den) on the interior (blockIdx.y = shot).
__global__ void k_batch_max(BShot *shots, const int *ncols, int nz) {
  BShot &S = shots[blockIdx.y];
  const int nx = ncols[blockIdx.y];
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nx * nz;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), z = (int)(i / nx);
    m = fmaxf(m, S.den[lay_off(S.L, x + S.ix0, 0, z + S.iz0)]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&S.maxbits, __float_as_uint(m));
}

// Eq. 3 ratio of every shot, stacked at its aperture offset (blockIdx.y = shot).
__global__ void k_batch_image(const BShot *shots, const int *ncols, int nz, float eps_rel, float *image, int sx) {
  const BShot &S = shots[blockIdx.y];
  const int nx = ncols[blockIdx.y];
  const float e = eps_rel * __uint_as_float(S.maxbits);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nx * nz;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), z = (int)(i / nx);
    const int o = lay_off(S.L, x + S.ix0, 0, z + S.iz0);
    atomicAdd(image + (long long)z * sx + x + S.off_x, S.num[o] / (S.den[o] + e));
  }
}

} // namespace

// ------------------------------------------------------------------ host --
struct rbc_batch {
  rbc_grid g;  // shared nz, nb, h, dt, nt (nx per shot)
  int nshots = 0;
  std::vector<int> nx;
  std::vector<Lay> L;
  std::vector<BShot> hs;
  float *arena = nullptr;
  BShot *ds = nullptr;
  int *d_ncols = nullptr;
  int *d_item_f = nullptr, *d_item_r = nullptr;
  int nitems_f = 0, nitems_r = 0;
  int rzf = 4, rzr = 2;  // rows per warp (rzf == 0: the streaming forward kernel)
  int *err_host = nullptr, *err_dev = nullptr;  // bounded waits that gave up (mapped)
  float tune_ms[8] = {};  // per-launch ms of the candidates: forward 0/1/2/4 rows, reverse 1/2/0/3
  int grid_f = 0, grid_r = 0;
  int rec_cap = 0, tile_cap = 0;
  int *d_rec_off = nullptr, *d_tile_ptr = nullptr, *d_tile_rec = nullptr;
  float *d_seis_t = nullptr;
  float *d_wav = nullptr;
  cudaStream_t cap = nullptr;
  // shots migrated together, so that a group's fields stay in L2 for its whole
  // time loop: group g = shots grp[g] .. grp[g+1]-1
  std::vector<int> grp;
  std::vector<cudaGraphExec_t> gexec;  // [kind * groups + g], kind 0 forward, 1 reverse
  bool use_graph = true;
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // three per group of every timed call
  int timed_calls = 0;
};

namespace {

// z rows of a reverse work item (rzr == 0: the streaming kernel's warp task)
int rev_tile_rows(const rbc_batch *b) { return b->rzr == 3 ? kBTileT : b->rzr ? k2dWarps * b->rzr : kSZ; }

int bfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return rbc::set_error(code, buf);
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(e_ == cudaErrorMemoryAllocation ? RBC_ENOMEM : RBC_ECUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                \
  } while (0)

void drop_graphs(rbc_batch *b) {
  for (size_t k = 0; k < b->gexec.size(); ++k) {
    if (b->gexec[k]) cudaGraphExecDestroy(b->gexec[k]);
    b->gexec[k] = nullptr;
  }
}

// Work lists for the chosen rows per warp: item -> shot, per-shot tile bases.
int build_items(rbc_batch *b) {
  std::vector<int> itf, itr;
  for (int s = 0; s < b->nshots; ++s) {
    BShot &S = b->hs[s];
    S.gx = cdiv(S.L.NX, kTileX);
    S.gzf = b->rzf ? cdiv(S.L.NZ, kBWarpsF * b->rzf) : cdiv(S.L.NZ, kSZ);
    S.gzr = cdiv(S.L.NZ, rev_tile_rows(b));
    S.tbase_f = (int)itf.size();
    S.tbase_r = (int)itr.size();
    itf.insert(itf.end(), (size_t)S.gx * S.gzf, s);
    itr.insert(itr.end(), (size_t)S.gx * S.gzr, s);
  }
  cudaFree(b->d_item_f);
  cudaFree(b->d_item_r);
  b->d_item_f = b->d_item_r = nullptr;
  b->nitems_f = (int)itf.size();
  b->nitems_r = (int)itr.size();
  BCK(cudaMalloc(&b->d_item_f, sizeof(int) * itf.size()));
  BCK(cudaMalloc(&b->d_item_r, sizeof(int) * itr.size()));
  BCK(cudaMemcpy(b->d_item_f, itf.data(), sizeof(int) * itf.size(), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->d_item_r, itr.data(), sizeof(int) * itr.size(), cudaMemcpyHostToDevice));
  return RBC_OK;
}

template <typename K>
int resident_grid(K kern, int items, size_t smem = 0, int warps = k2dWarps) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * warps, smem);
  const int slots = std::max(1, sms) * std::max(1, per);
  return std::max(1, std::min(items, slots));
}

// Work items [i0, i1) of a time step (all items by default).  The persistent
// grid shrinks to the items when a group has fewer than the resident slots.
bool launch_fwd_b(rbc_batch *b, int n, cudaStream_t s, int i0 = 0, int i1 = -1) {
  if (i1 < 0) i1 = b->nitems_f;
  const dim3 blk(32, k2dWarps);
  const float sc = 1.0f;  // h^(2-d) in 2-D
  const int items = i1 - i0;
  switch (b->rzf) {
  case 0: {
    const int gr = std::max(1, std::min(b->grid_f, cdiv(items, k2dWarps)));
    launch_pdl(k_fwd2d_stream, dim3(gr), blk, kStreamSmem, s, (const BShot *)b->ds, (const int *)b->d_item_f, i0, i1,
               n, (const float *)b->d_wav, sc, b->err_dev);
    break;
  }
  case 1:
    launch_pdl(k_fwd2d_batch<1>, dim3(std::min(b->grid_f, items)), dim3(32, kBWarpsF), 0, s, (const BShot *)b->ds,
               (const int *)b->d_item_f, i0, i1, n, (const float *)b->d_wav, sc);
    break;
  case 2:
    launch_pdl(k_fwd2d_batch<2>, dim3(std::min(b->grid_f, items)), dim3(32, kBWarpsF), 0, s, (const BShot *)b->ds,
               (const int *)b->d_item_f, i0, i1, n, (const float *)b->d_wav, sc);
    break;
  default:
    launch_pdl(k_fwd2d_batch<4>, dim3(std::min(b->grid_f, items)), dim3(32, kBWarpsF), 0, s, (const BShot *)b->ds,
               (const int *)b->d_item_f, i0, i1, n, (const float *)b->d_wav, sc);
    break;
  }
  return cudaPeekAtLastError() == cudaSuccess;
}

bool launch_rev_b(rbc_batch *b, int n, cudaStream_t s, int i0 = 0, int i1 = -1) {
  if (i1 < 0) i1 = b->nitems_r;
  const dim3 blk(32, k2dWarps);
  const int nt = b->g.nt;
  const int items = i1 - i0;
  switch (b->rzr) {
  case 0: {
    const int gr = std::max(1, std::min(b->grid_r, cdiv(items, k2dWarps)));
    launch_pdl(k_rev2d_stream, dim3(gr), blk, kStreamSmemR, s, (const BShot *)b->ds, (const int *)b->d_item_r, i0,
               i1, n, nt, (const float *)b->d_wav, 1.f, 1.f, b->err_dev);
    break;
  }
  case 1:
    launch_pdl(k_rev2d_batch<1>, dim3(std::min(b->grid_r, items)), blk, 0, s, (const BShot *)b->ds,
               (const int *)b->d_item_r, i0, i1, n, nt, (const float *)b->d_wav, 1.f, 1.f);
    break;
  case 3: {
    // the shots of the items [i0, i1) (whole shots), kBGMax per launch
    int sh = 0;
    while (sh < b->nshots && b->hs[sh].tbase_r < i0) ++sh;
    while (sh < b->nshots && b->hs[sh].tbase_r < i1) {
      BRevGroup G = {};
      G.shot0 = sh;
      const int base = b->hs[sh].tbase_r;
      for (; G.nshot < kBGMax && sh < b->nshots && b->hs[sh].tbase_r < i1; ++sh, ++G.nshot) {
        const BShot &H = b->hs[sh];
        G.tbase[G.nshot] = H.tbase_r - base;
        G.s[G.nshot] = BRevShot{H.L, H.a, H.p0, H.p1, H.q0, H.q1, H.num, H.den, H.gx, H.ix0, H.ix1, H.iz0, H.iz1};
      }
      const BShot &last = b->hs[G.shot0 + G.nshot - 1];
      G.tbase[G.nshot] = last.tbase_r + last.gx * last.gzr - base;
      launch_pdl(k_rev2d_batch_tile, dim3(G.tbase[G.nshot]), dim3(32, kBTileW), 0, s, G, (const BShot *)b->ds, n,
                 nt, (const float *)b->d_wav, 1.f, 1.f);
    }
    break;
  }
  default:
    launch_pdl(k_rev2d_batch<2>, dim3(std::min(b->grid_r, items)), blk, 0, s, (const BShot *)b->ds,
               (const int *)b->d_item_r, i0, i1, n, nt, (const float *)b->d_wav, 1.f, 1.f);
    break;
  }
  return cudaPeekAtLastError() == cudaSuccess;
}

void set_grids(rbc_batch *b) {
  switch (b->rzf) {
  case 0: b->grid_f = resident_grid(k_fwd2d_stream, cdiv(b->nitems_f, k2dWarps), kStreamSmem); break;
  case 1: b->grid_f = resident_grid(k_fwd2d_batch<1>, b->nitems_f, 0, kBWarpsF); break;
  case 2: b->grid_f = resident_grid(k_fwd2d_batch<2>, b->nitems_f, 0, kBWarpsF); break;
  default: b->grid_f = resident_grid(k_fwd2d_batch<4>, b->nitems_f, 0, kBWarpsF); break;
  }
  switch (b->rzr) {
  case 0: b->grid_r = resident_grid(k_rev2d_stream, cdiv(b->nitems_r, k2dWarps), kStreamSmemR); break;
  case 1: b->grid_r = resident_grid(k_rev2d_batch<1>, b->nitems_r); break;
  case 3: b->grid_r = b->nitems_r; break;  // one block per item
  default: b->grid_r = resident_grid(k_rev2d_batch<2>, b->nitems_r); break;
  }
}

void group_items(const rbc_batch *b, int g, bool fwd, int *i0, int *i1);

// Autotuner: time every rows-per-warp candidate of both kernels on the first
// shot group of the batch itself (zero fields, no receivers), as the time
// loop runs it, and keep the fastest.
int autotune(rbc_batch *b) {
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  auto time_it = [&](bool fwd) -> float {
    set_grids(b);
    int i0, i1;
    group_items(b, 0, fwd, &i0, &i1);
    auto go = [&](int n) { fwd ? launch_fwd_b(b, n, 0, i0, i1) : launch_rev_b(b, n, 0, i0, i1); };
    for (int k = 0; k < 3; ++k) go(10);
    float best = 1e30f;  // the fastest of three runs of 20 launches
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, 0);
      for (int k = 0; k < 20; ++k) go(10 + (k & 1));
      cudaEventRecord(e1, 0);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  int best_f = 4, best_r = 2;
  float tf = 1e30f, tr = 1e30f;
  // RBC_BATCH_TILES="f,r" restricts the candidates (a tuning and test knob)
  int force_f = -1, force_r = -1;
  if (const char *env = getenv("RBC_BATCH_TILES")) sscanf(env, "%d,%d", &force_f, &force_r);
  const int cf[4] = {0, 1, 2, 4}, cr[4] = {1, 2, 0, 3};
  for (int i = 0; i < 4; ++i) {
    if (force_f >= 0 && cf[i] != force_f) continue;
    b->rzf = cf[i];
    int rc = build_items(b);
    if (rc) return rc;
    BCK(cudaMemcpy(b->ds, b->hs.data(), sizeof(BShot) * b->nshots, cudaMemcpyHostToDevice));
    const float t = time_it(true);
    b->tune_ms[i] = t / 20;
    if (t < tf) tf = t, best_f = cf[i];
  }
  b->rzf = best_f;
  for (int i = 0; i < 4; ++i) {
    if (force_r >= 0 && cr[i] != force_r) continue;
    b->rzr = cr[i];
    int rc = build_items(b);
    if (rc) return rc;
    BCK(cudaMemcpy(b->ds, b->hs.data(), sizeof(BShot) * b->nshots, cudaMemcpyHostToDevice));
    const float t = time_it(false);
    b->tune_ms[4 + i] = t / 20;
    if (t < tr) tr = t, best_r = cr[i];
  }
  b->rzr = best_r;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = build_items(b);
  if (rc) return rc;
  set_grids(b);
  BCK(cudaMemcpy(b->ds, b->hs.data(), sizeof(BShot) * b->nshots, cudaMemcpyHostToDevice));
  BCK(cudaGetLastError());
  return RBC_OK;
}

// Work items of group g: the items of its shots are contiguous in both lists.
void group_items(const rbc_batch *b, int g, bool fwd, int *i0, int *i1) {
  const BShot &f = b->hs[b->grp[g]], &l = b->hs[b->grp[g + 1] - 1];
  *i0 = fwd ? f.tbase_f : f.tbase_r;
  *i1 = fwd ? l.tbase_f + l.gx * l.gzf : l.tbase_r + l.gx * l.gzr;
}

int enq_fwd(rbc_batch *b, int g, cudaStream_t s) {
  for (int i = b->grp[g]; i < b->grp[g + 1]; ++i) {
    const size_t bytes = sizeof(float) * (size_t)b->L[i].total;
    BCK(cudaMemsetAsync(b->hs[i].p0, 0, bytes, s));
    BCK(cudaMemsetAsync(b->hs[i].p1, 0, bytes, s));
  }
  int i0, i1;
  group_items(b, g, true, &i0, &i1);
  for (int n = 0; n < b->g.nt; ++n)
    if (!launch_fwd_b(b, n, s, i0, i1)) return bfail(RBC_ECUDA, "batched forward launch failed");
  return RBC_OK;
}

int enq_rev(rbc_batch *b, int g, cudaStream_t s) {
  for (int i = b->grp[g]; i < b->grp[g + 1]; ++i) {
    const size_t bytes = sizeof(float) * (size_t)b->L[i].total;
    BCK(cudaMemsetAsync(b->hs[i].q0, 0, bytes, s));
    BCK(cudaMemsetAsync(b->hs[i].q1, 0, bytes, s));
    BCK(cudaMemsetAsync(b->hs[i].num, 0, bytes, s));
    BCK(cudaMemsetAsync(b->hs[i].den, 0, bytes, s));
  }
  int i0, i1;
  group_items(b, g, false, &i0, &i1);
  for (int n = b->g.nt; n >= 0; --n)
    if (!launch_rev_b(b, n, s, i0, i1)) return bfail(RBC_ECUDA, "batched reverse launch failed");
  return RBC_OK;
}

// One phase (kind 0 forward, 1 reverse) of group g, as its cached graph.
int run_b(rbc_batch *b, int kind, int g, cudaStream_t s, long long *launches) {
  // the tiled reverse launches once per kBGMax shots of the group and step
  const long long chunks = b->rzr == 3 ? cdiv(b->grp[g + 1] - b->grp[g], kBGMax) : 1;
  const long long per = kind == 0 ? b->g.nt : (b->g.nt + 1) * chunks;
  if (!b->use_graph) {
    *launches += per;
    return kind == 0 ? enq_fwd(b, g, s) : enq_rev(b, g, s);
  }
  const int ng = (int)b->grp.size() - 1;
  if ((int)b->gexec.size() != 2 * ng) b->gexec.assign(2 * ng, nullptr);
  cudaGraphExec_t &ge = b->gexec[kind * ng + g];
  if (!ge) {
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    int rc = kind == 0 ? enq_fwd(b, g, b->cap) : enq_rev(b, g, b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return bfail(RBC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ge = nullptr;
      return bfail(RBC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  BCK(cudaGraphLaunch(ge, s));
  *launches += per;
  return RBC_OK;
}

} // namespace

extern "C" {

int rbc_batch_create(const rbc_grid *g, int nshots, const int *nx_host, const float *const *a_dev,
                     rbc_batch **out) {
  if (!g || !nx_host || !a_dev || !out || nshots < 1) return bfail(RBC_EINVAL, "rbc_batch_create: bad arguments");
  if (g->ndim != 2) return bfail(RBC_ENOTSUP, "rbc_batch_create: batches are 2-D");
  if (g->nz < 1 || g->nb < 2 || g->nt < 1 || !(g->h > 0) || !(g->dt > 0) || g->free_surface)
    return bfail(RBC_EINVAL, "rbc_batch_create: bad grid");
  *out = nullptr;
  rbc_batch *b = new rbc_batch();
  b->g = *g;
  b->nshots = nshots;
  const char *env = getenv("RBC_GRAPH");
  b->use_graph = !(env && env[0] == '0');
  cudaFuncSetAttribute(k_fwd2d_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStreamSmem);
  cudaFuncSetAttribute(k_rev2d_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStreamSmemR);
  if (cudaHostAlloc((void **)&b->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&b->err_dev, b->err_host, 0) != cudaSuccess) {
    delete b;
    return bfail(RBC_ENOMEM, "rbc_batch_create: error word allocation failed");
  }
  *b->err_host = 0;
  size_t total = 0;
  for (int s = 0; s < nshots; ++s) {
    if (nx_host[s] < 1 || !a_dev[s]) {
      delete b;
      return bfail(RBC_EINVAL, "rbc_batch_create: shot %d has no width or no coefficient", s);
    }
    b->nx.push_back(nx_host[s]);
    Lay L;
    if (!lay_make(2, (long long)nx_host[s] + 2LL * g->nb, 1, (long long)g->nz + 2LL * g->nb, &L)) {
      delete b;
      return bfail(RBC_EINVAL, "rbc_batch_create: shot %d is too large for 32-bit offsets", s);
    }
    b->L.push_back(L);
    total += 7 * (size_t)L.total;
  }
  // stability of every shot, as rbc_create checks it
  unsigned int *dmax = nullptr;
  if (cudaMalloc(&dmax, sizeof(unsigned int) * nshots) != cudaSuccess) {
    delete b;
    return bfail(RBC_ENOMEM, "rbc_batch_create: allocation failed");
  }
  cudaMemset(dmax, 0, sizeof(unsigned int) * nshots);
  for (int s = 0; s < nshots; ++s) launch_max(a_dev[s], (long long)b->L[s].NX * b->L[s].NZ, dmax + s, 0);
  std::vector<unsigned int> bits(nshots);
  cudaMemcpy(bits.data(), dmax, sizeof(unsigned int) * nshots, cudaMemcpyDeviceToHost);
  cudaFree(dmax);
  for (int s = 0; s < nshots; ++s) {
    float am;
    memcpy(&am, &bits[s], sizeof am);
    if (!(am * 2 * kSymbolMax < 4.0)) {
      delete b;
      return bfail(RBC_ECFL, "rbc_batch_create: shot %d is unstable (max (v dt/h)^2 = %g)", s, am);
    }
  }
  if (cudaMalloc(&b->arena, sizeof(float) * total) != cudaSuccess || cudaMemset(b->arena, 0, sizeof(float) * total) ||
      cudaMalloc(&b->ds, sizeof(BShot) * nshots) != cudaSuccess ||
      cudaMalloc(&b->d_ncols, sizeof(int) * nshots) != cudaSuccess ||
      cudaMalloc(&b->d_wav, sizeof(float) * g->nt) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    rbc_batch_destroy(b);
    return bfail(RBC_ENOMEM, "rbc_batch_create: allocation of %zu bytes failed", sizeof(float) * total);
  }
  cudaMemcpy(b->d_ncols, nx_host, sizeof(int) * nshots, cudaMemcpyHostToDevice);
  float *p = b->arena;
  b->hs.resize(nshots);
  for (int s = 0; s < nshots; ++s) {
    BShot &S = b->hs[s];
    memset(&S, 0, sizeof S);
    S.L = b->L[s];
    const long long T = S.L.total;
    S.a = p; S.p0 = p + T; S.p1 = p + 2 * T; S.q0 = p + 3 * T; S.q1 = p + 4 * T; S.num = p + 5 * T; S.den = p + 6 * T;
    p += 7 * T;
    S.ix0 = g->nb; S.ix1 = g->nb + b->nx[s]; S.iz0 = g->nb; S.iz1 = g->nb + g->nz;
    launch_copy_in(S.L, a_dev[s], S.a, 0);
  }
  // tuning-time receiver tables: every tile of every shot with no receiver
  int rc = RBC_OK;
  {
    size_t maxt = 0;
    for (int s = 0; s < nshots; ++s) maxt = std::max(maxt, (size_t)cdiv(b->L[s].NX, kTileX) * cdiv(b->L[s].NZ, k2dWarps) + 1);
    if (cudaMalloc(&b->d_tile_ptr, sizeof(int) * maxt) != cudaSuccess) {
      rbc_batch_destroy(b);
      return bfail(RBC_ENOMEM, "rbc_batch_create: allocation failed");
    }
    cudaMemset(b->d_tile_ptr, 0, sizeof(int) * maxt);
    b->tile_cap = (int)maxt;
    for (int s = 0; s < nshots; ++s) b->hs[s].tile_ptr = b->d_tile_ptr;
  }
  cudaMemset(b->d_wav, 0, sizeof(float) * g->nt);
  // shot groups: the fewest runs of consecutive shots whose seven fields fit
  // the L2 budget on average (RBC_BATCH_L2MB, megabytes; 0 puts every shot
  // in one group), cut where the running total crosses a multiple of the
  // mean group size, so that no group is left with a remainder of shots
  {
    double budget = 96.0;
    if (const char *e2 = getenv("RBC_BATCH_L2MB")) budget = atof(e2);
    std::vector<double> mb(nshots);
    double total_mb = 0;
    for (int s = 0; s < nshots; ++s) total_mb += mb[s] = 7.0 * sizeof(float) * (double)b->L[s].total / 1e6;
    const int ng = budget > 0 ? std::max(1, std::min(nshots, (int)ceil(total_mb / budget))) : 1;
    const double target = total_mb / ng;
    b->grp.assign(1, 0);
    double acc = 0;
    for (int s = 0; s < nshots; ++s) {
      const int k = std::min(ng - 1, (int)((acc + 0.5 * mb[s]) / target));  // group of shot s
      if (s > 0 && k > (int)b->grp.size() - 1) b->grp.push_back(s);
      acc += mb[s];
    }
    b->grp.push_back(nshots);
  }
  rc = autotune(b);
  if (rc) {
    rbc_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RBC_OK;
}

int rbc_batch_destroy(rbc_batch *b) {
  if (!b) return RBC_OK;
  cudaDeviceSynchronize();
  drop_graphs(b);
  cudaFree(b->arena);
  cudaFree(b->ds);
  cudaFree(b->d_ncols);
  cudaFree(b->d_item_f);
  cudaFree(b->d_item_r);
  cudaFree(b->d_rec_off);
  cudaFree(b->d_tile_ptr);
  cudaFree(b->d_tile_rec);
  cudaFree(b->d_seis_t);
  cudaFree(b->d_wav);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  const bool timed_out = b->err_host && *(volatile int *)b->err_host;
  if (b->err_host) cudaFreeHost(b->err_host);
  delete b;
  return timed_out ? bfail(RBC_ETIMEOUT, "rbc_batch_destroy: a bounded wait gave up; the last results are invalid")
                   : RBC_OK;
}

int rbc_batch_rtm(rbc_batch *b, const rbc_shot *shots, const float *wavelet_dev, int flags, float eps_rel,
                  float *image_dev, int survey_nx, void *stream) {
  if (!b || !shots || !wavelet_dev || !image_dev) return bfail(RBC_EINVAL, "rbc_batch_rtm: NULL argument");
  if (flags != RBC_REINJECT_SOURCE) return bfail(RBC_EINVAL, "rbc_batch_rtm: flags must be RBC_REINJECT_SOURCE");
  if (!(eps_rel >= 0)) return bfail(RBC_EINVAL, "rbc_batch_rtm: eps_rel must be >= 0");
  if (*(volatile int *)b->err_host) {
    *(volatile int *)b->err_host = 0;
    return bfail(RBC_ETIMEOUT, "rbc_batch_rtm: a bounded wait of an earlier call gave up; its results are invalid");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nt = b->g.nt;
  // receiver tables of every shot (counting sort by reverse tile)
  std::vector<int> off, ptr, order;
  std::vector<int> rec_base(b->nshots), ptr_base(b->nshots);
  long long seis_total = 0;
  std::vector<long long> seis_base(b->nshots);
  for (int i = 0; i < b->nshots; ++i) {
    const rbc_shot &sh = shots[i];
    const Lay &L = b->L[i];
    if (sh.off_x < 0 || sh.off_x + b->nx[i] > survey_nx)
      return bfail(RBC_EINVAL, "rbc_batch_rtm: shot %d window does not fit the survey", i);
    if (sh.nrec < 0 || (sh.nrec > 0 && (!sh.rec_host || !sh.seis_dev)))
      return bfail(RBC_EINVAL, "rbc_batch_rtm: shot %d has a bad receiver list", i);
    auto inside = [&](const int *r) { return r[0] >= 0 && r[0] < L.NX && r[1] == 0 && r[2] >= 0 && r[2] < L.NZ; };
    if (!inside(sh.src)) return bfail(RBC_EINVAL, "rbc_batch_rtm: shot %d source outside its grid", i);
    const int gx = cdiv(L.NX, kTileX), gz = cdiv(L.NZ, rev_tile_rows(b));
    rec_base[i] = (int)off.size();
    ptr_base[i] = (int)ptr.size();
    std::vector<int> cnt(gx * gz + 1, 0), tile(sh.nrec);
    for (int r = 0; r < sh.nrec; ++r) {
      const int *q = sh.rec_host + 3 * r;
      if (!inside(q)) return bfail(RBC_EINVAL, "rbc_batch_rtm: shot %d receiver %d outside its grid", i, r);
      off.push_back(lay_off(L, q[0], 0, q[2]));
      tile[r] = (q[2] / rev_tile_rows(b)) * gx + q[0] / kTileX;
      cnt[tile[r] + 1]++;
    }
    for (int t = 0; t < gx * gz; ++t) cnt[t + 1] += cnt[t];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1), ord(std::max(sh.nrec, 0));
    for (int r = 0; r < sh.nrec; ++r) ord[fill[tile[r]]++] = r;
    const int obase = (int)order.size();
    for (int t = 0; t <= gx * gz; ++t) ptr.push_back(obase + cnt[t]);
    order.insert(order.end(), ord.begin(), ord.end());
    seis_base[i] = seis_total;
    seis_total += (long long)(nt + 1) * sh.nrec;
  }
  // grow the capacity buffers (invalidates the graphs)
  const int nr = std::max(1, (int)off.size()), np = std::max(1, (int)ptr.size());
  if (nr > b->rec_cap || np > b->tile_cap || !b->d_seis_t || !b->d_rec_off) {
    drop_graphs(b);
    cudaFree(b->d_rec_off);
    cudaFree(b->d_tile_rec);
    cudaFree(b->d_tile_ptr);
    cudaFree(b->d_seis_t);
    b->d_rec_off = b->d_tile_rec = b->d_tile_ptr = nullptr;
    b->d_seis_t = nullptr;
    b->rec_cap = std::max(nr, b->rec_cap);
    b->tile_cap = std::max(np, b->tile_cap);
    BCK(cudaMalloc(&b->d_rec_off, sizeof(int) * b->rec_cap));
    BCK(cudaMalloc(&b->d_tile_rec, sizeof(int) * b->rec_cap));
    BCK(cudaMalloc(&b->d_tile_ptr, sizeof(int) * b->tile_cap));
    BCK(cudaMalloc(&b->d_seis_t, sizeof(float) * (size_t)b->rec_cap * (nt + 1)));
  }
  for (int i = 0; i < b->nshots; ++i) {
    BShot &S = b->hs[i];
    S.src_off = lay_off(b->L[i], shots[i].src[0], 0, shots[i].src[2]);
    S.nrec = shots[i].nrec;
    S.rec_off = b->d_rec_off + rec_base[i];
    S.tile_rec = b->d_tile_rec;  // the CSR holds positions in the whole list
    S.tile_ptr = b->d_tile_ptr + ptr_base[i];
    S.seis_t = b->d_seis_t + seis_base[i];
    S.off_x = shots[i].off_x;
    S.maxbits = 0;
  }
  // the CSR holds global positions into d_tile_rec, and d_tile_rec holds
  // shot-local receiver indices
  BCK(cudaMemcpyAsync(b->ds, b->hs.data(), sizeof(BShot) * b->nshots, cudaMemcpyHostToDevice, s));
  if (!off.empty()) {
    BCK(cudaMemcpyAsync(b->d_rec_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(b->d_tile_rec, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s));
  }
  BCK(cudaMemcpyAsync(b->d_tile_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(b->d_wav, wavelet_dev, sizeof(float) * nt, cudaMemcpyDeviceToDevice, s));
  long long launches = 0;
  for (int i = 0; i < b->nshots; ++i)
    if (shots[i].nrec > 0) {
      launch_transpose(shots[i].seis_dev, b->d_seis_t + seis_base[i], shots[i].nrec, nt + 1, s);
      ++launches;
    }
  // each group: forward phase then reverse phase, while its fields sit in L2
  const int ng = (int)b->grp.size() - 1;
  for (int g = 0; g < ng; ++g) {
    cudaEvent_t e3[3] = {nullptr, nullptr, nullptr};
    if (b->timing)
      for (int k = 0; k < 3; ++k) {
        BCK(cudaEventCreate(&e3[k]));
        b->ev.push_back(e3[k]);
      }
    if (b->timing) BCK(cudaEventRecord(e3[0], s));
    int rc = run_b(b, 0, g, s, &launches);
    if (rc) return rc;
    if (b->timing) BCK(cudaEventRecord(e3[1], s));
    rc = run_b(b, 1, g, s, &launches);
    if (rc) return rc;
    if (b->timing) BCK(cudaEventRecord(e3[2], s));
  }
  if (b->timing) b->timed_calls++;
  int maxnx = 0;
  for (int x : b->nx) maxnx = std::max(maxnx, x);
  const long long per = (long long)maxnx * b->g.nz;
  const int gxb = (int)std::min<long long>(1024, std::max<long long>(1, (per + 255) / 256));
  k_batch_max<<<dim3(gxb, b->nshots), 256, 0, s>>>(b->ds, b->d_ncols, b->g.nz);
  k_batch_image<<<dim3(gxb, b->nshots), 256, 0, s>>>(b->ds, b->d_ncols, b->g.nz, eps_rel, image_dev, survey_nx);
  launches += 2;
  rbc::add_launches(launches);
  BCK(cudaGetLastError());
  return RBC_OK;
}

int rbc_batch_timing(rbc_batch *b, int enable, double *out) {
  if (!b) return bfail(RBC_EINVAL, "rbc_batch_timing: NULL batch");
  double f = 0, r = 0;
  const size_t triples = b->ev.size() / 3, calls = (size_t)b->timed_calls;
  if (!enable || b->timing) {
    for (size_t k = 0; k < triples; ++k) {
      float t1 = 0, t2 = 0;
      BCK(cudaEventSynchronize(b->ev[3 * k + 2]));
      BCK(cudaEventElapsedTime(&t1, b->ev[3 * k], b->ev[3 * k + 1]));
      BCK(cudaEventElapsedTime(&t2, b->ev[3 * k + 1], b->ev[3 * k + 2]));
      f += t1;
      r += t2;
    }
  }
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  b->ev.clear();
  b->timed_calls = 0;
  b->timing = enable != 0;
  if (!enable && out) {
    out[0] = f;
    out[1] = r;
    out[2] = (double)calls * b->g.nt;
    out[3] = (double)calls * (b->g.nt + 1);
    out[4] = (double)calls;
  }
  return RBC_OK;
}

int rbc_batch_info(const rbc_batch *b, int *out) {
  if (!b || !out) return bfail(RBC_EINVAL, "rbc_batch_info: NULL argument");
  out[0] = b->rzf;
  out[1] = b->rzr;
  out[2] = b->nitems_f;
  out[3] = b->nitems_r;
  out[4] = b->grid_f;
  out[5] = b->grid_r;
  for (int i = 0; i < 8; ++i) out[6 + i] = (int)(b->tune_ms[i] * 1000.0f + 0.5f);  // microseconds
  out[14] = (int)b->grp.size() - 1;
  return RBC_OK;
}

} // extern "C"
