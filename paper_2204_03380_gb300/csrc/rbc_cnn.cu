// rbc_cnn.cu -- the learned random-boundary-noise denoiser: a 5-layer 3x3
// CNN (1 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU after layers 1-4, the
// input added to the last layer's output), bf16 operands with fp32
// accumulation.  Not in the paper: it stands in for stacking many random
// boundary realizations of an RTM image (Section 4.3's noise is incoherent
// between realizations).
//
// The 32-channel activations are bf16 and channel-group planar:
// [image][channel / 8][row][col][channel % 8] (16 bytes per pixel and group,
// so a row of one group is contiguous for the TMA copies and the tensor-core
// operands); one-channel images are [image][row][col].  Weights are stored
// [tap][out][in] (tap = 3 * dy + dx, dy, dx in 0..2 for offsets -1..1).
// The 32 -> 32 convolutions (three hidden layers, and their backward-data
// passes: the same kernel with the taps mirrored and the channel roles
// swapped, its epilogue applying the ReLU mask of the layer below) and the
// 32 -> 1 last layer run as implicit GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, operands in shared memory, fp32 accumulators in tensor
// memory).  The one-channel first layer runs on the warp-level tensor cores
// (mma.sync m16n8k16, the 9 taps padded to K = 16): as its own kernel in the
// training forward (its output is kept for the backward pass), inside the
// second layer's kernel for inference.  The weight gradients of
// the 32 -> 32 layers run on tcgen05 too (one MMA per 16 pixels covers all
// nine taps); those of the one-channel end layers on mma.sync with the taps
// on M.  Persistent blocks add their sums to the fp32 gradient once each.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <cstdlib>
#include <cstring>

#include "../../include/rbc.h"
#include "rbc_internal.cuh"

namespace rbc {
int set_error(int code, const char *msg);  // rbc_abi.cu
void add_launches(long long n);
}

namespace {

constexpr int C = 32;           // hidden channels
// parameter offsets (fp32 master copy): W1 b1 W2 b2 W3 b3 W4 b4 W5 b5
constexpr int kW1 = 0, kB1 = kW1 + 9 * C, kW2 = kB1 + C, kB2 = kW2 + 9 * C * C, kW3 = kB2 + C,
              kB3 = kW3 + 9 * C * C, kW4 = kB3 + C, kB4 = kW4 + 9 * C * C, kW5 = kB4 + C, kB5 = kW5 + 9 * C,
              kNParams = kB5 + 1;

__device__ __forceinline__ void mma16816(float *c, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

enum { kHidden = 0, kLast = 1, kBackData = 2, kFused = 3 };

// The one-channel first layer (1 -> 32 channels, and the last layer's
// backward-data pass) on the warp-level tensor cores:
//   wt [tap][32] (bf16);  MODE kHidden: relu(conv + bias);  kBackData: conv * (mask > 0)
// Per 16 pixels of a row, one m16n8k16 MMA per group of 8 output channels with K = the 9 taps
// (padded to 16, zero weights): the im2col operand A[pixel][tap] is gathered
// from the staged halo straight into the A fragments, the weights are the B
// fragments, held in registers for the whole kernel (the bias is the
// accumulator's initial value).  A block of 8 warps covers 8 rows x 128
// pixels (one warp per row); persistent blocks prefetch the next tile's halo
// into registers.  The output fragment of lane (g, t) holds channels
// 8n + 2t, 8n + 2t + 1 of pixels g and g + 8: 4-byte pieces of the pixels'
// 16-byte channel groups, stored 128 contiguous bytes per warp and group
// (rounded and clamped at zero by one conversion for the forward layer;
// masked by a packed compare of the layer's activation for the
// backward-data pass).  The backward-data pass stages each warp's mask row
// (8 KB) in shared memory by 16-byte cp.async copies issued before the
// tile's barrier, so that the copies of the blocks on an SM keep enough bytes
// in flight without holding registers.
// Tile counts are ints: a tile holds 1024 pixels of 64-byte activations.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}

constexpr int kM1R = 8, kM1C = 128;               // tile rows, columns
constexpr int kM1HW = kM1C + 2, kM1HP = (kM1R + 2) * kM1HW;  // halo columns, halo values
// halo row pitch in shared memory (2-byte values): 72 words, 8 banks apart,
// so the A-fragment gathers of a warp (three halo rows) are conflict-free
constexpr int kM1P = 144;
constexpr int kM1Pre = (kM1HP + 255) / 256;       // halo values per thread
constexpr int kM1MaskWords = 4 * kM1C * 4;        // a warp's staged mask row: [group][pixel][4 words]
template <int MODE> constexpr int smem_1to32() { return MODE == kBackData ? 8 * kM1MaskWords * 4 : 0; }
__device__ __forceinline__ uint32_t pack_u16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
// {lo, hi} rounded to bf16 (and clamped at zero for kRelu) in one 4-byte word
template <bool kRelu>
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
  uint32_t r;
  if (kRelu) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

template <int MODE>
__global__ void __launch_bounds__(256, 3) k_conv_1to32(const __nv_bfloat16 *__restrict__ in,
                                                        const __nv_bfloat16 *__restrict__ wt,
                                                        const float *__restrict__ bias,
                                                        const __nv_bfloat16 *__restrict__ mask,
                                                        __nv_bfloat16 *__restrict__ out, int nimg, int H, int W) {
  __shared__ __align__(16) uint16_t s_x[2][(kM1R + 2) * kM1P];
  extern __shared__ __align__(16) uint32_t s_m[];  // kBackData: the warps' mask rows
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int ntx = (W + kM1C - 1) / kM1C, tpi = ntx * ((H + kM1R - 1) / kM1R), ntiles = tpi * nimg;
  const long long HWp = (long long)H * W;
  const uint16_t *win = reinterpret_cast<const uint16_t *>(wt);
  // B fragments: B[k][co] = w[tap k][co] for k < 9, zero above
  uint32_t bf[4][2];
  float2 bs[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int co = 8 * n + g;
    bf[n][0] = pack_u16(win[(2 * t) * 32 + co], win[(2 * t + 1) * 32 + co]);
    bf[n][1] = t == 0 ? pack_u16(win[8 * 32 + co], 0) : 0u;
    bs[n] = MODE == kHidden ? make_float2(bias[8 * n + 2 * t], bias[8 * n + 2 * t + 1]) : make_float2(0.f, 0.f);
  }
  // halo offsets of this lane's taps: 2t, 2t + 1 (and 8 for t = 0), tap = 3 dy + dx
  const int o0 = ((2 * t) / 3) * kM1P + (2 * t) % 3, o1 = ((2 * t + 1) / 3) * kM1P + (2 * t + 1) % 3;
  constexpr int o8 = 2 * kM1P + 2;
  auto origin = [&](int tt, int &img, int &y0, int &x0) {
    img = tt / tpi;
    const int rem = tt - img * tpi, ty = rem / ntx;
    y0 = ty * kM1R;
    x0 = (rem - ty * ntx) * kM1C;
  };
  const uint16_t *xin = reinterpret_cast<const uint16_t *>(in);
  auto fetch = [&](int img, int y0, int x0, uint16_t *v) {
    const uint16_t *src = xin + (long long)img * HWp;
#pragma unroll
    for (int k = 0; k < kM1Pre; ++k) {
      const int i = tid + 256 * k, r = i / kM1HW;
      const int yy = y0 + r - 1, xx = x0 + (i - r * kM1HW) - 1;
      v[k] = (i < kM1HP && (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W) ? src[(long long)yy * W + xx]
                                                                                      : (uint16_t)0;
    }
  };
  auto park = [&](const uint16_t *v, int b) {
#pragma unroll
    for (int k = 0; k < kM1Pre; ++k) {
      const int i = tid + 256 * k, r = i / kM1HW;
      if (i < kM1HP) s_x[b][r * kM1P + (i - r * kM1HW)] = v[k];
    }
  };
  uint16_t v[kM1Pre];
  int img = 0, y0 = 0, x0 = 0;
  if ((int)blockIdx.x < ntiles) {
    origin(blockIdx.x, img, y0, x0);
    fetch(img, y0, x0, v);
    park(v, 0);
  }
  uint32_t *o32 = reinterpret_cast<uint32_t *>(out);
  int b = 0;
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x, b ^= 1) {
    const int tn = tt + gridDim.x;
    int img_n = 0, y0_n = 0, x0_n = 0;
    if (tn < ntiles) {  // in flight during this tile
      origin(tn, img_n, y0_n, x0_n);
      fetch(img_n, y0_n, x0_n, v);
    }
    const int y = y0 + warp;
    const int nx = min(kM1C, W - x0);  // columns of the tile inside the image
    uint32_t *sm = s_m + warp * kM1MaskWords;
    if (MODE == kBackData && y < H) {
      __syncwarp();  // the warp's reads of its previous mask row are done
      const uint4 *m16 = reinterpret_cast<const uint4 *>(mask) + ((long long)img * 4 * HWp + (long long)y * W + x0);
#pragma unroll
      for (int k = 0; k < 4 * kM1C / 32; ++k) {
        const int c = lane + 32 * k, n = c / kM1C, px = c % kM1C;
        if (px < nx) cp_async16((uint32_t)__cvta_generic_to_shared(sm + 4 * c), m16 + n * HWp + px, true);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __syncthreads();  // s_x[b] holds tile tt
    if (y < H) {
      if (MODE == kBackData) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
      }
      const uint16_t *sr = s_x[b] + warp * kM1P + g;
      // 4-byte piece t of pixel (y, x0 + g) in each channel group
      uint32_t *orow[4];
#pragma unroll
      for (int n = 0; n < 4; ++n) orow[n] = o32 + (((long long)img * 4 + n) * HWp + (long long)y * W + x0 + g) * 4 + t;
#pragma unroll
      for (int sg = 0; sg < kM1C / 16; ++sg) {
        if (16 * sg >= nx) break;
        const uint16_t *p0 = sr + 16 * sg, *p1 = p0 + 8;
        uint32_t a[4];
        a[0] = pack_u16(p0[o0], p0[o1]);
        a[1] = pack_u16(p1[o0], p1[o1]);
        a[2] = t == 0 ? (uint32_t)p0[o8] : 0u;
        a[3] = t == 0 ? (uint32_t)p1[o8] : 0u;
        float d[4][4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          d[n][0] = d[n][2] = bs[n].x;
          d[n][1] = d[n][3] = bs[n].y;
          mma16816(d[n], a, bf[n]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // pixels g (h = 0) and g + 8
          const int px = 16 * sg + 8 * h;
          if (px + g >= nx) continue;
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            uint32_t r;
            if (MODE == kHidden) {
              r = cvt_bf16x2<true>(d[n][2 * h], d[n][2 * h + 1]);
            } else {
              __nv_bfloat162 m2;
              *reinterpret_cast<uint32_t *>(&m2) = sm[(n * kM1C + px + g) * 4 + t];
              r = cvt_bf16x2<false>(d[n][2 * h], d[n][2 * h + 1]) & __hgt2_mask(m2, __float2bfloat162_rn(0.f));
            }
            orow[n][px * 4] = r;
          }
        }
      }
    }
    if (tn < ntiles) {  // read two tiles on, after the next barrier
      park(v, b ^ 1);
      img = img_n;
      y0 = y0_n;
      x0 = x0_n;
    }
  }
}

// ---------------------------------------------------------------------------
// 32 -> 32 channel layers on the 5th-generation tensor cores (tcgen05).
//
// A tile is R output rows x 126 columns of one image.  The accumulator
// of output row rr is a 128 (pixels) x 32 (channels) fp32 matrix in tensor
// memory:
//   D_rr[px][co] = sum_(dy, dx) sum_ci halo[rr + dy][px + dx][ci] * w[dy][dx][co][ci].
// Halo row h enters the accumulators of up to three output rows (rr = h - dy,
// dy = 0, 1, 2), each time with the same shifted operand and a different
// weight slice.  So the MMAs run per (halo row h, dx, half of the input
// channels) with M = 128 pixels, K = 16 channels and N = 32 x (number of
// output rows h reaches): B stacks the weights of those dy values, and the
// output rows' accumulators sit in tensor memory in descending row order
// (row rr at column (R - 1 - rr) * 32), so the N columns of one MMA are
// exactly the accumulators it feeds.  Against one N = 32 MMA per (row, tap,
// half) this reads each shifted halo operand once instead of up to three
// times: 6 (R + 2) MMAs per tile instead of 18 R, and 40 % less
// shared-memory operand traffic at R = 4.  Every MMA accumulates; the
// epilogue clears each accumulator after reading it.
// Both operands sit in shared memory in the no-swizzle K-major layout: a
// "core matrix" is 8 rows of 16 bytes (8 channels) stored contiguously.  The
// activations are kept channel-group planar in memory ([image][group of 8
// channels][row][column][8]), so one 4-D TMA copy (rows of 8-byte elements)
// lands a tile's halo as four planes (one per channel group) of halo pixels
// in row-major order at 16 bytes each: 8 consecutive pixels of any halo row
// are one core matrix, and
// the operand of a shifted tap is the same planes with the start address
// moved by (h * 128 + dx) * 16 bytes (stride between 8-pixel groups 128
// bytes, between channel groups one plane).  Weights in shared memory:
// [dx][ci / 8][dy][co][8], so the 96 (dy, co) rows of one (dx, ci group) are
// consecutive core matrices (stride 128 bytes) and the two channel groups of a
// K = 16 slice are 1536 bytes apart.
//
// Per block (one per SM, persistent over tiles), three roles: warp kTcEpi
// streams each tile's halo (zero-filled outside the image) into a shared-
// memory ring of tc_stages(R) stages (in the fused first-layer mode, builder
// warps compute it there instead); the next warp issues the 6 (R + 2)
// MMAs of a tile into one of two tensor-memory accumulators and commits them
// to the ring's "empty" and the accumulator's "full" barrier; warps 0 ..
// kTcEpi - 1 (two per tensor-memory lane quarter, one pixel per thread, half
// of the rows each) drain the other accumulator with tcgen05.ld, apply the
// epilogue (the backward-data pass reads its ReLU mask from global memory,
// issued before the accumulator wait) and store.  Copies of the next tiles,
// MMAs of tile k and the epilogue of tile k-1 overlap.  Every wait is bounded; a
// block that gives up flags the error word and stops.
// A tile is kTcOut = 126 output columns: its halo row is then 128 pixels of
// 16 bytes, 2 KB, which one tensor copy moves as 256 8-byte elements (the
// box limit), against a box whose innermost dimension is one pixel's 16
// bytes; measured on GB300 streaming such halos on every SM: 9.2 TB/s for
// the 2 KB rows, 4.4 TB/s for the 16-byte rows.  The MMAs keep M = 128:
// rows 126 and 127 of a shifted operand run into the next halo row and
// their outputs are discarded.
constexpr int kTcOut = 126;                                  // output columns per tile
constexpr int kTcHW = 128;                                   // halo row width (pixels)
constexpr int kTcWBytes = 9 * 4 * 32 * 16;                   // weights, 18432 B
constexpr long long kTcWaitCycles = 4000000000LL;            // about two seconds
constexpr int kTcEpi = 8;                                    // epilogue warps
// Tiles of R output rows: halo planes of R + 2 rows per channel group, a
// ring of 4 stages for R = 4, 3 for R = 6 and 2 for R = 8 (what fits in
// 227 KB); R = 8 fills tensor memory with the two accumulator buffers.
// Measured at 32 x 512^2 with 126-column tiles (inference / training step):
// R = 8 0.951 / 5.20 ms, R = 6 0.969 / 5.37 ms, R = 4 1.071 / 5.49 ms; with
// 128-column tiles and the 16-byte-row halo copy: R = 6 1.14 / 5.51 ms, R = 4
// 1.18 / 5.57 ms, R = 4 with 4 epilogue warps 1.23 / 5.88 ms.
constexpr int kTcR = 8;
constexpr int tc_plane(int R) { return (R + 2) * kTcHW * 16; }
constexpr int tc_stages(int R) { return R <= 4 ? 4 : R <= 6 ? 3 : 2; }
constexpr int tc_smem(int R) { return kTcWBytes + tc_stages(R) * 4 * tc_plane(R) + 256; }
static_assert(tc_smem(6) <= 227 * 1024, "the R = 6 ring must fit in shared memory");
static_assert(2 * 8 * 32 <= 512, "two accumulator buffers must fit in tensor memory");
static_assert(tc_smem(8) <= 227 * 1024, "the R = 8 ring must fit in shared memory");

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // no swizzle; start, leading (K) and stride (M/N) byte offsets in 16-byte
  // units; bits 46-47 = 1 (descriptor version of this architecture)
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: fp32 accumulator, bf16 A and B, both
// K-major, M = 128, N = n (a multiple of 16, at most 256).
constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}


__device__ __forceinline__ void tmem_ld32(uint32_t ta, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

// Clear 32 columns of this warp's 32 tensor-memory lanes (completion by
// tcgen05.wait::st).
__device__ __forceinline__ void tmem_zero32(uint32_t ta) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(ta), "r"(0u)
      : "memory");
}

__device__ __forceinline__ void tc_mbar_init(uint32_t b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool tc_try(uint32_t b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(b), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait that gives up when another role of the block has flagged an
// abort, and flags one itself when its time runs out.
__device__ __forceinline__ bool tc_wait(uint32_t b, uint32_t parity, volatile int *abort_blk) {
  if (tc_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!tc_try(b, parity)) {
    if (*abort_blk) return false;
    if (clock64() - t0 > kTcWaitCycles) {
      *abort_blk = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tc_tma4(uint32_t dst, const CUtensorMap *tm, int c0, int c1, int c3, uint32_t bar) {
  // coordinates (8-byte element along the row, y, group 0, image)
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(0), "r"(c3), "r"(bar)
      : "memory");
}

// Tensor-memory columns to allocate for c columns (a power of two >= 32).
constexpr int tmem_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

__device__ __forceinline__ float tmem_ld1(uint32_t ta) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return __uint_as_float(r);
}
__device__ __forceinline__ void tmem_zero1(uint32_t ta) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(ta), "r"(0u) : "memory");
}

//   MODE kHidden:   out = relu(conv(in) + bias)                        (32 -> 32)
//   MODE kBackData: out = conv(in) * (mask > 0)   (weights mirrored and transposed)
//   MODE kLast:     out_f = resid + conv(in) + bias                    (32 -> 1)
//   MODE kFused:    out = relu(conv(a1) + bias) with a1 = relu(conv1(x1) + b1)
//                   computed in the block (the first two layers, for inference)
// The last layer's single output channel is padded to N = 16 per output row
// (the smallest N of an M = 128 MMA); the 15 padding channels have zero
// weights, so their accumulators stay zero and only channel 0 is read out.
// kTcEpi epilogue warps: warp e drains TMEM lane quarter e % 4 (pixels
// 32 (e % 4) .. +31) for the output rows of its share (R * 4 / kTcEpi rows,
// starting at row (e / 4) * R * 4 / kTcEpi); warps kTcEpi .. kTcEpi +
// tc_nprod(MODE) - 1 are the producers, the next warp the MMA issuer.
//
// kFused: instead of the tensor copy of a stored first-layer output, ten
// builder warps compute it over the tile's halo (R + 2 rows x 128 pixels,
// one row per warp) into the ring stage, in the layout the copy would have
// produced: the fp32 one-channel input's halo (R + 4 rows x 130 pixels,
// prefetched a tile ahead into registers, rounded to bf16) is parked in
// shared memory, and each 16 pixels of a halo row are one m16n8k16 MMA per 8
// channels as in k_conv_1to32 (taps padded to K = 16, bias as the
// accumulator's start, relu and rounding in one conversion), stored as
// 4-byte pieces of the pixels' 16-byte channel groups at constant offsets
// from the row's base; outside the image the stage holds zeros (the second
// layer's padding).  The builders then make their writes visible to the
// tensor cores and arrive on the stage's "full" barrier.  The first layer's
// output never passes through global memory.
constexpr int tc_nprod(int mode) { return mode == kFused ? 10 : 1; }
constexpr int tc_threads(int mode) { return 32 * (kTcEpi + tc_nprod(mode) + 1); }
constexpr int kFxR = 4;                  // x halo rows beyond the tile's R (two on each side)
constexpr int kFxC = kTcHW + 2;          // x halo columns (x0 - 2 .. x0 + 127)
constexpr int kFxP = 144;                // x halo row pitch (2-byte values; conflict-free gathers)
constexpr int tc_fx_bytes(int R) { return (R + kFxR) * kFxP * 2; }
constexpr int tc_fx_vals(int R) { return (R + kFxR) * kFxC; }  // x halo values of a tile
constexpr int tc_smem_mode(int mode, int R) { return tc_smem(R) + (mode == kFused ? tc_fx_bytes(R) : 0); }
static_assert(tc_smem(kTcR) + tc_fx_bytes(kTcR) <= 227 * 1024, "the fused ring must fit in shared memory");

template <int MODE, int R>
__global__ void __launch_bounds__(tc_threads(MODE), 1) k_conv_tc(const __grid_constant__ CUtensorMap tm_in,
                                                    const __nv_bfloat16 *__restrict__ wt,
                                                    const float *__restrict__ bias,
                                                    const __nv_bfloat16 *__restrict__ mask,
                                                    __nv_bfloat16 *__restrict__ out, float *__restrict__ out_f,
                                                    const float *__restrict__ resid, int nimg, int H, int W,
                                                    int *err, const float *__restrict__ x1 = nullptr,
                                                    const __nv_bfloat16 *__restrict__ w1 = nullptr,
                                                    const float *__restrict__ b1 = nullptr) {
  constexpr bool kHid = MODE == kHidden || MODE == kFused;  // relu(conv + bias) epilogue
  constexpr int kMma = kTcEpi + tc_nprod(MODE);             // the MMA issuer warp
  constexpr int NCO = MODE == kLast ? 16 : 32;  // output channels per row accumulator
  constexpr int WCG = 3 * NCO * 16;              // weight bytes per (dx, channel group)
  constexpr int WDX = 4 * WCG;                   // weight bytes per dx
  constexpr int BUF = R * NCO;             // accumulator columns per tile buffer
  constexpr int TCOLS = tmem_cols(2 * BUF);
  constexpr int PLANE = tc_plane(R), STAGES = tc_stages(R), STAGE = 4 * PLANE;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t s_w = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t s_h = s_w + kTcWBytes;  // halo ring
  unsigned char *tail = smem + kTcWBytes + STAGES * STAGE;
  float *s_bias = reinterpret_cast<float *>(tail);
  // barriers: full[STAGES], empty[STAGES], tfull[2], tempty[2]
  uint64_t *bars = reinterpret_cast<uint64_t *>(tail + 128);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 4);
  volatile int *abort_blk = reinterpret_cast<volatile int *>(tslot + 1);
  const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(bars);
  auto full = [&](int i) { return b0 + 8u * i; };
  auto empty = [&](int i) { return b0 + 8u * (STAGES + i); };
  auto tfull = [&](int i) { return b0 + 8u * (2 * STAGES + i); };
  auto tempty = [&](int i) { return b0 + 8u * (2 * STAGES + 2 + i); };
  // weights [tap][co][ci] (tap = 3 dy + dx) -> [dx][ci / 8][dy][co][8]
  if (MODE == kLast) {
    for (int i = tid; i < 9 * 4 * (NCO - 1); i += blockDim.x) {  // padding channels 1..15: zero
      const int co = 1 + i % (NCO - 1), r = i / (NCO - 1), j = r & 3, t = r >> 2;
      *reinterpret_cast<uint4 *>(smem + (t % 3) * WDX + j * WCG + (t / 3) * NCO * 16 + co * 16) =
          make_uint4(0u, 0u, 0u, 0u);
    }
    for (int i = tid; i < 9 * 4; i += blockDim.x) {
      const int j = i & 3, t = i >> 2;
      cp_async16(s_w + (t % 3) * WDX + j * WCG + (t / 3) * NCO * 16, wt + t * 32 + j * 8, true);
    }
  } else {
    for (int i = tid; i < 9 * 32 * 4; i += blockDim.x) {
      const int j = i & 3, co = (i >> 2) & 31, t = i >> 7, dy = t / 3, dx = t % 3;
      cp_async16(s_w + dx * WDX + j * WCG + dy * NCO * 16 + co * 16, wt + (t * 32 + co) * 32 + j * 8, true);
    }
  }
  if (kHid && tid < 32) s_bias[tid] = bias[tid];
  if (MODE == kLast && tid == 0) s_bias[0] = bias[0];
  if (tid == 0) {
    *abort_blk = 0;
    for (int i = 0; i < STAGES; ++i) {
      tc_mbar_init(full(i), MODE == kFused ? 32 * tc_nprod(MODE) : 1);
      tc_mbar_init(empty(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc_mbar_init(tfull(i), 1);
      tc_mbar_init(tempty(i), 32 * kTcEpi);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
        (uint32_t)__cvta_generic_to_shared(tslot)), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (warp < 4) {  // every MMA accumulates: both accumulator buffers start at zero
#pragma unroll 1
    for (int c = 0; c < 2 * BUF; c += 32) tmem_zero32(tmem + ((uint32_t)(warp * 32) << 16) + c);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int ntx = (W + kTcOut - 1) / kTcOut, nty = (H + R - 1) / R;
  const long long ntiles = (long long)ntx * nty * nimg;
  // Each block takes a contiguous range of tiles, ordered down the image
  // columns (y fastest): a tile's two halo rows are rows of the block's
  // previous tile, fetched a moment earlier and still in L2, so DRAM reads
  // each activation row about once instead of 1.5 times.
  // persistent blocks over the tiles, x fastest (measured against a
  // contiguous y-fastest range per block, which lost: 1.36 vs 1.27 ms per
  // 32 x 512^2 inference)
  auto tile_xy = [&](long long t, int &img, int &y0, int &x0) {
    img = (int)(t / ((long long)ntx * nty));
    const int rem = (int)(t % ((long long)ntx * nty));
    y0 = (rem / ntx) * R;
    x0 = (rem % ntx) * kTcOut;
  };
  if (MODE != kFused && warp == kTcEpi) {
    // ---- producer: one TMA copy of the halo per tile ----
    // (one bulk copy per channel group and halo row instead lost by 2.1x)
    if (lane == 0) {
      int issued = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++issued) {
        const int s = issued % STAGES, u = issued / STAGES;
        if (u > 0 && !tc_wait(empty(s), (u - 1) & 1, abort_blk)) break;
        int img, y0, x0;
        tile_xy(t, img, y0, x0);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(s)), "r"(STAGE) : "memory");
        tc_tma4(s_h + s * STAGE, &tm_in, 2 * (x0 - 1), y0 - 1, img, full(s));
      }
      if (*abort_blk) {  // let the copies in flight land before the block exits
        for (int k = (issued > STAGES ? issued - STAGES : 0); k < issued; ++k) {
          const long long t0 = clock64();
          while (!tc_try(full(k % STAGES), (k / STAGES) & 1) && clock64() - t0 < kTcWaitCycles) {
          }
        }
      }
    }
  } else if (MODE == kFused && warp >= kTcEpi && warp < kMma) {
    // ---- builders (kFused): the first layer's output over the tile's halo ----
    constexpr int NB = tc_nprod(MODE), NBT = 32 * NB;                    // builder warps, threads
    constexpr int XVALS = tc_fx_vals(R), NPRE = (XVALS + NBT - 1) / NBT;  // x values, per builder thread
    static_assert((R + 2) % NB == 0, "each builder warp owns the same number of halo rows");
    const int bt = tid - 32 * kTcEpi, g = lane >> 2, tq = lane & 3;
    const int bw = warp - kTcEpi;
    uint16_t *xs = reinterpret_cast<uint16_t *>(smem + tc_smem(R));
    unsigned char *hs = smem + kTcWBytes;  // generic address of the ring
    const uint16_t *w1u = reinterpret_cast<const uint16_t *>(w1);
    uint32_t bf[4][2];  // B fragments: B[k][co] = w1[tap k][co] for k < 9, zero above
    float2 bs[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int co = 8 * n + g;
      bf[n][0] = pack_u16(w1u[(2 * tq) * 32 + co], w1u[(2 * tq + 1) * 32 + co]);
      bf[n][1] = tq == 0 ? pack_u16(w1u[8 * 32 + co], 0) : 0u;
      bs[n] = make_float2(b1[8 * n + 2 * tq], b1[8 * n + 2 * tq + 1]);
    }
    const int o0 = ((2 * tq) / 3) * kFxP + (2 * tq) % 3, o1 = ((2 * tq + 1) / 3) * kFxP + (2 * tq + 1) % 3;
    constexpr int o8 = 2 * kFxP + 2;
    const long long HWp = (long long)H * W;
    auto bar_b = [] { asm volatile("bar.sync 1, %0;" ::"n"(NBT) : "memory"); };
    // barrier of the builders that returns whether any of them saw the abort
    // flag (one decision for all of them)
    auto bar_b_abort = [&]() -> bool {
      uint32_t any;
      asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
                   : "=r"(any)
                   : "r"((uint32_t)*abort_blk), "n"(NBT)
                   : "memory");
      return any != 0;
    };
    // this thread's share of tile t's x halo (rows y0 - 2 .., columns x0 - 2
    // ..), left in flight as fp32 until park() rounds and stores it
    auto fetch = [&](long long t, float *v) {
      int img, y0, x0;
      tile_xy(t, img, y0, x0);
      const float *src = x1 + (long long)img * HWp;
#pragma unroll
      for (int k = 0; k < NPRE; ++k) {
        const int i = bt + NBT * k, r = i / kFxC;
        const int yy = y0 - 2 + r, xx = x0 - 2 + (i - r * kFxC);
        v[k] = (i < XVALS && (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W) ? src[(long long)yy * W + xx]
                                                                                       : 0.f;
      }
    };
    auto park = [&](const float *v) {
#pragma unroll
      for (int k = 0; k < NPRE; ++k) {
        const int i = bt + NBT * k, r = i / kFxC;
        if (i < XVALS) xs[r * kFxP + (i - r * kFxC)] = __bfloat16_as_ushort(__float2bfloat16(v[k]));
      }
    };
    float v[NPRE];
    if ((long long)blockIdx.x < ntiles) {
      fetch(blockIdx.x, v);
      park(v);
    }
    bar_b();
    int issued = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++issued) {
      const int s = issued % STAGES, u = issued / STAGES;
      const long long tn = t + gridDim.x;
      if (tn < ntiles) fetch(tn, v);  // in flight while this tile is built
      if (u > 0) tc_wait(empty(s), (u - 1) & 1, abort_blk);
      if (bar_b_abort()) break;
      int img, y0, x0;
      tile_xy(t, img, y0, x0);
#pragma unroll 1
      for (int h = bw; h < R + 2; h += NB) {  // halo row h: image row y0 - 1 + h
        // this lane's 4-byte piece of pixel (h, g) in channel group 0
        unsigned char *row = hs + s * STAGE + (h * kTcHW + g) * 16 + 4 * tq;
        if ((unsigned)(y0 - 1 + h) >= (unsigned)H) {  // outside the image: the second layer's zero padding
#pragma unroll
          for (int i = 0; i < kTcHW; i += 8)
#pragma unroll
            for (int n = 0; n < 4; ++n) *reinterpret_cast<uint32_t *>(row + n * PLANE + i * 16) = 0u;
          continue;
        }
        const uint16_t *xr = xs + h * kFxP + g;
        const int xg = x0 - 1 + g;  // image column of pixel (h, g)
#pragma unroll
        for (int i0 = 0; i0 < kTcHW; i0 += 16) {
          const uint16_t *p0 = xr + i0, *p1 = p0 + 8;
          uint32_t a[4];
          a[0] = pack_u16(p0[o0], p0[o1]);
          a[1] = pack_u16(p1[o0], p1[o1]);
          a[2] = tq == 0 ? (uint32_t)p0[o8] : 0u;
          a[3] = tq == 0 ? (uint32_t)p1[o8] : 0u;
          float d[4][4];
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            d[n][0] = d[n][2] = bs[n].x;
            d[n][1] = d[n][3] = bs[n].y;
            mma16816(d[n], a, bf[n]);
          }
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {  // pixels g (hh = 0) and g + 8
            const bool in = (unsigned)(xg + i0 + 8 * hh) < (unsigned)W;
#pragma unroll
            for (int n = 0; n < 4; ++n)
              *reinterpret_cast<uint32_t *>(row + n * PLANE + (i0 + 8 * hh) * 16) =
                  in ? cvt_bf16x2<true>(d[n][2 * hh], d[n][2 * hh + 1]) : 0u;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_arrive(full(s));
      bar_b();  // every builder is done with the parked halo
      if (tn < ntiles) park(v);
      bar_b();
    }
  } else if (warp == kMma) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int k = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % STAGES, u = k / STAGES, b = k & 1, ub = k >> 1;
        if (!tc_wait(full(s), u & 1, abort_blk)) break;
        if (ub > 0 && !tc_wait(tempty(b), (ub - 1) & 1, abort_blk)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // descriptors differ only in their start-address field: one add per MMA
        // (fully unrolled, the offsets are constants; a single thread issues
        // all of them, so per-MMA arithmetic would bound the tile)
        const uint64_t a0 = umma_desc(s_h + s * STAGE, PLANE, 128), b0d = umma_desc(s_w, WCG, 128);
        const uint32_t d0 = tmem + b * BUF;
#pragma unroll
        for (int h = 0; h < R + 2; ++h) {
          // output rows h - j for j in [j0, j1] (those inside the tile)
          const int j0 = h > R - 1 ? h - (R - 1) : 0, j1 = h < 2 ? h : 2;
          const uint32_t idesc = tc_idesc(NCO * (j1 - j0 + 1));
          const uint32_t d = d0 + (uint32_t)((R - 1 - h + j0) * NCO);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint64_t ad = a0 + (uint64_t)((2 * ks * PLANE + (h * kTcHW + dx) * 16) >> 4);
              const uint64_t bd = b0d + (uint64_t)((dx * WDX + 2 * ks * WCG + j0 * NCO * 16) >> 4);
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                           "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d), "l"(ad),
                           "l"(bd), "r"(idesc), "r"(1u));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(s))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tfull(b))
                     : "memory");
      }
    }
  } else {
    // ---- epilogue: warps 0 .. kTcEpi-1, one accumulator row (pixel) per thread ----
    constexpr int RE = R * 4 / kTcEpi;  // output rows per epilogue warp
    const int lq = warp & 3, r0 = (warp >> 2) * RE;
    const uint32_t lanes = (uint32_t)(lq * 32) << 16;
    const long long HWp = (long long)H * W;
    int k = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int b = k & 1, ub = k >> 1;
      int img, y0, x0;
      tile_xy(t, img, y0, x0);
      const int px = lq * 32 + lane, xx = px < kTcOut ? x0 + px : W;  // MMA rows 126, 127: no pixel
      float rs[RE];     // last layer: this pixel's residual input, loaded while the MMAs run
      if (MODE == kLast) {
#pragma unroll
        for (int i = 0; i < RE; ++i)
          rs[i] = (y0 + r0 + i < H && xx < W) ? resid[(long long)img * HWp + (long long)(y0 + r0 + i) * W + xx] : 0.f;
      }
      uint4 mk[RE][4];  // backward-data: this pixel's masks, loaded while the MMAs run
      if (MODE == kBackData) {
#pragma unroll
        for (int i = 0; i < RE; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            mk[i][q] = (y0 + r0 + i < H && xx < W)
                           ? reinterpret_cast<const uint4 *>(mask)[((long long)img * 4 + q) * HWp +
                                                                  (long long)(y0 + r0 + i) * W + xx]
                           : make_uint4(0u, 0u, 0u, 0u);
      }
      const bool ok = tc_wait(tfull(b), ub & 1, abort_blk);
      if (__any_sync(0xffffffffu, !ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if constexpr (MODE == kLast) {
#pragma unroll
        for (int rr = r0; rr < r0 + RE; ++rr) {
          const uint32_t ta = tmem + lanes + b * BUF + (R - 1 - rr) * NCO;
          const float v0 = tmem_ld1(ta);
          tmem_zero1(ta);  // channel 0 only: the padding channels never leave zero
          const int yy = y0 + rr;
          if (yy < H && xx < W) out_f[(long long)img * HWp + (long long)yy * W + xx] = rs[rr - r0] + v0 + s_bias[0];
        }
      } else {
#pragma unroll 1
      for (int rr = r0; rr < r0 + RE; ++rr) {
        float v[32];
        const uint32_t ta = tmem + lanes + b * BUF + (R - 1 - rr) * NCO;
        tmem_ld32(ta, v);
        tmem_zero32(ta);  // the next tile in this buffer accumulates from zero
        const int yy = y0 + rr;
        if (yy < H && xx < W) {
          const long long pix = (long long)yy * W + xx;
          if (kHid) {
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + s_bias[c], 0.f);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint4 m4 = mk[rr - r0][q];
              const __nv_bfloat162 *m2 = reinterpret_cast<const __nv_bfloat162 *>(&m4);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 mf = __bfloat1622float2(m2[e]);
                v[q * 8 + 2 * e] = mf.x > 0.f ? v[q * 8 + 2 * e] : 0.f;
                v[q * 8 + 2 * e + 1] = mf.y > 0.f ? v[q * 8 + 2 * e + 1] : 0.f;
              }
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint4 pk;
            __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
            for (int e = 0; e < 4; ++e) p2[e] = __floats2bfloat162_rn(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1]);
            reinterpret_cast<uint4 *>(out)[((long long)img * 4 + q) * HWp + pix] = pk;
          }
        }
      }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      tc_arrive(tempty(b));
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_blk) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == kMma) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// ldmatrix of four 8 x 8 bf16 matrices, transposed (rows given by lanes 8j .. 8j + 7).
__device__ __forceinline__ void ldsm_x4_t(uint32_t *r, const void *smem_row) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sa));
}

// Weight and bias gradients of the 32 -> 32 layers on the 5th-generation
// tensor cores:
//   dW[dy][dx][co][ci] = sum_p dz[co][p] x[ci][p + (dy - 1, dx - 1)],   db[co] = sum_p dz[co][p].
// Re-indexed by q = p + (dy - 1) rows, the taps split between the operands:
//   dW[dy][dx][co][ci] = sum_q x[ci][q + (0, dx - 1)] dz[co][q - (dy - 1, 0)],
// so that one MMA per 16 pixels q of a row (K = 16) computes all nine taps,
// D[32 dx + ci][32 (2 - dy) + co] (M = 128, N = 96; fp32 in tensor memory).
// Both operands are MN-major (channels contiguous) in a pixel-major layout
// with the 64-byte swizzle: a pixel's 32 channels form one 64-byte row, and
// the swizzle is a function of the shared-memory address, so a descriptor
// may start at any pixel.  A = x: its 32-row M blocks start one pixel apart
// (leading byte offset 64), block j holding the tap dx = j (block 3 is read
// but not used); B = dz: its 32-column N blocks start one staged row apart,
// block i holding the tap dy = 2 - i; a K step of 8 pixels is 512 bytes.
// Tiles of 4 rows x 128 pixels: x is staged over the tile's rows and pixels
// x0 - 1 .. x0 + 130, dz over rows y0 - 1 .. y0 + 4 and pixels x0 .. x0 + 127,
// in two stages: the 512 threads load tile k + 1 into registers (16 bytes
// per chunk, consecutive lanes on consecutive pixels of a channel-group plane,
// so the loads coalesce; zero outside the image) while tile k is multiplied,
// and store the chunks into their swizzled places once tile k - 1's MMAs have
// released the stage.  (cp.async copies into the swizzled places do not
// coalesce: about 30 L2 requests per warp instruction against 4 for linear
// destinations, measured; and a tensor copy with the 64-byte swizzle pads a
// box whose rows are the planar layout's 16 bytes.)  One thread issues a
// tile's 32 MMAs into the accumulator the block keeps over all its tiles;
// meanwhile the block's threads sum dz over the tile's own rows for db (one
// pixel each).  At the end warps 0-2 read the accumulator
// (lane 32 dx + ci) and add it to dW.  Every wait is bounded; a block that
// gives up flags the error word.
constexpr int kWtR = 4, kWtC = 128, kWtXP = kWtC + 4;       // rows, pixels per row, staged x pixels per row
constexpr int kWtXB = kWtR * kWtXP * 64;                    // staged x bytes
constexpr int kWtZB = (kWtR + 2) * kWtC * 64;               // staged dz bytes
constexpr int kWtStage = kWtXB + kWtZB;
constexpr size_t kWtSmem = 2 * (size_t)kWtStage + 1024;
static_assert(kWtXB % 1024 == 0 && kWtStage % 1024 == 0, "staged regions start on the swizzle period");
static_assert(kWtSmem <= 227 * 1024, "two stages must fit in shared memory");
// kind::f16, fp32 accumulator, bf16 A and B, both MN-major, N = 96, M = 128
constexpr uint32_t kWtIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((96u >> 3) << 17) | ((128u >> 4) << 24);

// 64-byte swizzle of a byte offset from a 1024-byte-aligned base: the 16-byte
// chunk index (bits 4-5) XOR bits 7-8.
__device__ __forceinline__ uint32_t swz64(uint32_t off) { return off ^ (((off >> 7) & 3u) << 4); }
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start, leading (MN block) and stride (K block) byte offsets in 16-byte
  // units, descriptor version 1, layout type 4 (64-byte swizzle), base offset 0
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46) | (4ull << 61);
}

constexpr int kWtThreads = 512;
constexpr int kWtXC = 4 * kWtR * kWtXP, kWtZC = 4 * (kWtR + 2) * kWtC;  // 16-byte chunks of a tile's x and dz
constexpr int kWtPre = (kWtXC + kWtZC + kWtThreads - 1) / kWtThreads;   // chunks per thread
__global__ void __launch_bounds__(kWtThreads, 1) k_conv_wgrad_tc(const __nv_bfloat16 *__restrict__ x,
                                                                 const __nv_bfloat16 *__restrict__ dz,
                                                                 float *__restrict__ dw, float *__restrict__ db,
                                                                 int nimg, int H, int W, int *err) {
  extern __shared__ unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ float s_db[32];
  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(s_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *gbase = s_raw + (base - raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntx = (W + kWtC - 1) / kWtC, tpi = ntx * ((H + kWtR - 1) / kWtR), ntiles = tpi * nimg;
  const long long HWp = (long long)H * W;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
  if (tid == 0) {
    s_abort = 0;
    tc_mbar_init(bar0, 1);
    tc_mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) s_db[tid] = 0.f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        (uint32_t)__cvta_generic_to_shared(&s_tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  auto origin = [&](int tt, int &img, int &y0, int &x0) {
    img = tt / tpi;
    const int rem = tt - img * tpi, ty = rem / ntx;
    y0 = ty * kWtR;
    x0 = (rem - ty * ntx) * kWtC;
  };
  // chunk e of a tile: x chunks [group][row][pixel], then dz chunks [group][row][pixel]
  // (consecutive lanes read consecutive pixels of one group plane); its
  // global offset (in 16-byte units, -1 outside the image) and its shared-memory byte offset
  auto chunk = [&](int e, int img, int y0, int x0, long long &g, uint32_t &o) {
    int n, r, i, yy, xx;
    bool ok;
    if (e < kWtXC) {
      n = e / (kWtR * kWtXP);
      const int rem = e - n * (kWtR * kWtXP);
      r = rem / kWtXP;
      i = rem - r * kWtXP;
      yy = y0 + r;
      xx = x0 - 1 + i;
      ok = yy < H && xx >= 0 && xx < W;
      o = swz64((uint32_t)((r * kWtXP + i) * 64 + n * 16));
    } else {
      const int e2 = e - kWtXC;
      n = e2 / ((kWtR + 2) * kWtC);
      const int rem = e2 - n * ((kWtR + 2) * kWtC);
      r = rem / kWtC;
      i = rem - r * kWtC;
      yy = y0 - 1 + r;
      xx = x0 + i;
      ok = yy >= 0 && yy < H && xx < W;
      o = kWtXB + swz64((uint32_t)((r * kWtC + i) * 64 + n * 16));
    }
    g = ok ? ((long long)img * 4 + n) * HWp + (long long)yy * W + xx : -1;
  };
  // this thread's chunks of tile tt into registers (loads left in flight)
  auto load = [&](int tt, uint4 *v) {
    int img, y0, x0;
    origin(tt, img, y0, x0);
#pragma unroll
    for (int j = 0; j < kWtPre; ++j) {
      const int e = tid + kWtThreads * j;
      v[j] = make_uint4(0u, 0u, 0u, 0u);
      if (e < kWtXC + kWtZC) {
        long long g;
        uint32_t o;
        chunk(e, img, y0, x0, g, o);
        if (g >= 0) v[j] = __ldg(reinterpret_cast<const uint4 *>(e < kWtXC ? x : dz) + g);
      }
    }
  };
  auto store = [&](int tt, int sb, const uint4 *v) {
    int img, y0, x0;
    origin(tt, img, y0, x0);
    unsigned char *st = gbase + sb * kWtStage;
#pragma unroll
    for (int j = 0; j < kWtPre; ++j) {
      const int e = tid + kWtThreads * j;
      if (e < kWtXC + kWtZC) {
        long long g;
        uint32_t o;
        chunk(e, img, y0, x0, g, o);
        *reinterpret_cast<uint4 *>(st + o) = v[j];
      }
    }
  };
  float bsum[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) bsum[c] = 0.f;
  uint4 v[kWtPre];
  int k = 0;
  if ((int)blockIdx.x < ntiles) {
    load(blockIdx.x, v);
    store(blockIdx.x, 0, v);
  }
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x, ++k) {
    const int sb = k & 1, tn = tt + gridDim.x;
    if (tn < ntiles) load(tn, v);  // in flight while tile k is multiplied
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // this thread's stores, to the tensor cores
    __syncthreads();                                               // tile k is staged
    const uint32_t X = base + sb * kWtStage, Z = X + kWtXB;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t a0 = umma_desc_sw64(X, 64, 512), b0 = umma_desc_sw64(Z, kWtC * 64, 512);
#pragma unroll
      for (int r = 0; r < kWtR; ++r)
#pragma unroll
        for (int c = 0; c < kWtC / 16; ++c) {
          const uint64_t ad = a0 + (uint64_t)(((r * kWtXP + 16 * c) * 64) >> 4);
          const uint64_t bd = b0 + (uint64_t)(((r * kWtC + 16 * c) * 64) >> 4);
          const uint32_t acc = (k > 0 || r > 0 || c > 0) ? 1u : 0u;
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem), "l"(ad), "l"(bd),
                       "r"(kWtIdesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar0 + 8 * sb)
                   : "memory");
    }
    // db: dz of the tile's own rows (staged rows 1 .. 4), one pixel per thread
    static_assert(kWtThreads == kWtR * kWtC, "one pixel of the tile per thread");
    const unsigned char *zg = gbase + sb * kWtStage + kWtXB;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const uint4 q = *reinterpret_cast<const uint4 *>(zg + swz64((uint32_t)((kWtC + tid) * 64 + n * 16)));
      const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(h2[e]);
        bsum[8 * n + 2 * e] += f.x;
        bsum[8 * n + 2 * e + 1] += f.y;
      }
    }
    if (tn < ntiles) {
      // stage sb ^ 1 is free once tile k - 1's MMAs are done (its sums were
      // read before this iteration's barrier)
      if (k >= 1 && tid == 0) tc_wait(bar0 + 8 * (sb ^ 1), ((k - 1) >> 1) & 1, &s_abort);
      __syncthreads();
      if (s_abort) break;
      store(tn, sb ^ 1, v);
    }
  }
  if (k > 0 && tid == 0 && !s_abort) tc_wait(bar0 + 8 * ((k - 1) & 1), ((k - 1) >> 1) & 1, &s_abort);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = !s_abort;
  if (ok && k > 0 && warp < 3) {  // lanes 32 dx + ci; column 32 (2 - dy) + co
#pragma unroll 1
    for (int c0 = 0; c0 < 96; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      const int dyy = 2 - c0 / 32;
#pragma unroll
      for (int c = 0; c < 32; ++c) atomicAdd(dw + ((3 * dyy + warp) * 32 + c) * 32 + lane, v[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float v = bsum[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(&s_db[c], v);
  }
  __syncthreads();
  if (ok && tid < 32) atomicAdd(db + tid, s_db[tid]);
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// Weight and bias gradients of the two one-channel end layers, without
// widening the one channel to 32:
//   first layer:  dW1[tap][co] = sum_p dz1[co][p] x0[p + off(tap)],   db1[co] = sum_p dz1[co][p]
//   last layer:   dW5[tap][ci] = sum_q dy[q - off(tap)] x4[ci][q],    db5 = sum_q dy[q]
// (the last layer's sum re-indexed by q = p + off(tap); the zero padding
// makes both sums run over the image).  Each is a GEMM over the pixels,
// D[tap][c] = sum_p A[tap][p] B[p][c], on mma.sync m16n8k16: M = the 9 taps
// (row 9 all ones for db1, rows 10-15 zero), N = the 32 channels, K = 16
// pixels of a row.  A is the im2col of the one-channel image u (x0, or dy
// rounded to bf16), gathered from its staged halo straight into the A
// fragments; B is the 32-channel operand v (dz1, or x4), staged as it lies
// in global memory (channel-group planar) by 16-byte cp.async copies and read
// with ldmatrix.trans.  db5 is the centre tap's row times a column of ones.
// Persistent blocks of 4 warps walk tiles of 4 rows x 128 pixels (one warp
// per row), double-buffered: tile k + 1's copies and halo loads are in flight
// while tile k is multiplied.  A block sums its warps' partial results in
// shared memory and adds them to the fp32 gradient once.
constexpr int kW1R = 4, kW1C = 128;                       // tile rows, columns
constexpr int kW1HW = kW1C + 2, kW1HP = (kW1R + 2) * kW1HW;  // halo columns, halo values
constexpr int kW1P = 144;                                 // halo row pitch (conflict-free gathers)
constexpr int kW1Pre = (kW1HP + 127) / 128;               // halo values per thread
constexpr int kW1V = 4 * kW1R * kW1C * 8;                 // bf16 of a staged v tile: [group][row][px][8]
constexpr int kW1Red = 9 * 32 + 32;                       // dW [tap][32], then db
constexpr size_t kW1Smem = sizeof(__nv_bfloat16) * 2 * kW1V + sizeof(uint16_t) * 2 * (kW1R + 2) * kW1P +
                           sizeof(float) * kW1Red;

__device__ __forceinline__ uint16_t to_bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16(v)); }
__device__ __forceinline__ uint16_t to_bf16_bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }

template <bool kFirst, typename TU>
__global__ void __launch_bounds__(128) k_conv_wgrad1(const TU *__restrict__ u, const __nv_bfloat16 *__restrict__ v,
                                                     float *__restrict__ dw, float *__restrict__ db, int nimg, int H,
                                                     int W) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  __nv_bfloat16 *s_v = reinterpret_cast<__nv_bfloat16 *>(s_raw);                  // [2][kW1V]
  uint16_t *s_u = reinterpret_cast<uint16_t *>(s_v + 2 * kW1V);                     // [2][(kW1R + 2) * kW1P]
  float *s_red = reinterpret_cast<float *>(s_u + 2 * (kW1R + 2) * kW1P);            // [kW1Red]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int lj = lane >> 3, lr = lane & 7;  // ldmatrix: matrix and row of this lane's address
  const int ntx = (W + kW1C - 1) / kW1C, tpi = ntx * ((H + kW1R - 1) / kW1R), ntiles = tpi * nimg;
  const long long HWp = (long long)H * W;
  for (int i = tid; i < kW1Red; i += 128) s_red[i] = 0.f;
  // halo offsets of this lane's A rows: tap g, and tap 8 (g = 0); the last
  // layer reads u at q - off(tap), the mirrored tap
  const int tg = kFirst ? g : 8 - g;
  const int oT = (tg / 3) * kW1P + tg % 3, o8 = kFirst ? 2 * kW1P + 2 : 0;
  const uint32_t ones = 0x3F803F80u;  // bf16 1.0 pair
  auto origin = [&](int tt, int &img, int &y0, int &x0) {
    img = tt / tpi;
    const int rem = tt - img * tpi, ty = rem / ntx;
    y0 = ty * kW1R;
    x0 = (rem - ty * ntx) * kW1C;
  };
  auto stage_v = [&](int img, int y0, int x0, int b) {
    __nv_bfloat16 *dst = s_v + b * kW1V;
#pragma unroll 4
    for (int i = tid; i < 4 * kW1R * kW1C; i += 128) {
      const int n = i / (kW1R * kW1C), r = (i / kW1C) % kW1R, px = i % kW1C;
      const bool ok = y0 + r < H && x0 + px < W;
      const __nv_bfloat16 *src = ok ? v + (((long long)img * 4 + n) * HWp + (long long)(y0 + r) * W + x0 + px) * 8 : v;
      cp_async16((uint32_t)__cvta_generic_to_shared(dst + (size_t)i * 8), src, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto fetch_u = [&](int img, int y0, int x0, uint16_t *h) {
    const TU *src = u + (long long)img * HWp;
#pragma unroll
    for (int k = 0; k < kW1Pre; ++k) {
      const int i = tid + 128 * k, r = i / kW1HW;
      const int yy = y0 + r - 1, xx = x0 + (i - r * kW1HW) - 1;
      h[k] = (i < kW1HP && (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W)
                 ? to_bf16_bits(src[(long long)yy * W + xx])
                 : (uint16_t)0;
    }
  };
  auto park_u = [&](const uint16_t *h, int b) {
#pragma unroll
    for (int k = 0; k < kW1Pre; ++k) {
      const int i = tid + 128 * k, r = i / kW1HW;
      if (i < kW1HP) s_u[b * (kW1R + 2) * kW1P + r * kW1P + (i - r * kW1HW)] = h[k];
    }
  };
  float acc[4][4], accb[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    accb[n] = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[n][r] = 0.f;
  }
  uint16_t h[kW1Pre];
  int img = 0, y0 = 0, x0 = 0;
  if ((int)blockIdx.x < ntiles) {
    origin(blockIdx.x, img, y0, x0);
    stage_v(img, y0, x0, 0);
    fetch_u(img, y0, x0, h);
    park_u(h, 0);
  }
  int b = 0;
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x, b ^= 1) {
    const int tn = tt + gridDim.x;
    int img_n = 0, y0_n = 0, x0_n = 0;
    if (tn < ntiles) {
      origin(tn, img_n, y0_n, x0_n);
      stage_v(img_n, y0_n, x0_n, b ^ 1);
      fetch_u(img_n, y0_n, x0_n, h);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // tile tt's v and u are staged
    if (y0 + warp < H) {
      const uint16_t *ur = s_u + b * (kW1R + 2) * kW1P + warp * kW1P + 2 * t;
      const __nv_bfloat16 *vr = s_v + b * kW1V + warp * kW1C * 8;
      const int nx = min(kW1C, W - x0);
#pragma unroll 2
      for (int c0 = 0; c0 < nx; c0 += 16) {
        uint32_t a[4];
        a[0] = pack_u16(ur[c0 + oT], ur[c0 + oT + 1]);
        a[2] = pack_u16(ur[c0 + oT + 8], ur[c0 + oT + 9]);
        const uint32_t r8a = pack_u16(ur[c0 + o8], ur[c0 + o8 + 1]), r8b = pack_u16(ur[c0 + o8 + 8], ur[c0 + o8 + 9]);
        const uint32_t rone = kFirst && g == 1 ? ones : 0u;
        a[1] = g == 0 ? r8a : rone;
        a[3] = g == 0 ? r8b : rone;
        uint32_t bf[4][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {  // channel groups 2q, 2q + 1; pixels 0-7 | 8-15
          uint32_t r4[4];
          ldsm_x4_t(r4, vr + ((2 * q + (lj >> 1)) * kW1R * kW1C + c0 + (lj & 1) * 8 + lr) * 8);
          bf[2 * q][0] = r4[0];
          bf[2 * q][1] = r4[1];
          bf[2 * q + 1][0] = r4[2];
          bf[2 * q + 1][1] = r4[3];
        }
#pragma unroll
        for (int n = 0; n < 4; ++n) mma16816(acc[n], a, bf[n]);
        if (!kFirst) {
          const uint32_t bo[2] = {ones, ones};
          mma16816(accb, a, bo);
        }
      }
    }
    if (tn < ntiles) {
      park_u(h, b ^ 1);
      img = img_n;
      y0 = y0_n;
      x0 = x0_n;
    }
    __syncthreads();  // buffer b is refilled by the copies two tiles on
  }
  // D rows: tap g (acc[n][0..1]) and row g + 8 (acc[n][2..3]): tap 8 for
  // g = 0, the ones row (db1) for g = 1; columns 8n + 2t, 8n + 2t + 1
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int c = 8 * n + 2 * t;
    atomicAdd(&s_red[g * 32 + c], acc[n][0]);
    atomicAdd(&s_red[g * 32 + c + 1], acc[n][1]);
    if (g == 0 || (kFirst && g == 1)) {
      atomicAdd(&s_red[(8 + g) * 32 + c], acc[n][2]);
      atomicAdd(&s_red[(8 + g) * 32 + c + 1], acc[n][3]);
    }
  }
  if (!kFirst && g == 4 && t == 0) atomicAdd(&s_red[9 * 32], accb[0]);  // centre tap x ones: db5
  __syncthreads();
  for (int i = tid; i < 9 * 32; i += 128) atomicAdd(dw + i, s_red[i]);
  if (kFirst) {
    if (tid < 32) atomicAdd(db + tid, s_red[9 * 32 + tid]);
  } else if (tid == 0) {
    atomicAdd(db, s_red[9 * 32]);
  }
}

// fp32 master weights -> bf16 compute weights: forward copies and the
// mirrored / transposed copies for the backward-data pass.
__global__ void k_prep_weights(const float *__restrict__ prm, __nv_bfloat16 *__restrict__ wf, __nv_bfloat16 *__restrict__ wb) {
  // forward: same layout as the master; backward: layer l's [t][co][ci] ->
  // [8 - t][ci][co] (only layers 2..5 are needed backwards)
  const int offs[5] = {kW1, kW2, kW3, kW4, kW5};
  const int cin[5] = {1, C, C, C, C}, cout[5] = {C, C, C, C, 1};
  for (int l = 0; l < 5; ++l) {
    const int n = 9 * cin[l] * cout[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const float v = prm[offs[l] + i];
      wf[offs[l] + i] = __float2bfloat16(v);
      const int ci = i % cin[l], co = (i / cin[l]) % cout[l], t = i / (cin[l] * cout[l]);
      wb[offs[l] + ((8 - t) * cin[l] + ci) * cout[l] + co] = __float2bfloat16(v);
    }
  }
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// loss = mean((y - t)^2) (fp64 accumulate); dy = 2 (y - t) / n
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, long long n, float *__restrict__ dy,
                      double *loss) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    if (dy) dy[i] = 2.f * d / (float)n;
    acc += (double)d * d;
  }
  // one atomic per block (atomics of every warp on one address serialise)
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) atomicAdd(loss, acc / (double)n);
  }
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

void set_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_conv_tc<kHidden, kTcR>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(kTcR));
  cudaFuncSetAttribute(k_conv_tc<kBackData, kTcR>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(kTcR));
  cudaFuncSetAttribute(k_conv_tc<kLast, kTcR>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(kTcR));
  cudaFuncSetAttribute(k_conv_tc<kFused, kTcR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tc_smem_mode(kFused, kTcR));
  cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWtSmem);
  cudaFuncSetAttribute(k_conv_wgrad1<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW1Smem);
  cudaFuncSetAttribute(k_conv_wgrad1<true, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW1Smem);
  done = true;
}

// Persistent grid of the tcgen05 weight-gradient kernel: one block per SM (its shared memory).
int grid_wgrad_tc(int nimg, int H, int W) {
  static int sms = 0;
  if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const long long tiles = (long long)((W + kWtC - 1) / kWtC) * ((H + kWtR - 1) / kWtR) * nimg;
  return (int)(tiles < sms ? tiles : sms);
}

// Persistent grid of the one-channel weight-gradient kernel (attributes set by set_attrs).
template <bool kFirst, typename TU>
int grid_wgrad1(int nimg, int H, int W) {
  static int slots = 0;
  if (!slots) {
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_wgrad1<kFirst, TU>, 128, kW1Smem);
    slots = sms * (per > 0 ? per : 1);
  }
  const long long tiles = (long long)((W + kW1C - 1) / kW1C) * ((H + kW1R - 1) / kW1R) * nimg;
  return (int)(tiles < slots ? tiles : slots);
}

// Persistent grid of the one-channel kernel: its resident blocks, at most one per tile.
template <int MODE>
int grid_1to32(int nimg, int H, int W) {
  static int slots = 0;
  if (!slots) {
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (smem_1to32<MODE>() > 48 * 1024)
      cudaFuncSetAttribute(k_conv_1to32<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_1to32<MODE>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv_1to32<MODE>, 256, smem_1to32<MODE>());
    slots = sms * (per > 0 ? per : 1);
  }
  const long long tiles = (long long)((W + kM1C - 1) / kM1C) * ((H + kM1R - 1) / kM1R) * nimg;
  return (int)(tiles < slots ? tiles : slots);
}


int grid_of(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// Workspace layout (bytes): bf16 weights fwd, bf16 weights bwd, x (bf16),
// four hidden activations (bf16, 32 ch), two 32-channel gradient buffers
// (bf16) and the last-layer output gradient (bf16).
struct Ws {
  __nv_bfloat16 *wf, *wb, *x0, *act[4], *dz[2], *dy1;
};

size_t ws_bytes(long long npx) {
  return sizeof(__nv_bfloat16) * (2 * (size_t)kNParams + 256 + (size_t)npx * (1 + 4 * C + 2 * C + 1)) + 1024;
}

Ws carve(void *ws, long long npx) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char *p = static_cast<char *>(ws);
  Ws w;
  w.wf = reinterpret_cast<__nv_bfloat16 *>(p); p += al(sizeof(__nv_bfloat16) * kNParams);
  w.wb = reinterpret_cast<__nv_bfloat16 *>(p); p += al(sizeof(__nv_bfloat16) * kNParams);
  w.x0 = reinterpret_cast<__nv_bfloat16 *>(p); p += al(sizeof(__nv_bfloat16) * npx);
  for (int l = 0; l < 4; ++l) { w.act[l] = reinterpret_cast<__nv_bfloat16 *>(p); p += al(sizeof(__nv_bfloat16) * npx * C); }
  for (int l = 0; l < 2; ++l) { w.dz[l] = reinterpret_cast<__nv_bfloat16 *>(p); p += al(sizeof(__nv_bfloat16) * npx * C); }
  w.dy1 = reinterpret_cast<__nv_bfloat16 *>(p);
  return w;
}

// Error word of the tensor-core kernels' bounded waits (mapped host memory,
// read at the next call).
int *tc_err_host = nullptr, *tc_err_dev = nullptr;

int tc_err() {
  if (!tc_err_host) {
    if (cudaHostAlloc((void **)&tc_err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&tc_err_dev, tc_err_host, 0) != cudaSuccess) {
      tc_err_host = nullptr;
      return rbc::set_error(RBC_ENOMEM, "error word allocation failed");
    }
    *tc_err_host = 0;
  }
  if (*(volatile int *)tc_err_host) {
    *(volatile int *)tc_err_host = 0;
    return rbc::set_error(RBC_ETIMEOUT, "a tensor-core convolution gave up waiting for its MMAs; results of the "
                                        "calls since the last check are invalid");
  }
  return RBC_OK;
}

// 4-D tensor map over a channel-group planar bf16 activation buffer (32
// channels) seen as 8-byte elements: dims (2 W elements of a row -- two per
// pixel --, y, group, image); box (256 = 128 pixels, by rows, 4 groups, 1).
bool act_map(CUtensorMap *m, const __nv_bfloat16 *buf, int nimg, int H, int W, int by) {
  auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(rbc::tmap_encode_fn());
  if (!fn) return false;
  cuuint64_t dims[4] = {2 * (cuuint64_t)W, (cuuint64_t)H, 4, (cuuint64_t)nimg};
  cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)W * H * 16, (cuuint64_t)W * H * 64};
  cuuint32_t box[4] = {2 * kTcHW, (cuuint32_t)by, 4, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<__nv_bfloat16 *>(buf), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
bool launch_conv_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias, const __nv_bfloat16 *mask,
                    __nv_bfloat16 *out, int nimg, int H, int W, cudaStream_t s, float *out_f = nullptr,
                    const float *resid = nullptr) {
  static int sms = 0;
  if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const long long tiles = (long long)((W + kTcOut - 1) / kTcOut) * ((H + kTcR - 1) / kTcR) * nimg;
  const int grid = (int)(tiles < sms ? tiles : sms);
  CUtensorMap tin;
  if (!act_map(&tin, in, nimg, H, W, kTcR + 2)) return false;
  k_conv_tc<MODE, kTcR><<<grid, tc_threads(MODE), tc_smem(kTcR), s>>>(tin, wt, bias, mask, out, out_f, resid, nimg,
                                                                      H, W, tc_err_dev);
  return true;
}

// The first two layers in one launch (kFused): x (fp32) -> act1.
void launch_conv_fused(const float *x, const __nv_bfloat16 *w1, const float *b1, const __nv_bfloat16 *w2,
                       const float *b2, __nv_bfloat16 *out, int nimg, int H, int W, cudaStream_t s) {
  static int sms = 0;
  if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const long long tiles = (long long)((W + kTcOut - 1) / kTcOut) * ((H + kTcR - 1) / kTcR) * nimg;
  const int grid = (int)(tiles < sms ? tiles : sms);
  CUtensorMap unused;  // the fused mode builds its operand instead of copying it
  memset(&unused, 0, sizeof unused);
  k_conv_tc<kFused, kTcR><<<grid, tc_threads(kFused), tc_smem_mode(kFused, kTcR), s>>>(
      unused, w2, b2, nullptr, out, nullptr, nullptr, nimg, H, W, tc_err_dev, x, w1, b1);
}

// The network's forward pass; `keep` stores what the backward pass reads
// (the bf16 input and the first layer's output: two launches for the first
// two layers); without it the first two layers are one fused launch.
int cnn_forward(const float *params_dev, int nimg, int H, int W, const float *x_dev, float *y_dev, void *ws_dev,
                void *stream, bool keep, const char *who) {
  if (!params_dev || !x_dev || !y_dev || !ws_dev || nimg < 1 || H < 1 || W < 1)
    return rbc::set_error(RBC_EINVAL, who);
  if (int rc = tc_err()) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const long long npx = (long long)nimg * H * W;
  Ws w = carve(ws_dev, npx);
  k_prep_weights<<<36, 256, 0, s>>>(params_dev, w.wf, w.wb);
  if (keep) k_to_bf16<<<grid_of(npx), 256, 0, s>>>(x_dev, w.x0, npx);
  set_attrs();
  bool ok_tc = true;
  if (keep) {  // the backward pass reads the first layer's output
    k_conv_1to32<kHidden><<<grid_1to32<kHidden>(nimg, H, W), 256, smem_1to32<kHidden>(), s>>>(
        w.x0, w.wf + kW1, params_dev + kB1, nullptr, w.act[0], nimg, H, W);
    ok_tc = launch_conv_tc<kHidden>(w.act[0], w.wf + kW2, params_dev + kB2, nullptr, w.act[1], nimg, H, W, s);
  } else {
    launch_conv_fused(x_dev, w.wf + kW1, params_dev + kB1, w.wf + kW2, params_dev + kB2, w.act[1], nimg, H, W, s);
  }
  ok_tc = ok_tc && launch_conv_tc<kHidden>(w.act[1], w.wf + kW3, params_dev + kB3, nullptr, w.act[2], nimg, H, W, s);
  ok_tc = ok_tc && launch_conv_tc<kHidden>(w.act[2], w.wf + kW4, params_dev + kB4, nullptr, w.act[3], nimg, H, W, s);
  ok_tc = ok_tc && launch_conv_tc<kLast>(w.act[3], w.wf + kW5, params_dev + kB5, nullptr, nullptr, nimg, H, W, s,
                                         y_dev, x_dev);
  if (!ok_tc) return rbc::set_error(RBC_ECUDA, "rbc_cnn_forward: launch failed");
  rbc::add_launches(keep ? 7 : 5);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

} // namespace

extern "C" {

long long rbc_cnn_param_count(void) { return kNParams; }

long long rbc_cnn_workspace_bytes(int nimg, int H, int W) { return (long long)ws_bytes((long long)nimg * H * W); }

int rbc_cnn_forward(const float *params_dev, int nimg, int H, int W, const float *x_dev, float *y_dev, void *ws_dev,
                    void *stream) {
  return cnn_forward(params_dev, nimg, H, W, x_dev, y_dev, ws_dev, stream, true, "rbc_cnn_forward: bad arguments");
}

int rbc_cnn_infer(const float *params_dev, int nimg, int H, int W, const float *x_dev, float *y_dev, void *ws_dev,
                  void *stream) {
  return cnn_forward(params_dev, nimg, H, W, x_dev, y_dev, ws_dev, stream, false, "rbc_cnn_infer: bad arguments");
}

int rbc_cnn_backward(const float *params_dev, int nimg, int H, int W, const float *dy_dev, float *grad_dev, void *ws_dev,
                     void *stream) {
  if (!params_dev || !dy_dev || !grad_dev || !ws_dev || nimg < 1 || H < 1 || W < 1)
    return rbc::set_error(RBC_EINVAL, "rbc_cnn_backward: bad arguments");
  if (int rc = tc_err()) return rc;
  set_attrs();
  cudaStream_t s = (cudaStream_t)stream;
  const long long npx = (long long)nimg * H * W;
  Ws w = carve(ws_dev, npx);  // activations from the preceding rbc_cnn_forward

  // layer 5: dW5, db5 from dy; dz4 = conv^T(dy) masked by act4 > 0
  k_conv_wgrad1<false, float><<<grid_wgrad1<false, float>(nimg, H, W), 128, kW1Smem, s>>>(
      dy_dev, w.act[3], grad_dev + kW5, grad_dev + kB5, nimg, H, W);
  k_to_bf16<<<grid_of(npx), 256, 0, s>>>(dy_dev, w.dy1, npx);
  set_attrs();
  k_conv_1to32<kBackData><<<grid_1to32<kBackData>(nimg, H, W), 256, smem_1to32<kBackData>(), s>>>(
      w.dy1, w.wb + kW5, nullptr, w.act[3], w.dz[0], nimg, H, W);
  // layers 4, 3, 2: dW from dz; dz below = conv^T(dz) masked
  int cur = 0;
  bool ok_tc = true;
  const int woff[3] = {kW4, kW3, kW2}, boff[3] = {kB4, kB3, kB2};
  for (int l = 0; l < 3; ++l) {
    const int layer_in = 2 - l;  // act index of this layer's input: act3 (l=0) ... act1
    k_conv_wgrad_tc<<<grid_wgrad_tc(nimg, H, W), kWtThreads, kWtSmem, s>>>(w.act[layer_in], w.dz[cur], grad_dev + woff[l],
                                                                     grad_dev + boff[l], nimg, H, W, tc_err_dev);
    ok_tc = ok_tc && launch_conv_tc<kBackData>(w.dz[cur], w.wb + woff[l], nullptr, w.act[layer_in], w.dz[1 - cur], nimg, H, W, s);
    cur = 1 - cur;
  }
  // layer 1
  k_conv_wgrad1<true, __nv_bfloat16><<<grid_wgrad1<true, __nv_bfloat16>(nimg, H, W), 128, kW1Smem, s>>>(
      w.x0, w.dz[cur], grad_dev + kW1, grad_dev + kB1, nimg, H, W);
  if (!ok_tc) return rbc::set_error(RBC_ECUDA, "rbc_cnn_backward: launch failed");
  rbc::add_launches(10);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

int rbc_cnn_mse(const float *y_dev, const float *t_dev, long long n, float *dy_dev, double *loss_dev, void *stream) {
  if (!y_dev || !t_dev || !loss_dev || n < 1) return rbc::set_error(RBC_EINVAL, "rbc_cnn_mse: bad arguments");
  k_mse<<<grid_of(n), 256, 0, (cudaStream_t)stream>>>(y_dev, t_dev, n, dy_dev, loss_dev);
  rbc::add_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

int rbc_cnn_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, float lr, float b1, float b2,
                 float eps, int step, void *stream) {
  if (!params_dev || !grad_dev || !m_dev || !v_dev || step < 1) return rbc::set_error(RBC_EINVAL, "rbc_cnn_adam: bad arguments");
  // bias corrections formed in fp64: 1 - b2^step cancels badly in fp32 at small steps
  const float c1 = (float)(1.0 - pow((double)b1, (double)step)), c2 = (float)(1.0 - pow((double)b2, (double)step));
  k_adam<<<grid_of(kNParams), 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, kNParams, lr, b1, b2,
                                                              eps, c1, c2);
  rbc::add_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

} // extern "C"
