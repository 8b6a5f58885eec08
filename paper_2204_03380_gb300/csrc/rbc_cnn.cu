// rbc_cnn.cu -- the learned random-boundary-noise denoiser: a 5-layer 3x3
// CNN (1 -> 32 -> 32 -> 32 -> 32 -> 1 channels, ReLU after layers 1-4, the
// input added to the last layer's output), bf16 operands with fp32
// accumulation.  Not in the paper: it stands in for stacking many random
// boundary realizations of an RTM image (Section 4.3's noise is incoherent
// between realizations).
//
// Activations are NHWC bf16 ([image][row][col][channel]); weights are stored
// [tap][out][in] (tap = 3 * dy + dx, dy, dx in 0..2 for offsets -1..1).
// Convolutions run as implicit GEMMs on the tensor cores (mma.sync
// m16n8k16, bf16 in, fp32 accumulate): a block computes an 8 x 32 pixel tile
// for all output channels, one warp per tile row (two 16-pixel m tiles),
// with the input halo tile and the weights staged in shared memory.  The
// backward pass of the input is the same kernel with the taps mirrored and
// the channel roles swapped, its epilogue applying the ReLU mask of the
// layer below.  Weight gradients are per-tap GEMMs over the pixels, also on
// the tensor cores, reduced by persistent blocks and added to the fp32
// gradient once per block.
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/rbc.h"
#include "rbc_internal.cuh"

namespace rbc {
int set_error(int code, const char *msg);  // rbc_abi.cu
void add_launches(long long n);
}

namespace {

constexpr int TH = 8, TW = 32;  // output tile: 8 rows x 32 columns, one warp per row
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

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

enum { kHidden = 0, kLast = 1, kBackData = 2 };

// Implicit-GEMM 3x3 convolution with zero padding.
//   CIN in {1, 32}, COUT in {1, 32}.  in: NHWC bf16 with CIN channels.
//   wt: bf16 weights [9][COUT][CIN] (already mirrored / transposed for the
//   backward-data pass).
//   MODE kHidden:   out_bf = relu(conv + bias)                (bf16, COUT ch)
//   MODE kLast:     out_f  = resid + conv + bias              (fp32, COUT = 1)
//   MODE kBackData: out_bf = conv * (mask > 0)                (bf16, COUT ch)
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(256) k_conv3x3(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ wt,
                                                 const float *__restrict__ bias, const float *__restrict__ resid,
                                                 const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ out_bf,
                                                 float *__restrict__ out_f, int H, int W) {
  constexpr int CP = (CIN == 32) ? 40 : 2;      // padded channel stride in shared memory (bank spread)
  constexpr int NT = (COUT == 32) ? 4 : 1;      // n tiles of 8 output channels
  constexpr int NW = NT * 8;                    // padded output channels
  constexpr int KP = (CIN == 32) ? 40 : 16;     // padded K per tap (CIN = 1: K is the 9 taps, padded to 16)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16 *s_in = reinterpret_cast<__nv_bfloat16 *>(smem_raw);                  // [(TH+2)(TW+2)][CP]
  __nv_bfloat16 *s_w = s_in + (TH + 2) * (TW + 2) * CP;                                // [taps][NW][KP]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int img = blockIdx.z;
  const int y0 = blockIdx.y * TH, x0 = blockIdx.x * TW;
  const long long ibase = (long long)img * H * W;
  // weights -> shared (zero padding for the n / k tails)
  if (CIN == 32) {
    for (int i = threadIdx.x; i < 9 * NW * KP; i += blockDim.x) {
      const int k = i % KP, n = (i / KP) % NW, t = i / (KP * NW);
      s_w[i] = (k < CIN && n < COUT) ? wt[(t * COUT + n) * CIN + k] : __float2bfloat16(0.f);
    }
  } else {
    for (int i = threadIdx.x; i < NW * KP; i += blockDim.x) {
      const int k = i % KP, n = i / KP;  // k = tap
      s_w[i] = (k < 9 && n < COUT) ? wt[k * COUT + n] : __float2bfloat16(0.f);
    }
  }
  // input halo tile -> shared (zero outside the image)
  for (int i = threadIdx.x; i < (TH + 2) * (TW + 2) * CIN; i += blockDim.x) {
    const int c = i % CIN, px = (i / CIN) % (TW + 2), py = i / (CIN * (TW + 2));
    const int yy = y0 + py - 1, xx = x0 + px - 1;
    s_in[(py * (TW + 2) + px) * CP + c] =
        (yy >= 0 && yy < H && xx >= 0 && xx < W) ? in[(ibase + (long long)yy * W + xx) * CIN + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[m][n][r] = 0.f;
  if (CIN == 32) {
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3, dx = t % 3;
#pragma unroll
      for (int kk = 0; kk < 32; kk += 16) {
        uint32_t b[NT][2];
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const __nv_bfloat16 *wp = s_w + (t * NW + n * 8 + g) * KP + kk + tig * 2;
          b[n][0] = *reinterpret_cast<const uint32_t *>(wp);
          b[n][1] = *reinterpret_cast<const uint32_t *>(wp + 8);
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const int px = m * 16 + g + dx;
          const __nv_bfloat16 *r0 = s_in + ((warp + dy) * (TW + 2) + px) * CP + kk + tig * 2;
          const __nv_bfloat16 *r1 = r0 + 8 * CP;
          uint32_t a[4];
          a[0] = *reinterpret_cast<const uint32_t *>(r0);
          a[1] = *reinterpret_cast<const uint32_t *>(r1);
          a[2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
          a[3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
#pragma unroll
          for (int n = 0; n < NT; ++n) mma16816(acc[m][n], a, b[n]);
        }
      }
    }
  } else {
    // CIN = 1: the K dimension is the tap index (9, padded to 16)
    uint32_t b[NT][2];
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const __nv_bfloat16 *wp = s_w + (n * 8 + g) * KP + tig * 2;
      b[n][0] = *reinterpret_cast<const uint32_t *>(wp);
      b[n][1] = *reinterpret_cast<const uint32_t *>(wp + 8);
    }
    auto tapv = [&](int px, int k) -> __nv_bfloat16 {
      if (k >= 9) return __float2bfloat16(0.f);
      return s_in[((warp + k / 3) * (TW + 2) + px + k % 3) * CP];
    };
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int px = m * 16 + g;
      const int k0 = tig * 2;
      uint32_t a[4];
      a[0] = pack2(tapv(px, k0), tapv(px, k0 + 1));
      a[1] = pack2(tapv(px + 8, k0), tapv(px + 8, k0 + 1));
      a[2] = pack2(tapv(px, k0 + 8), tapv(px, k0 + 9));
      a[3] = pack2(tapv(px + 8, k0 + 8), tapv(px + 8, k0 + 9));
#pragma unroll
      for (int n = 0; n < NT; ++n) mma16816(acc[m][n], a, b[n]);
    }
  }
  // epilogue: C fragment rows g / g + 8 (pixels), columns tig*2, +1 (channels)
  const int yy = y0 + warp;
  if (yy >= H) return;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int xx = x0 + m * 16 + g + half * 8;
      if (xx >= W) continue;
      const long long p = ibase + (long long)yy * W + xx;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int co = n * 8 + tig * 2;
        float v0 = acc[m][n][half * 2], v1 = acc[m][n][half * 2 + 1];
        if (MODE == kLast) {
          if (co == 0) out_f[p] = resid[p] + v0 + bias[0];
        } else if (co < COUT) {
          if (MODE == kHidden) {
            v0 = fmaxf(v0 + bias[co], 0.f);
            v1 = fmaxf(v1 + bias[co + 1], 0.f);
          } else {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + p * COUT + co);
            v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
            v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
          }
          *reinterpret_cast<__nv_bfloat162 *>(out_bf + p * COUT + co) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return sizeof(__nv_bfloat16) * ((TH + 2) * (TW + 2) * ((CIN == 32) ? 40 : 2) +
                                  (CIN == 32 ? 9 : 1) * ((COUT == 32) ? 32 : 8) * ((CIN == 32) ? 40 : 16));
}

// Weight and bias gradients of one layer, on the tensor cores:
//   dW[t][co][ci] += sum_p dz[p][co] x[p + off(t)][ci],  db[co] += sum_p dz[p][co]
// For every tap this is a GEMM with M = output channels, N = input channels
// and K = pixels; warp t of the block owns tap t.  The tile's dz (256 pixels)
// and x halo are staged channel-major in shared memory so that consecutive K
// (pixels) are adjacent.  dz: NHWC bf16 (COUT ch) or fp32 (dzf, COUT = 1).
// Persistent blocks walk 8 x 32 pixel tiles, keep the partial sums in
// registers and add them to dW / db once.
template <int CIN, int COUT>
__global__ void __launch_bounds__(288) k_conv_wgrad(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ dz,
                                                    const float *__restrict__ dzf, float *__restrict__ dw,
                                                    float *__restrict__ db, int nimg, int H, int W) {
  constexpr int MT = (COUT + 15) / 16, NT = (CIN + 7) / 8;
  constexpr int CM = MT * 16, CN = NT * 8;   // padded channel counts
  constexpr int HP = (TH + 2) * (TW + 2);    // halo pixels
  __shared__ __nv_bfloat16 s_x[CN * HP];     // [ci][halo pixel]
  __shared__ __nv_bfloat16 s_dz[CM * TH * TW];  // [co][pixel]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int dy = warp / 3, dx = warp % 3;    // this warp's tap
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[m][n][r] = 0.f;
  float bacc = 0.f;
  const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
  const long long ntiles = (long long)tx * ty * nimg;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int img = (int)(tile / ((long long)tx * ty));
    const int rem = (int)(tile % ((long long)tx * ty));
    const int y0 = (rem / tx) * TH, x0 = (rem % tx) * TW;
    const long long ibase = (long long)img * H * W;
    __syncthreads();
    for (int i = threadIdx.x; i < HP * CN; i += blockDim.x) {
      const int c = i % CN, hp = i / CN;
      const int yy = y0 + hp / (TW + 2) - 1, xx = x0 + hp % (TW + 2) - 1;
      s_x[c * HP + hp] = (c < CIN && yy >= 0 && yy < H && xx >= 0 && xx < W)
                             ? x[(ibase + (long long)yy * W + xx) * CIN + c] : zero;
    }
    for (int i = threadIdx.x; i < TH * TW * CM; i += blockDim.x) {
      const int c = i % CM, q = i / CM;
      const int yy = y0 + q / TW, xx = x0 + q % TW;
      __nv_bfloat16 v = zero;
      if (c < COUT && yy < H && xx < W) {
        const long long p = ibase + (long long)yy * W + xx;
        v = dzf ? __float2bfloat16(dzf[p]) : dz[p * COUT + c];
      }
      s_dz[c * TH * TW + q] = v;
    }
    __syncthreads();
    if (warp < 9) {
#pragma unroll 1
      for (int q0 = 0; q0 < TH * TW; q0 += 16) {
        const int row = q0 / TW, col0 = q0 % TW;
        uint32_t a[MT][4], b[NT][2];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          const __nv_bfloat16 *r0 = s_dz + (m * 16 + g) * TH * TW + q0 + tig * 2;
          const __nv_bfloat16 *r1 = r0 + 8 * TH * TW;
          a[m][0] = pack2(r0[0], r0[1]);
          a[m][1] = pack2(r1[0], r1[1]);
          a[m][2] = pack2(r0[8], r0[9]);
          a[m][3] = pack2(r1[8], r1[9]);
        }
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const __nv_bfloat16 *c0 = s_x + (n * 8 + g) * HP + (row + dy) * (TW + 2) + col0 + dx + tig * 2;
          b[n][0] = pack2(c0[0], c0[1]);
          b[n][1] = pack2(c0[8], c0[9]);
        }
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
          for (int n = 0; n < NT; ++n) mma16816(acc[m][n], a[m], b[n]);
      }
    }
    if (threadIdx.x < COUT) {
      float sb = 0.f;
      for (int q = 0; q < TH * TW; ++q) sb += __bfloat162float(s_dz[threadIdx.x * TH * TW + q]);
      bacc += sb;
    }
  }
  if (warp < 9) {
    const int t = warp;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < NT; ++n)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int co = m * 16 + g + (r >> 1) * 8, ci = n * 8 + tig * 2 + (r & 1);
          if (co < COUT && ci < CIN) atomicAdd(dw + (t * COUT + co) * CIN + ci, acc[m][n][r]);
        }
  }
  if (threadIdx.x < COUT) atomicAdd(db + threadIdx.x, bacc);
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
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)n);
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
  cudaFuncSetAttribute(k_conv3x3<C, C, kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<C, C>());
  cudaFuncSetAttribute(k_conv3x3<C, C, kBackData>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<C, C>());
  cudaFuncSetAttribute(k_conv3x3<C, 1, kLast>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem<C, 1>());
  done = true;
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

} // namespace

extern "C" {

long long rbc_cnn_param_count(void) { return kNParams; }

long long rbc_cnn_workspace_bytes(int nimg, int H, int W) { return (long long)ws_bytes((long long)nimg * H * W); }

int rbc_cnn_forward(const float *params_dev, int nimg, int H, int W, const float *x_dev, float *y_dev, void *ws_dev,
                    void *stream) {
  if (!params_dev || !x_dev || !y_dev || !ws_dev || nimg < 1 || H < 1 || W < 1)
    return rbc::set_error(RBC_EINVAL, "rbc_cnn_forward: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const long long npx = (long long)nimg * H * W;
  Ws w = carve(ws_dev, npx);
  k_prep_weights<<<36, 256, 0, s>>>(params_dev, w.wf, w.wb);
  k_to_bf16<<<grid_of(npx), 256, 0, s>>>(x_dev, w.x0, npx);
  set_attrs();
  const dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, nimg);
  k_conv3x3<1, C, kHidden><<<grid, 256, conv_smem<1, C>(), s>>>(w.x0, w.wf + kW1, params_dev + kB1, nullptr, nullptr,
                                                                w.act[0], nullptr, H, W);
  k_conv3x3<C, C, kHidden><<<grid, 256, conv_smem<C, C>(), s>>>(w.act[0], w.wf + kW2, params_dev + kB2, nullptr, nullptr,
                                                                w.act[1], nullptr, H, W);
  k_conv3x3<C, C, kHidden><<<grid, 256, conv_smem<C, C>(), s>>>(w.act[1], w.wf + kW3, params_dev + kB3, nullptr, nullptr,
                                                                w.act[2], nullptr, H, W);
  k_conv3x3<C, C, kHidden><<<grid, 256, conv_smem<C, C>(), s>>>(w.act[2], w.wf + kW4, params_dev + kB4, nullptr, nullptr,
                                                                w.act[3], nullptr, H, W);
  k_conv3x3<C, 1, kLast><<<grid, 256, conv_smem<C, 1>(), s>>>(w.act[3], w.wf + kW5, params_dev + kB5, x_dev, nullptr,
                                                              nullptr, y_dev, H, W);
  rbc::add_launches(7);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

int rbc_cnn_backward(const float *params_dev, int nimg, int H, int W, const float *dy_dev, float *grad_dev, void *ws_dev,
                     void *stream) {
  if (!params_dev || !dy_dev || !grad_dev || !ws_dev || nimg < 1 || H < 1 || W < 1)
    return rbc::set_error(RBC_EINVAL, "rbc_cnn_backward: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const long long npx = (long long)nimg * H * W;
  Ws w = carve(ws_dev, npx);  // activations from the preceding rbc_cnn_forward
  const dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, nimg);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int pg = 2 * sms;
  // layer 5: dW5, db5 from dy; dz4 = conv^T(dy) masked by act4 > 0
  k_conv_wgrad<C, 1><<<pg, 288, 0, s>>>(w.act[3], nullptr, dy_dev, grad_dev + kW5, grad_dev + kB5, nimg, H, W);
  k_to_bf16<<<grid_of(npx), 256, 0, s>>>(dy_dev, w.dy1, npx);
  set_attrs();
  k_conv3x3<1, C, kBackData><<<grid, 256, conv_smem<1, C>(), s>>>(w.dy1, w.wb + kW5, nullptr, nullptr, w.act[3], w.dz[0],
                                                                  nullptr, H, W);
  // layers 4, 3, 2: dW from dz; dz below = conv^T(dz) masked
  int cur = 0;
  const int woff[3] = {kW4, kW3, kW2}, boff[3] = {kB4, kB3, kB2};
  for (int l = 0; l < 3; ++l) {
    const int layer_in = 2 - l;  // act index of this layer's input: act3 (l=0) ... act1
    k_conv_wgrad<C, C><<<pg, 288, 0, s>>>(w.act[layer_in], w.dz[cur], nullptr, grad_dev + woff[l], grad_dev + boff[l],
                                           nimg, H, W);
    k_conv3x3<C, C, kBackData><<<grid, 256, conv_smem<C, C>(), s>>>(w.dz[cur], w.wb + woff[l], nullptr, nullptr,
                                                                     w.act[layer_in], w.dz[1 - cur], nullptr, H, W);
    cur = 1 - cur;
  }
  // layer 1
  k_conv_wgrad<1, C><<<pg, 288, 0, s>>>(w.x0, w.dz[cur], nullptr, grad_dev + kW1, grad_dev + kB1, nimg, H, W);
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
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<grid_of(kNParams), 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, kNParams, lr, b1, b2,
                                                              eps, c1, c2);
  rbc::add_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rbc::set_error(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}

} // extern "C"
