// rbc_internal.cuh -- shared device/host definitions of librbc (sm_103a).
//
// Internal wavefield layout ("pitched, zero-haloed"): a field of the padded
// grid NX x NY x NZ lives in a buffer where node (x, y, z) sits at
//   origin + z * plane + y * pitch + x
// with 32 zero floats before x = 0 (so rows start 128-byte aligned), at least
// 32 after the last computed column, 4 zero rows before/after in y (3-D) and
// 4 zero planes before/after in z.  The zeros are never written: they are the
// p = 0 boundary of Eq. 1 seen by the 8th-order stencil (radius 4).  Columns
// in [NX, NX4) (NX4 = NX rounded up to 4) carry a = 0 and stay exactly zero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rbc {

// 8th-order central second-derivative weights c1..c4 (Section 4).  The
// kernels evaluate h^2 lap p as sum_k c_k [(p_{-k} - p) + (p_{+k} - p)] per
// axis, which equals c0 p + sum_k c_k (p_{-k} + p_{+k}) because
// c0 = -2 (c1 + c2 + c3 + c4); differences from the centre keep the fp32
// rounding relative to the (small) second differences instead of |p|.
constexpr float kC1 = 1.6f;
constexpr float kC2 = -0.2f;
constexpr float kC3 = 0.025396825396825397f;   // 8/315
constexpr float kC4 = -0.0017857142857142857f; // -1/560
// |symbol of L8| at the Nyquist wavenumber: stability needs a * ndim * it < 4.
constexpr double kSymbolMax = 6.501587301587302;

// Programmatic dependent launch: the kernels of consecutive time steps are
// launched with programmatic stream serialisation, so the next step's grid
// can be scheduled while this one drains; each kernel waits for its
// predecessor's completion (and memory) before touching the fields and lets
// its dependents launch after its own stores.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

constexpr int kTileX = 128;  // x extent of a block tile: 32 lanes x float4
constexpr int kHaloX = 32;   // zero floats before x = 0
constexpr int kHaloR = 4;    // stencil radius

struct Lay {
  int ndim;
  int NX, NY, NZ;  // padded grid
  int NX4;         // NX rounded up to 4
  int pitch;       // floats per row (multiple of 32)
  int rows;        // rows per z-plane (1 in 2-D)
  int plane;       // floats per z-plane
  int origin;      // offset of node (0, 0, 0)
  long long total; // floats per buffer
};

__host__ __device__ inline int lay_off(const Lay &L, int x, int y, int z) {
  return L.origin + z * L.plane + y * L.pitch + x;
}

// Per-shot values read by the kernels from device memory, so that a captured
// CUDA graph stays valid from shot to shot.
struct ShotInfo {
  int src_off;     // source node offset in the pitched layout
  int nrec;        // receivers of this shot
  float src_fwd;   // h^(2-d): forward injection scale
  float src_rev;   // h^(2-d) or 0: reconstruction re-subtraction scale
  float rec_scale; // +h^(2-d): receiver injection scale (Eq. 2)
  int fault;       // test hook: 1 = the first 3-D forward launch withholds one plane
  int pad[2];
};

struct StepArgs {
  Lay L;
  const float *__restrict__ a;
  const float *__restrict__ cur;  // p^n
  float *__restrict__ nxt;        // in: p^{n-1}; out: p^{n+1}
  const ShotInfo *info;
  const float *wav;               // f[0..nt-1]
  const int *rec_off;             // receiver offsets (pitched layout)
  float *seis_t;                  // [nt+1][nrec] time-major record
  int n;                          // time level held in `cur`
  int sample;                     // record cur at the receivers
  int zc;                         // z planes per block (3-D)
  int *err;                       // error word (bounded waits that gave up)
};

struct RevArgs {
  Lay L;
  const float *__restrict__ a;
  const float *__restrict__ rc;   // p^R_n
  float *__restrict__ rn;         // in: p^R_{n+1}; out: p^R_{n-1}
  const float *__restrict__ bc;   // pbar_n
  float *__restrict__ bn;         // in: pbar_{n+1}; out: pbar_{n-1}
  float *__restrict__ num;        // pitched image accumulators
  float *__restrict__ den;
  const ShotInfo *info;
  const float *wav;
  const int *rec_off;
  const int *tile_ptr;            // receivers of each block tile (CSR)
  const int *tile_rec;
  const float *seis_t;            // [nt+1][nrec]
  int n;
  int do_r, do_b;                 // update p^R / pbar at this level
  int ix0, ix1, iy0, iy1, iz0, iz1; // interior box [lo, hi) in padded nodes
  int zc;
  int *err;
  int mode;                       // 0: imaging integrals; 1: FWI gradient (2-D)
  int n_src;                      // time index of the re-subtracted source
};

// ---- launch geometry shared by the host (CSR) and the kernels ----
constexpr int k2dWarps = 8;   // warps per block, stacked in z (2-D reverse and batched kernels)
constexpr int k2dWarpsF = 4;  // warps per block of the single-shot 2-D forward kernel (swept: 2, 4, 8)
constexpr int k2dWarpsR = 8;  // warps per block of the single-shot 2-D reverse kernel (swept: 6, 8, 16)
constexpr int k2dRowsF = 2;   // rows per warp, forward kernel (swept on GB300: 1, 2, 4, 8)
constexpr int k2dRowsR = 2;   // rows per warp, reverse kernel (swept: 1, 2, 3, 4)
constexpr int k3dBY = 16;     // y rows covered by the layout's row padding (3-D)
constexpr int k3dZC = 32;     // z planes per block (3-D)

// Fill L for a padded grid NX x NY x NZ (NY = 1 in 2-D).  Every extent and
// offset is formed in 64-bit first: the grid is refused (false, L untouched)
// when a buffer would not be addressable by the kernels' 32-bit offsets.
inline bool lay_make(int ndim, long long NX, long long NY, long long NZ, Lay *out) {
  if (NX < 1 || NY < 1 || NZ < 1 || NX >= (1LL << 31) || NY >= (1LL << 31) || NZ >= (1LL << 31)) return false;
  const long long pitch = (NX + kTileX - 1) / kTileX * kTileX + 2 * kHaloX;
  long long rows = 1, plane = pitch, origin = kHaloR * pitch + kHaloX;
  if (ndim == 3) {
    rows = (NY + k3dBY - 1) / k3dBY * k3dBY + 2 * kHaloR;
    plane = pitch * rows;
    origin = kHaloR * plane + kHaloR * pitch + kHaloX;
  }
  const long long total = (NZ + 2 * kHaloR) * plane;
  if (total >= (1LL << 31)) return false;
  Lay L;
  L.ndim = ndim;
  L.NX = (int)NX;
  L.NY = (int)NY;
  L.NZ = (int)NZ;
  L.NX4 = (int)((NX + 3) / 4 * 4);
  L.pitch = (int)pitch;
  L.rows = (int)rows;
  L.plane = (int)plane;
  L.origin = (int)origin;
  L.total = total;
  *out = L;
  return true;
}

} // namespace rbc

// kernel launchers (rbc_kernels.cu)
namespace rbc {
bool launch_fwd(const StepArgs &A, cudaStream_t s);
// Two forward levels per launch (2-D): (prev = p^{n-1}, A.cur = p^n) ->
// (out1 = p^{n+1}, out2 = p^{n+2}); tiles of 128 x fwd2_tile_rows() with the
// receivers of each tile in (tile_ptr, tile_rec).
bool launch_fwd2_2d(const StepArgs &A, const float *prev, float *out1, float *out2, const int *tile_ptr,
                    const int *tile_rec, cudaStream_t s);
int fwd2_tile_rows();
bool launch_rev(const RevArgs &A, cudaStream_t s);
// rbc_kernels3d.cu (TMA-fed 3-D kernels)
bool launch_fwd3d(const StepArgs &A, cudaStream_t s);
bool launch_rev3d(const RevArgs &A, cudaStream_t s);
int tile_rows_3d();
int zc_for_3d(const Lay &L, bool fwd);  // z planes per tile of the forward / reverse 3-D kernel
void *tmap_encode_fn();  // cuTensorMapEncodeTiled from the driver, or NULL
void rev_tiling(const Lay &L, int zc, int *gx, int *gy, int *gz, int *tz_or_by);
void launch_copy_in(const Lay &L, const float *dense, float *pitched, cudaStream_t s);
void launch_copy_out(const Lay &L, const float *pitched, float *dense, cudaStream_t s);
void launch_transpose(const float *in, float *out, int rows, int cols, cudaStream_t s);
void launch_accum_interior(const Lay &L, const float *pitched, float *dense, int nb, int top, int nx,
                           int ny, int nz, int overwrite, cudaStream_t s);
void launch_max(const float *x, long long n, unsigned int *out_bits, cudaStream_t s);
void launch_image_stack(const float *num, const float *den, const unsigned int *maxbits,
                        float eps_rel, int nx, int ny, int nz, int off_x, int off_y, int sx,
                        int sy, float *image, cudaStream_t s);
void launch_fwi_residual(const float *seis_t, const float *dobs, float *resid, double *misfit, int nrec,
                         int nt, cudaStream_t s);
void launch_fwi_adjoint_source(const float *resid, float *seis_t, int nrec, int nt, float scale,
                               cudaStream_t s);
void launch_fwi_finalize(const Lay &L, const float *num, const float *a, float *grad, int nb, int nx,
                         int nz, double dt, double h, cudaStream_t s);
// RTM with wavefield storage (Algorithm 2, Eq. 7 stride)
void launch_store_level(const Lay &L, const float *p, float *slot, int nb, int top, int nx, int ny, int nz,
                        cudaStream_t s);
void launch_store_image(const Lay &L, const float *slot, const float *pb, float *num, float *den, int nb, int top,
                        int nx, int ny, int nz, cudaStream_t s);
void launch_rec_inject(const float *a, float *bn, const int *rec_off, const ShotInfo *info, const float *seis_t,
                       int n, int nrec_cap, cudaStream_t s);
void launch_rbc_build(int ndim, int nx, int ny, int nz, int nb, int top, const float *v_int, double v_lo,
                      double v_hi, double v_max, uint64_t seed, int mode, double dt, double h,
                      float *v_pad, float *a, cudaStream_t s);
} // namespace rbc
