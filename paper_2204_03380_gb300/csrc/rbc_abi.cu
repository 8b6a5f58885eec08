// rbc_abi.cu -- the C ABI of librbc (declared in include/rbc.h): argument
// checks, the per-model context (internal wavefields in the pitched layout),
// per-shot tables, and the time loops of Algorithms 1 and 3 issued either as
// plain launches or as one captured CUDA graph per context and loop kind.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rbc.h"
#include "rbc_internal.cuh"

using namespace rbc;

namespace {

thread_local std::string g_err;
thread_local long long g_launches = 0;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? RBC_ENOMEM : RBC_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                     \
  } while (0)

#define CKL()                                                                         \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) return fail(RBC_ECUDA, "launch: %s", cudaGetErrorString(e_)); \
  } while (0)

int check_grid(const rbc_grid *g) {
  if (!g) return fail(RBC_EINVAL, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(RBC_EINVAL, "ndim must be 2 or 3 (got %d)", g->ndim);
  if (g->nx < 1 || g->nz < 1 || (g->ndim == 3 && g->ny < 1))
    return fail(RBC_EINVAL, "interior sizes must be >= 1");
  if (g->nb < 2) return fail(RBC_EINVAL, "nb must be >= 2 (got %d)", g->nb);
  if (g->free_surface != 0 && g->free_surface != 1) return fail(RBC_EINVAL, "free_surface must be 0 or 1");
  if (!(g->h > 0) || !(g->dt > 0)) return fail(RBC_EINVAL, "h and dt must be > 0");
  if (g->nt < 1) return fail(RBC_EINVAL, "nt must be >= 1");
  return RBC_OK;
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Rows above the interior: the random pad, or with a free surface (Section 5)
// half the stencil length (4) of zero-pressure rows.
inline int top_rows(const rbc_grid *g) { return g->free_surface ? kHaloR : g->nb; }

// The context layout of grid g; false when a buffer would not be
// addressable by 32-bit offsets (extents formed in 64-bit first).
bool make_layout(const rbc_grid *g, Lay *L) {
  const long long NX = (long long)g->nx + 2LL * g->nb;
  const long long NY = (g->ndim == 3) ? (long long)g->ny + 2LL * g->nb : 1;
  const long long NZ = (long long)g->nz + g->nb + top_rows(g);
  return lay_make(g->ndim, NX, NY, NZ, L);
}

} // namespace

namespace rbc {
// Set this thread's error message from another translation unit.
int set_error(int code, const char *msg) {
  g_err = msg;
  return code;
}
// Count kernel launches queued by another translation unit.
void add_launches(long long n) { g_launches += n; }
void static_inject_fault(int mode);  // rbc_static.cu
} // namespace rbc

struct rbc_ctx {
  rbc_grid g;
  Lay L;
  int dev = 0;
  float *buf = nullptr;  // one allocation: a, p0, p1, q0, q1, num, den
  float *a = nullptr, *p[2] = {nullptr, nullptr}, *q[2] = {nullptr, nullptr};
  float *num = nullptr, *den = nullptr;
  ShotInfo *info = nullptr;  // [0]: this shot; [1]: no source, no receivers (Algorithm 2's pbar steps)
  float *wav = nullptr;
  int rec_cap = 0;
  int *rec_off = nullptr;
  int *tile_rec = nullptr;
  int *tile_ptr = nullptr;
  int ntiles = 0;
  float *seis_t = nullptr;
  cudaStream_t cap = nullptr;
  // cached graphs: 0 = modeling loop, 1 = RTM forward phase, 2 = RTM reverse phase,
  // 3 = FWI adjoint phase, 4/5 = storage-RTM forward/reverse phase (for store, stride)
  static constexpr int kGraphs = 6;
  cudaGraphExec_t gexec[kGraphs] = {};
  long long gnodes[kGraphs] = {};
  float *store = nullptr;  // Algorithm 2: the kept levels of the graphs 4/5
  int stride = 0;
  double *misfit_tmp = nullptr;
  unsigned int *dmax = nullptr;  // rbc_set_coef's stability check
  // phase timing (rbc_phase_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // three events per timed shot
  std::vector<cudaEvent_t> ev_free;
  bool use_graph = true;
  int levels_per_launch = 1;  // 2: the 2-D forward phases advance two levels per launch (RBC_TEMPORAL=2)
  int zc = k3dZC, zc_r = k3dZC;  // z planes per tile of the 3-D forward / reverse kernels
  // snapshots
  std::vector<int> snap;
  float *pf = nullptr, *pr = nullptr, *pb = nullptr;
  // panel location after the last forward phase
  int have_panels = 0;
  // error word of the kernels' bounded waits (mapped host memory)
  int *err_host = nullptr;
  int *err_dev = nullptr;
  int fault = 0;  // rbc_inject_fault: applies to the next call only
};

namespace {

void drop_graphs(rbc_ctx *c) {
  for (int k = 0; k < rbc_ctx::kGraphs; ++k) {
    if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
    c->gexec[k] = nullptr;
  }
}

// Report (once) a bounded device wait that gave up in an earlier launch.
int check_device_error(rbc_ctx *c) {
  if (c->err_host && *(volatile int *)c->err_host) {
    *(volatile int *)c->err_host = 0;
    return fail(RBC_ETIMEOUT, "a kernel's bounded wait gave up (data in flight did not arrive); results of the "
                              "calls since the last check are invalid");
  }
  return RBC_OK;
}

int ensure_receivers(rbc_ctx *c, int nrec) {
  if (nrec <= c->rec_cap && c->rec_off) return RBC_OK;
  int cap = std::max(nrec, std::max(64, c->rec_cap * 2));
  drop_graphs(c);
  cudaFree(c->rec_off);
  cudaFree(c->tile_rec);
  cudaFree(c->seis_t);
  c->rec_off = nullptr;
  c->tile_rec = nullptr;
  c->seis_t = nullptr;
  c->rec_cap = 0;
  CK(cudaMalloc(&c->rec_off, sizeof(int) * cap));
  CK(cudaMalloc(&c->tile_rec, sizeof(int) * cap));
  CK(cudaMalloc(&c->seis_t, sizeof(float) * (size_t)cap * (c->g.nt + 2)));  // + 1 row for the FWI adjoint
  c->rec_cap = cap;
  return RBC_OK;
}

int node_ok(const rbc_ctx *c, const int *r) {
  const Lay &L = c->L;
  const int y = r[1];
  if (r[0] < 0 || r[0] >= L.NX || r[2] < 0 || r[2] >= L.NZ) return 0;
  if (L.ndim == 2) return y == 0;
  return y >= 0 && y < L.NY;
}

// Upload the per-shot tables: source offset and scales, receiver offsets and
// the receiver list of every reverse-kernel tile (counting sort by tile).
int upload_shot(rbc_ctx *c, const int *src, int nrec, const int *rec, int reinject,
                cudaStream_t s) {
  if (!src) return fail(RBC_EINVAL, "src is NULL");
  if (!node_ok(c, src)) return fail(RBC_EINVAL, "source node (%d,%d,%d) outside the padded grid", src[0], src[1], src[2]);
  if (nrec < 0 || (nrec > 0 && !rec)) return fail(RBC_EINVAL, "bad receiver list");
  for (int r = 0; r < nrec; ++r)
    if (!node_ok(c, rec + 3 * r))
      return fail(RBC_EINVAL, "receiver %d node (%d,%d,%d) outside the padded grid", r, rec[3 * r],
                  rec[3 * r + 1], rec[3 * r + 2]);
  int rc = ensure_receivers(c, std::max(nrec, 1));
  if (rc) return rc;
  const Lay &L = c->L;
  const double ps = (L.ndim == 3) ? 1.0 / c->g.h : 1.0;  // h^(2-d)
  ShotInfo info{};
  info.src_off = lay_off(L, src[0], src[1], src[2]);
  info.nrec = nrec;
  info.src_fwd = (float)ps;
  info.src_rev = reinject ? (float)ps : 0.f;
  info.rec_scale = (float)ps;
  info.fault = c->fault;
  c->fault = 0;
  int gx, gy, gz, t;
  rev_tiling(L, c->zc_r, &gx, &gy, &gz, &t);
  std::vector<int> off(std::max(nrec, 1)), tile(std::max(nrec, 1)), ptr(c->ntiles + 1, 0),
      order(std::max(nrec, 1));
  for (int r = 0; r < nrec; ++r) {
    const int x = rec[3 * r], y = rec[3 * r + 1], z = rec[3 * r + 2];
    off[r] = lay_off(L, x, y, z);
    int b;
    if (L.ndim == 2) b = (z / t) * gx + x / kTileX;
    else b = (((z / c->zc_r) * gy + y / t) * gx + x / kTileX) * t + y % t;  // (tile, row) cells
    tile[r] = b;
    ptr[b + 1]++;
  }
  for (int b = 0; b < c->ntiles; ++b) ptr[b + 1] += ptr[b];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int r = 0; r < nrec; ++r) order[fill[tile[r]]++] = r;
  CK(cudaMemcpyAsync(c->info, &info, sizeof info, cudaMemcpyHostToDevice, s));
  if (nrec > 0) {
    CK(cudaMemcpyAsync(c->rec_off, off.data(), sizeof(int) * nrec, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->tile_rec, order.data(), sizeof(int) * nrec, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(c->tile_ptr, ptr.data(), sizeof(int) * (c->ntiles + 1), cudaMemcpyHostToDevice, s));
  return RBC_OK;
}

int snap_index(const rbc_ctx *c, int n) {
  for (size_t k = 0; k < c->snap.size(); ++k)
    if (c->snap[k] == n) return (int)k;
  return -1;
}

long long field_elems(const rbc_ctx *c) { return (long long)c->L.NX * c->L.NY * c->L.NZ; }

// Algorithm 1 time loop: p^n lives in p[n & 1]; step n overwrites p^{n-1}
// with p^{n+1}.
// Two levels per launch (2-D, no snapshots): level m lives in buffer m mod 4
// of (p0, p1, q0, q1) -- the q fields are free until the reverse phase, which
// clears them -- so a launch never writes a buffer that a neighbouring block
// still reads; an odd nt ends with one single-level step, and the last two
// levels are left in p[(nt - 1) & 1] and p[nt & 1] as the single-level loop
// leaves them.
int enqueue_forward2(rbc_ctx *c, cudaStream_t s, int sample) {
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  float *B[4] = {c->p[0], c->p[1], c->q[0], c->q[1]};
  CK(cudaMemsetAsync(B[0], 0, bytes, s));  // level 0
  CK(cudaMemsetAsync(B[3], 0, bytes, s));  // level -1
  StepArgs A{};
  A.L = L;
  A.a = c->a;
  A.info = c->info;
  A.wav = c->wav;
  A.rec_off = c->rec_off;
  A.seis_t = c->seis_t;
  A.sample = sample;
  A.zc = c->zc;
  A.err = c->err_dev;
  const int nt = c->g.nt;
  float *loc_prev = B[3], *loc_cur = B[0];  // buffers of levels n - 1 and n
  int n = 0;
  for (; n + 2 <= nt; n += 2) {
    A.cur = loc_cur;
    A.n = n;
    if (!launch_fwd2_2d(A, loc_prev, B[(n + 1) & 3], B[(n + 2) & 3], c->tile_ptr, c->tile_rec, s))
      return fail(RBC_ECUDA, "launch failed");
    ++g_launches;
    loc_prev = B[(n + 1) & 3];
    loc_cur = B[(n + 2) & 3];
  }
  if (n < nt) {  // one single-level step: p^{n+1} overwrites p^{n-1} in place
    A.cur = loc_cur;
    A.nxt = loc_prev;
    A.n = n;
    if (!launch_fwd(A, s)) return fail(RBC_ECUDA, "launch failed");
    ++g_launches;
    float *t = loc_prev;
    loc_prev = loc_cur;
    loc_cur = t;
  }
  // the panels where the reverse phase, rbc_get_panels and the last sample
  // expect them; a copy never overwrites a panel that is still to be copied
  float *want_prev = c->p[(nt - 1) & 1], *want_cur = c->p[nt & 1];
  auto copy = [&](float *dst, const float *src) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
  };
  if (loc_cur == want_prev && loc_prev == want_cur) {  // swapped: through a q buffer
    CK(copy(c->q[0], loc_cur));
    CK(copy(want_prev, loc_prev));
    CK(copy(want_cur, c->q[0]));
  } else if (loc_prev == want_cur) {
    CK(copy(want_prev, loc_prev));
    if (loc_cur != want_cur) CK(copy(want_cur, loc_cur));
  } else {
    if (loc_cur != want_cur) CK(copy(want_cur, loc_cur));
    if (loc_prev != want_prev) CK(copy(want_prev, loc_prev));
  }
  CKL();
  return RBC_OK;
}

int enqueue_forward(rbc_ctx *c, cudaStream_t s, int sample) {
  if (c->levels_per_launch == 2 && c->snap.empty() && c->g.nt >= 2) return enqueue_forward2(c, s, sample);
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  CK(cudaMemsetAsync(c->p[0], 0, bytes, s));
  CK(cudaMemsetAsync(c->p[1], 0, bytes, s));
  StepArgs A{};
  A.L = L;
  A.a = c->a;
  A.info = c->info;
  A.wav = c->wav;
  A.rec_off = c->rec_off;
  A.seis_t = c->seis_t;
  A.sample = sample;
  A.zc = c->zc;
  A.err = c->err_dev;
  const int nt = c->g.nt;
  for (int n = 0; n < nt; ++n) {
    const int k = snap_index(c, n);
    if (k >= 0 && c->pf) {
      launch_copy_out(L, c->p[n & 1], c->pf + k * field_elems(c), s);
      ++g_launches;
    }
    A.cur = c->p[n & 1];
    A.nxt = c->p[(n + 1) & 1];
    A.n = n;
    if (!launch_fwd(A, s)) return fail(RBC_ECUDA, "tensor map encoding failed");
    ++g_launches;
  }
  const int k = snap_index(c, nt);
  if (k >= 0 && c->pf) {
    launch_copy_out(L, c->p[nt & 1], c->pf + k * field_elems(c), s);
    ++g_launches;
  }
  CKL();
  return RBC_OK;
}

__global__ void k_sample_info(const float *__restrict__ p, const int *__restrict__ rec_off,
                              const ShotInfo *info, float *__restrict__ seis_t, int n) {
  const int nrec = info->nrec;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
    seis_t[(long long)n * nrec + r] = p[rec_off[r]];
}

// Algorithm 3 reverse loop, n = nt .. 0: p^R_n in p[n & 1], pbar_n in q[n & 1].
int enqueue_reverse(rbc_ctx *c, cudaStream_t s) {
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  CK(cudaMemsetAsync(c->q[0], 0, bytes, s));
  CK(cudaMemsetAsync(c->q[1], 0, bytes, s));
  CK(cudaMemsetAsync(c->num, 0, bytes, s));
  CK(cudaMemsetAsync(c->den, 0, bytes, s));
  RevArgs A{};
  A.L = L;
  A.a = c->a;
  A.num = c->num;
  A.den = c->den;
  A.info = c->info;
  A.wav = c->wav;
  A.rec_off = c->rec_off;
  A.tile_ptr = c->tile_ptr;
  A.tile_rec = c->tile_rec;
  A.seis_t = c->seis_t;
  const int nb = c->g.nb, top = top_rows(&c->g);
  A.ix0 = nb;
  A.ix1 = nb + c->g.nx;
  A.iz0 = top;
  A.iz1 = top + c->g.nz;
  A.iy0 = (L.ndim == 3) ? nb : 0;
  A.iy1 = (L.ndim == 3) ? nb + c->g.ny : 1;
  A.zc = c->zc_r;
  A.err = c->err_dev;
  const int nt = c->g.nt;
  for (int n = nt; n >= 0; --n) {
    const int k = snap_index(c, n);
    if (k >= 0 && c->pr) { launch_copy_out(L, c->p[n & 1], c->pr + k * field_elems(c), s); ++g_launches; }
    if (k >= 0 && c->pb) { launch_copy_out(L, c->q[n & 1], c->pb + k * field_elems(c), s); ++g_launches; }
    A.rc = c->p[n & 1];
    A.rn = c->p[(n + 1) & 1];
    A.bc = c->q[n & 1];
    A.bn = c->q[(n + 1) & 1];
    A.n = n;
    A.do_r = (n < nt && n > 0) ? 1 : 0;  // p^R_{nt-1} is the stored panel
    A.do_b = (n > 0) ? 1 : 0;
    A.n_src = n;
    A.mode = 0;
    if (!launch_rev(A, s)) return fail(RBC_ECUDA, "tensor map encoding failed");
    ++g_launches;
  }
  CKL();
  return RBC_OK;
}

typedef int (*enqueue_fn)(rbc_ctx *, cudaStream_t, int);

int enq_model(rbc_ctx *c, cudaStream_t s, int) {
  int rc = enqueue_forward(c, s, 1);
  if (rc) return rc;
  k_sample_info<<<cdiv(std::max(c->rec_cap, 1), 256), 256, 0, s>>>(c->p[c->g.nt & 1], c->rec_off, c->info,
                                                                    c->seis_t, c->g.nt);
  ++g_launches;
  CKL();
  return RBC_OK;
}

int enq_rtm_fwd(rbc_ctx *c, cudaStream_t s, int) { return enqueue_forward(c, s, 0); }

int enq_rtm_rev(rbc_ctx *c, cudaStream_t s, int) { return enqueue_reverse(c, s); }

// FWI adjoint phase (2-D): at kernel level m = nt+1 .. 1 the adjoint field
// mu = a lambda goes from (mu^m, mu^{m+1}) to mu^{m-1} with the adjoint record
// row m injected, while the reconstruction runs one level behind: (p^{m-1},
// p^m) -> p^{m-2}, so that num += mu^m (p^m - 2 p^{m-1} + p^{m-2}).
int enq_fwi_adj(rbc_ctx *c, cudaStream_t s, int) {
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  CK(cudaMemsetAsync(c->q[0], 0, bytes, s));
  CK(cudaMemsetAsync(c->q[1], 0, bytes, s));
  CK(cudaMemsetAsync(c->num, 0, bytes, s));
  RevArgs A{};
  A.L = L;
  A.a = c->a;
  A.num = c->num;
  A.den = c->den;
  A.info = c->info;
  A.wav = c->wav;
  A.rec_off = c->rec_off;
  A.tile_ptr = c->tile_ptr;
  A.tile_rec = c->tile_rec;
  A.seis_t = c->seis_t;
  const int nb = c->g.nb;
  A.ix0 = nb;
  A.ix1 = nb + c->g.nx;
  A.iz0 = nb;
  A.iz1 = nb + c->g.nz;
  A.iy0 = 0;
  A.iy1 = 1;
  A.zc = c->zc_r;
  A.err = c->err_dev;
  A.mode = 1;
  const int nt = c->g.nt;
  for (int m = nt + 1; m >= 1; --m) {
    A.rc = c->p[(m - 1) & 1];
    A.rn = c->p[m & 1];
    A.bc = c->q[m & 1];
    A.bn = c->q[(m + 1) & 1];
    A.n = m;           // adjoint record row injected
    A.n_src = m - 1;   // source term of the reconstructed step
    A.do_r = (m <= nt) ? 1 : 0;  // p^{nt-1} is a stored panel
    A.do_b = 1;
    if (!launch_rev(A, s)) return fail(RBC_ECUDA, "launch failed");
    ++g_launches;
  }
  CKL();
  return RBC_OK;
}

// Algorithm 2, first loop: Algorithm 1 without recording; the interior of
// every k-th level p^n (n = 0, k, ..., <= nt) goes to slot n / k of the store.
int enq_store_fwd(rbc_ctx *c, cudaStream_t s, int) {
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  CK(cudaMemsetAsync(c->p[0], 0, bytes, s));
  CK(cudaMemsetAsync(c->p[1], 0, bytes, s));
  const rbc_grid &g = c->g;
  const long long nint = (long long)g.nx * g.ny * g.nz;
  StepArgs A{};
  A.L = L;
  A.a = c->a;
  A.info = c->info;
  A.wav = c->wav;
  A.rec_off = c->rec_off;
  A.seis_t = c->seis_t;
  A.sample = 0;
  A.zc = c->zc;
  A.err = c->err_dev;
  for (int n = 0; n <= g.nt; ++n) {
    if (n % c->stride == 0) {
      launch_store_level(L, c->p[n & 1], c->store + (n / c->stride) * nint, g.nb, top_rows(&g), g.nx, g.ny, g.nz,
                         s);
      ++g_launches;
    }
    if (n == g.nt) break;
    A.cur = c->p[n & 1];
    A.nxt = c->p[(n + 1) & 1];
    A.n = n;
    if (!launch_fwd(A, s)) return fail(RBC_ECUDA, "tensor map encoding failed");
    ++g_launches;
  }
  CKL();
  return RBC_OK;
}

// Algorithm 2, second loop, n = nt .. 0: Eq. 3 integrals at the kept levels
// (p^n read from the store), then pbar_{n-1} by the leapfrog step (the step
// is symmetric in time, so the forward kernel runs it with the silent shot
// record info[1]) and the record row n injected at the receivers.
int enq_store_rev(rbc_ctx *c, cudaStream_t s, int) {
  const Lay &L = c->L;
  const size_t bytes = sizeof(float) * (size_t)L.total;
  CK(cudaMemsetAsync(c->q[0], 0, bytes, s));
  CK(cudaMemsetAsync(c->q[1], 0, bytes, s));
  CK(cudaMemsetAsync(c->num, 0, bytes, s));
  CK(cudaMemsetAsync(c->den, 0, bytes, s));
  const rbc_grid &g = c->g;
  const long long nint = (long long)g.nx * g.ny * g.nz;
  StepArgs B{};
  B.L = L;
  B.a = c->a;
  B.info = c->info + 1;
  B.wav = c->wav;
  B.rec_off = c->rec_off;
  B.seis_t = c->seis_t;
  B.sample = 0;
  B.n = 0;  // the silent info scales f[0] by 0
  B.zc = c->zc;
  B.err = c->err_dev;
  for (int n = g.nt; n >= 0; --n) {
    if (n % c->stride == 0) {
      launch_store_image(L, c->store + (n / c->stride) * nint, c->q[n & 1], c->num, c->den, g.nb, top_rows(&g),
                         g.nx, g.ny,
                         g.nz, s);
      ++g_launches;
    }
    if (n == 0) break;
    B.cur = c->q[n & 1];
    B.nxt = c->q[(n + 1) & 1];
    if (!launch_fwd(B, s)) return fail(RBC_ECUDA, "tensor map encoding failed");
    launch_rec_inject(c->a, c->q[(n + 1) & 1], c->rec_off, c->info, c->seis_t, n, c->rec_cap, s);
    g_launches += 2;
  }
  CKL();
  return RBC_OK;
}

int record_event(rbc_ctx *c, cudaStream_t s) {
  cudaEvent_t e;
  if (!c->ev_free.empty()) {
    e = c->ev_free.back();
    c->ev_free.pop_back();
  } else {
    CK(cudaEventCreate(&e));
  }
  c->ev.push_back(e);
  CK(cudaEventRecord(e, s));
  return RBC_OK;
}

// Run a loop either directly on `s` or as this context's cached graph.
int run_loop(rbc_ctx *c, int kind, enqueue_fn fn, cudaStream_t s) {
  if (!c->use_graph || !c->snap.empty()) return fn(c, s, 0);
  if (!c->gexec[kind]) {
    long long before = g_launches;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int rc = fn(c, c->cap, 0);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
    c->gnodes[kind] = g_launches - before;
    g_launches = before;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(RBC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec[kind], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->gexec[kind] = nullptr;
      return fail(RBC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  CK(cudaGraphLaunch(c->gexec[kind], s));
  g_launches += c->gnodes[kind];
  return RBC_OK;
}

} // namespace

// ===================================================================== ABI ==
extern "C" {

const char *rbc_last_error(void) { return g_err.c_str(); }

long long rbc_launch_count(int reset) {
  long long v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

int rbc_build_velocity(const rbc_grid *g, const float *v_int_dev, float v_lo, float v_hi, float v_max,
                       uint64_t seed, int mode, float *v_pad_dev, float *a_dev, void *stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!v_int_dev || !a_dev) return fail(RBC_EINVAL, "v_int_dev and a_dev must not be NULL");
  if (!(v_lo <= v_hi) || !(v_lo > 0) || !(v_max > 0)) return fail(RBC_EINVAL, "need 0 < v_lo <= v_hi, v_max > 0");
  if (mode != 0 && mode != 1) return fail(RBC_EINVAL, "mode must be 0 (blend) or 1 (literal)");
  launch_rbc_build(g->ndim, g->nx, g->ny, g->nz, g->nb, top_rows(g), v_int_dev, v_lo, v_hi, v_max, seed, mode,
                   g->dt, g->h,
                   v_pad_dev, a_dev, (cudaStream_t)stream);
  ++g_launches;
  CKL();
  return RBC_OK;
}

int rbc_create(const rbc_grid *g, const float *a_dev, rbc_ctx **out) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!a_dev || !out) return fail(RBC_EINVAL, "a_dev and out must not be NULL");
  *out = nullptr;
  Lay L;
  if (!make_layout(g, &L)) return fail(RBC_EINVAL, "grid too large for 32-bit offsets");
  // stability: max(a) * ndim * |symbol|max < 4
  const long long n = (long long)L.NX * L.NY * L.NZ;
  unsigned int *dmax = nullptr;
  CK(cudaMalloc(&dmax, sizeof(unsigned int)));
  cudaMemset(dmax, 0, sizeof(unsigned int));
  launch_max(a_dev, n, dmax, 0);
  unsigned int bits = 0;
  cudaError_t e = cudaMemcpy(&bits, dmax, sizeof bits, cudaMemcpyDeviceToHost);
  cudaFree(dmax);
  if (e != cudaSuccess) return fail(RBC_ECUDA, "stability check: %s", cudaGetErrorString(e));
  float amax;
  std::memcpy(&amax, &bits, sizeof amax);
  if (!(amax * g->ndim * kSymbolMax < 4.0))
    return fail(RBC_ECFL, "unstable: max (v dt/h)^2 = %g exceeds %g for %d-D", amax, 4.0 / (g->ndim * kSymbolMax),
                g->ndim);
  rbc_ctx *c = new rbc_ctx();
  c->g = *g;
  if (g->ndim == 2) c->g.ny = 1;
  c->L = L;
  cudaGetDevice(&c->dev);
  const char *env = getenv("RBC_GRAPH");
  c->use_graph = !(env && env[0] == '0');
  // temporal blocking of the 2-D forward phases; it uses the receiver lists of
  // the 2-D reverse tiling, so it needs that tiling's 8-row tiles
  const char *tenv = getenv("RBC_TEMPORAL");
  if (tenv && atoi(tenv) == 2 && L.ndim == 2) {
    int gx, gy, gz, t;
    rev_tiling(L, c->zc_r, &gx, &gy, &gz, &t);
    if (t == fwd2_tile_rows()) c->levels_per_launch = 2;
  }
  const char *zenv = getenv("RBC_ZC");  // tuning knob: z planes per 3-D block
  if (L.ndim == 3) {
    c->zc = zc_for_3d(L, true);
    c->zc_r = zc_for_3d(L, false);
  }
  if (zenv && atoi(zenv) >= 8) c->zc = c->zc_r = atoi(zenv);
  const size_t fb = sizeof(float) * (size_t)L.total;
  cudaError_t ea = cudaMalloc(&c->buf, 7 * fb);
  if (ea != cudaSuccess) {
    delete c;
    return fail(RBC_ENOMEM, "cudaMalloc of %zu bytes: %s", 7 * fb, cudaGetErrorString(ea));
  }
  c->a = c->buf;
  c->p[0] = c->buf + L.total;
  c->p[1] = c->buf + 2 * L.total;
  c->q[0] = c->buf + 3 * L.total;
  c->q[1] = c->buf + 4 * L.total;
  c->num = c->buf + 5 * L.total;
  c->den = c->buf + 6 * L.total;
  int gx, gy, gz, t;
  rev_tiling(L, c->zc_r, &gx, &gy, &gz, &t);
  c->ntiles = gx * gy * gz * (L.ndim == 3 ? t : 1);  // 3-D: one receiver list per (tile, row)
  if (cudaHostAlloc((void **)&c->err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void **)&c->err_dev, c->err_host, 0) != cudaSuccess) {
    rbc_destroy(c);
    return fail(RBC_ENOMEM, "error word allocation failed");
  }
  *c->err_host = 0;
  if (cudaMalloc(&c->tile_ptr, sizeof(int) * (c->ntiles + 1)) != cudaSuccess ||
      cudaMalloc(&c->info, 2 * sizeof(ShotInfo)) != cudaSuccess ||
      cudaMalloc(&c->wav, sizeof(float) * g->nt) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    rbc_destroy(c);
    return fail(RBC_ENOMEM, "context allocation failed");
  }
  ShotInfo silent{};
  silent.src_off = -1;  // no node: the kernels' point test never matches
  if (cudaMemset(c->buf, 0, 7 * fb) != cudaSuccess ||
      cudaMemcpy(c->info + 1, &silent, sizeof silent, cudaMemcpyHostToDevice) != cudaSuccess) {
    rbc_destroy(c);
    return fail(RBC_ECUDA, "memset failed");
  }
  launch_copy_in(L, a_dev, c->a, 0);
  ++g_launches;
  rc = ensure_receivers(c, 64);
  if (rc) {
    rbc_destroy(c);
    return rc;
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rbc_destroy(c);
    return fail(RBC_ECUDA, "create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return RBC_OK;
}

int rbc_set_coef(rbc_ctx *c, const float *a_dev, int check, void *stream) {
  if (!c || !a_dev) return fail(RBC_EINVAL, "ctx and a_dev must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const Lay &L = c->L;
  if (check) {
    const long long n = (long long)L.NX * L.NY * L.NZ;
    if (!c->dmax) CK(cudaMalloc(&c->dmax, sizeof(unsigned int)));
    CK(cudaMemsetAsync(c->dmax, 0, sizeof(unsigned int), s));
    launch_max(a_dev, n, c->dmax, s);
    ++g_launches;
    unsigned int bits = 0;
    CK(cudaMemcpyAsync(&bits, c->dmax, sizeof bits, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float amax;
    std::memcpy(&amax, &bits, sizeof amax);
    if (!(amax * c->g.ndim * kSymbolMax < 4.0))
      return fail(RBC_ECFL, "unstable: max (v dt/h)^2 = %g exceeds %g for %d-D", amax,
                  4.0 / (c->g.ndim * kSymbolMax), c->g.ndim);
  }
  launch_copy_in(L, a_dev, c->a, s);
  ++g_launches;
  CKL();
  return RBC_OK;
}

int rbc_destroy(rbc_ctx *c) {
  if (!c) return RBC_OK;
  cudaDeviceSynchronize();
  const int pending = check_device_error(c);
  drop_graphs(c);
  cudaFree(c->buf);
  cudaFree(c->info);
  cudaFree(c->wav);
  cudaFree(c->rec_off);
  cudaFree(c->tile_rec);
  cudaFree(c->tile_ptr);
  cudaFree(c->seis_t);
  cudaFree(c->dmax);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->err_host) cudaFreeHost(c->err_host);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  delete c;
  return pending;
}

int rbc_model(rbc_ctx *c, const int *src_host, const float *wavelet_dev, int nrec, const int *rec_host,
              float *seis_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (!wavelet_dev || (nrec > 0 && !seis_dev)) return fail(RBC_EINVAL, "wavelet_dev / seis_dev is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_device_error(c);
  if (rc) return rc;
  rc = upload_shot(c, src_host, nrec, rec_host, 1, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->wav, wavelet_dev, sizeof(float) * c->g.nt, cudaMemcpyDeviceToDevice, s));
  rc = run_loop(c, 0, enq_model, s);
  if (rc) return rc;
  if (nrec > 0) {
    launch_transpose(c->seis_t, seis_dev, c->g.nt + 1, nrec, s);
    ++g_launches;
  }
  CKL();
  c->have_panels = 1;
  return RBC_OK;
}

int rbc_rtm_shot(rbc_ctx *c, const int *src_host, const float *wavelet_dev, int nrec, const int *rec_host,
                 const float *seis_dev, int flags, float *num_dev, float *den_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (!wavelet_dev || !num_dev || !den_dev || (nrec > 0 && !seis_dev))
    return fail(RBC_EINVAL, "NULL device pointer");
  if (flags & ~(RBC_REINJECT_SOURCE | RBC_ZERO_FIRST)) return fail(RBC_EINVAL, "unknown flags 0x%x", flags);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_device_error(c);
  if (rc) return rc;
  rc = upload_shot(c, src_host, nrec, rec_host, flags & RBC_REINJECT_SOURCE, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->wav, wavelet_dev, sizeof(float) * c->g.nt, cudaMemcpyDeviceToDevice, s));
  if (nrec > 0) {
    launch_transpose(seis_dev, c->seis_t, nrec, c->g.nt + 1, s);
    ++g_launches;
  }
  if (c->timing && (rc = record_event(c, s))) return rc;
  rc = run_loop(c, 1, enq_rtm_fwd, s);
  if (rc) return rc;
  if (c->timing && (rc = record_event(c, s))) return rc;
  rc = run_loop(c, 2, enq_rtm_rev, s);
  if (rc) return rc;
  if (c->timing && (rc = record_event(c, s))) return rc;
  const int ow = (flags & RBC_ZERO_FIRST) ? 1 : 0;
  launch_accum_interior(c->L, c->num, num_dev, c->g.nb, top_rows(&c->g), c->g.nx, c->g.ny, c->g.nz, ow, s);
  launch_accum_interior(c->L, c->den, den_dev, c->g.nb, top_rows(&c->g), c->g.nx, c->g.ny, c->g.nz, ow, s);
  g_launches += 2;
  CKL();
  c->have_panels = 0;  // the reverse pass consumed the panels
  return RBC_OK;
}

int rbc_nyquist_stride(double dt, double f_max, double f_min) {
  if (!(dt > 0) || !(f_min >= 0) || !(f_max > f_min)) {
    fail(RBC_EINVAL, "need dt > 0 and 0 <= f_min < f_max");
    return 0;
  }
  const double dt_nyq = 1.0 / (2.0 * (f_max - f_min));  // Eq. 7
  const double k = std::floor(dt_nyq / dt + 1e-9);
  return k < 1.0 ? 1 : (int)std::min(k, 1e9);
}

long long rbc_storage_bytes(const rbc_grid *g, int stride) {
  if (check_grid(g)) return -1;
  if (stride < 1) {
    fail(RBC_EINVAL, "stride must be >= 1");
    return -1;
  }
  const long long nint = (long long)g->nx * (g->ndim == 3 ? g->ny : 1) * g->nz;
  return (long long)sizeof(float) * nint * (g->nt / stride + 1);
}

int rbc_rtm_storage(rbc_ctx *c, const int *src_host, const float *wavelet_dev, int nrec, const int *rec_host,
                    const float *seis_dev, int stride, float *store_dev, long long store_bytes, int flags,
                    float *num_dev, float *den_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (!wavelet_dev || !num_dev || !den_dev || !store_dev || (nrec > 0 && !seis_dev))
    return fail(RBC_EINVAL, "NULL device pointer");
  if (flags & ~RBC_ZERO_FIRST) return fail(RBC_EINVAL, "unknown flags 0x%x", flags);
  if (stride < 1) return fail(RBC_EINVAL, "stride must be >= 1 (got %d)", stride);
  const long long need = rbc_storage_bytes(&c->g, stride);
  if (store_bytes < need)
    return fail(RBC_EINVAL, "store of %lld bytes is smaller than the %lld the stride needs", store_bytes, need);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_device_error(c);
  if (rc) return rc;
  rc = upload_shot(c, src_host, nrec, rec_host, 0, s);
  if (rc) return rc;
  if (c->store != store_dev || c->stride != stride) {  // the storage graphs bake both in
    for (int k = 4; k < 6; ++k) {
      if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
      c->gexec[k] = nullptr;
    }
    c->store = store_dev;
    c->stride = stride;
  }
  CK(cudaMemcpyAsync(c->wav, wavelet_dev, sizeof(float) * c->g.nt, cudaMemcpyDeviceToDevice, s));
  if (nrec > 0) {
    launch_transpose(seis_dev, c->seis_t, nrec, c->g.nt + 1, s);
    ++g_launches;
  }
  if (c->timing && (rc = record_event(c, s))) return rc;
  rc = run_loop(c, 4, enq_store_fwd, s);
  if (rc) return rc;
  if (c->timing && (rc = record_event(c, s))) return rc;
  rc = run_loop(c, 5, enq_store_rev, s);
  if (rc) return rc;
  if (c->timing && (rc = record_event(c, s))) return rc;
  const int ow = (flags & RBC_ZERO_FIRST) ? 1 : 0;
  launch_accum_interior(c->L, c->num, num_dev, c->g.nb, top_rows(&c->g), c->g.nx, c->g.ny, c->g.nz, ow, s);
  launch_accum_interior(c->L, c->den, den_dev, c->g.nb, top_rows(&c->g), c->g.nx, c->g.ny, c->g.nz, ow, s);
  g_launches += 2;
  CKL();
  c->have_panels = 1;  // the forward loop leaves p^{nt-1}, p^{nt} in place
  return RBC_OK;
}

int rbc_image_stack(const rbc_grid *shot, const float *num_dev, const float *den_dev, float eps_rel, int off_x,
                    int off_y, const rbc_grid *survey, float *image_dev, void *stream) {
  if (!shot || !survey) return fail(RBC_EINVAL, "grid is NULL");
  if (!num_dev || !den_dev || !image_dev) return fail(RBC_EINVAL, "NULL device pointer");
  if (shot->ndim != survey->ndim || (shot->ndim != 2 && shot->ndim != 3))
    return fail(RBC_EINVAL, "shot and survey must have the same ndim (2 or 3)");
  const int ny = shot->ndim == 3 ? shot->ny : 1, sy = survey->ndim == 3 ? survey->ny : 1;
  if (shot->nx < 1 || ny < 1 || shot->nz < 1) return fail(RBC_EINVAL, "bad shot interior");
  if (shot->nz != survey->nz) return fail(RBC_EINVAL, "shot nz %d != survey nz %d", shot->nz, survey->nz);
  if (shot->ndim == 2 && off_y != 0) return fail(RBC_EINVAL, "off_y must be 0 in 2-D");
  if (off_x < 0 || off_y < 0 || off_x + shot->nx > survey->nx || off_y + ny > sy)
    return fail(RBC_EINVAL, "shot window does not fit the survey");
  if (!(eps_rel >= 0)) return fail(RBC_EINVAL, "eps_rel must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int *dmax = nullptr;
  CK(cudaMallocAsync((void **)&dmax, sizeof(unsigned int), s));
  CK(cudaMemsetAsync(dmax, 0, sizeof(unsigned int), s));
  const long long n = (long long)shot->nx * ny * shot->nz;
  launch_max(den_dev, n, dmax, s);
  launch_image_stack(num_dev, den_dev, dmax, eps_rel, shot->nx, ny, shot->nz, off_x, off_y, survey->nx, sy,
                     image_dev, s);
  g_launches += 2;
  CKL();
  CK(cudaFreeAsync(dmax, s));
  return RBC_OK;
}

int rbc_fwi_forward(rbc_ctx *c, const int *src_host, const float *wavelet_dev, int nrec, const int *rec_host,
                    const float *dobs_dev, float *resid_dev, double *misfit_dev, float *panels_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (c->L.ndim != 2 || c->g.free_surface)
    return fail(RBC_ENOTSUP, "the FWI gradient is built for 2-D grids with the random boundary on every side");
  if (!wavelet_dev || nrec < 1 || !dobs_dev || !resid_dev || !misfit_dev)
    return fail(RBC_EINVAL, "NULL pointer or no receivers");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_device_error(c);
  if (rc) return rc;
  rc = upload_shot(c, src_host, nrec, rec_host, 1, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->wav, wavelet_dev, sizeof(float) * c->g.nt, cudaMemcpyDeviceToDevice, s));
  rc = run_loop(c, 0, enq_model, s);
  if (rc) return rc;
  launch_fwi_residual(c->seis_t, dobs_dev, resid_dev, misfit_dev, nrec, c->g.nt, s);
  ++g_launches;
  const int nt = c->g.nt;
  const long long n = field_elems(c);
  if (panels_dev) {
    launch_copy_out(c->L, c->p[(nt - 1) & 1], panels_dev, s);
    launch_copy_out(c->L, c->p[nt & 1], panels_dev + n, s);
    g_launches += 2;
  }
  CKL();
  c->have_panels = 1;
  return RBC_OK;
}

int rbc_fwi_backward(rbc_ctx *c, const int *src_host, const float *wavelet_dev, int nrec, const int *rec_host,
                     const float *resid_dev, const float *panels_dev, float *grad_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (c->L.ndim != 2 || c->g.free_surface)
    return fail(RBC_ENOTSUP, "the FWI gradient is built for 2-D grids with the random boundary on every side");
  if (!wavelet_dev || nrec < 1 || !resid_dev || !grad_dev) return fail(RBC_EINVAL, "NULL pointer or no receivers");
  if (!panels_dev && !c->have_panels) return fail(RBC_EINVAL, "no panels: pass panels_dev or run rbc_fwi_forward");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_device_error(c);
  if (rc) return rc;
  rc = upload_shot(c, src_host, nrec, rec_host, 1, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->wav, wavelet_dev, sizeof(float) * c->g.nt, cudaMemcpyDeviceToDevice, s));
  const int nt = c->g.nt;
  if (panels_dev) {
    launch_copy_in(c->L, panels_dev, c->p[(nt - 1) & 1], s);
    launch_copy_in(c->L, panels_dev + field_elems(c), c->p[nt & 1], s);
    g_launches += 2;
  }
  // adjoint record: row m = -resid[.][m-1] / h^(2-d), injected as + h^(2-d) a row
  launch_fwi_adjoint_source(resid_dev, c->seis_t, nrec, nt, -1.0f, s);
  ++g_launches;
  rc = run_loop(c, 3, enq_fwi_adj, s);
  if (rc) return rc;
  launch_fwi_finalize(c->L, c->num, c->a, grad_dev, c->g.nb, c->g.nx, c->g.nz, c->g.dt, c->g.h, s);
  ++g_launches;
  CKL();
  c->have_panels = 0;
  return RBC_OK;
}

int rbc_set_snapshots(rbc_ctx *c, int nsnap, const int *levels_host, float *pf_dev, float *pr_dev, float *pb_dev) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (nsnap < 0 || (nsnap > 0 && !levels_host)) return fail(RBC_EINVAL, "bad snapshot list");
  for (int k = 0; k < nsnap; ++k)
    if (levels_host[k] < 0 || levels_host[k] > c->g.nt)
      return fail(RBC_EINVAL, "snapshot level %d outside [0, %d]", levels_host[k], c->g.nt);
  c->snap.assign(levels_host, levels_host + nsnap);
  c->pf = nsnap ? pf_dev : nullptr;
  c->pr = nsnap ? pr_dev : nullptr;
  c->pb = nsnap ? pb_dev : nullptr;
  return RBC_OK;
}

int rbc_phase_timing(rbc_ctx *c, int enable, double *out) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (enable) {
    CK(cudaDeviceSynchronize());
    for (cudaEvent_t e : c->ev) c->ev_free.push_back(e);
    c->ev.clear();
    c->timing = true;
    return RBC_OK;
  }
  c->timing = false;
  double fwd = 0, rev = 0;
  const size_t shots = c->ev.size() / 3;
  for (size_t k = 0; k < shots; ++k) {
    float t1 = 0, t2 = 0;
    CK(cudaEventSynchronize(c->ev[3 * k + 2]));
    CK(cudaEventElapsedTime(&t1, c->ev[3 * k], c->ev[3 * k + 1]));
    CK(cudaEventElapsedTime(&t2, c->ev[3 * k + 1], c->ev[3 * k + 2]));
    fwd += t1;
    rev += t2;
  }
  for (cudaEvent_t e : c->ev) c->ev_free.push_back(e);
  c->ev.clear();
  CK(cudaDeviceSynchronize());
  int perr = check_device_error(c);
  if (perr) return perr;
  if (out) {
    out[0] = fwd;
    out[1] = rev;
    out[2] = (double)shots * c->g.nt;
    out[3] = (double)shots * (c->g.nt + 1);
    out[4] = (double)shots;
  }
  return RBC_OK;
}

int rbc_inject_fault(rbc_ctx *c, int mode) {
  if (mode != 0 && mode != 1) return fail(RBC_EINVAL, "unknown fault mode %d", mode);
  if (!c) {  // the next 3-D rbc_model_static call
    static_inject_fault(mode);
    return RBC_OK;
  }
  if (mode == 1 && c->L.ndim != 3) return fail(RBC_ENOTSUP, "fault mode 1 needs a 3-D context");
  c->fault = mode;
  return RBC_OK;
}

int rbc_get_panels(rbc_ctx *c, float *prev_dev, float *last_dev, void *stream) {
  if (!c) return fail(RBC_EINVAL, "ctx is NULL");
  if (!c->have_panels) return fail(RBC_EINVAL, "no forward panels held (run rbc_model first)");
  cudaStream_t s = (cudaStream_t)stream;
  const int nt = c->g.nt;
  if (prev_dev) { launch_copy_out(c->L, c->p[(nt - 1) & 1], prev_dev, s); ++g_launches; }
  if (last_dev) { launch_copy_out(c->L, c->p[nt & 1], last_dev, s); ++g_launches; }
  CKL();
  return RBC_OK;
}

} // extern "C"
