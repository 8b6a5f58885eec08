// rbc_static.cu -- rbc_model_static: one-shot seismic modeling that allocates
// nothing.
//
// Who needs it: callers that cannot call cudaMalloc -- code running while a
// caching allocator owns (or has exhausted) the device heap, plugins hosted
// by a runtime that forbids allocation on its worker threads, and hard
// real-time loops where an allocation's implicit synchronisation or failure
// is not acceptable.  Instead of a context's cudaMalloc'd wavefields, this
// entry point keeps its scratch (the coefficient in the zero-haloed layout,
// two wavefield panels, the time-major record and the shot tables) in the
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.
//
// Limits and behaviour:
//   * the workspace is kStaticFloats floats (16 MiB); grids and records that
//     need more are rejected with RBC_EINVAL before any work is queued;
//   * all calls on a device share the one array, and it keeps the previous
//     call's contents: every call clears what must start at zero itself, and
//     calls whose work overlaps on the GPU (other streams, other host
//     threads) race on it -- serialise them;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture begins;
//   * the call checks stability like rbc_create, which waits on `stream`.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/rbc.h"
#include "rbc_internal.cuh"

using namespace rbc;

namespace rbc {
int set_error(int code, const char *msg);  // rbc_abi.cu
}

namespace {

constexpr long long kStaticFloats = 4LL << 20;  // 16 MiB of fp32 workspace
static_assert(sizeof(ShotInfo) <= 16 * sizeof(float), "the shot tables must end before the header's words");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_static_ws[kStaticFloats];

std::mutex g_static_mu;
float *g_static_ptr[kMaxDevices] = {nullptr};
// rbc_inject_fault(NULL, 1): the next 3-D call withholds one TMA plane copy
std::atomic<int> g_static_fault{0};


// The record and tables sit after the three fields; 64-float (256-byte)
// alignment keeps every region aligned for float4 access.
long long align64(long long n) { return (n + 63) / 64 * 64; }

__global__ void k_static_sample(const float *__restrict__ p, const int *__restrict__ rec_off, int nrec,
                                float *__restrict__ row) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
    row[r] = p[rec_off[r]];
}

// the library's thread-local error message (read with rbc_last_error)
int set_err(int code, const char *msg) { return rbc::set_error(code, msg); }

// Device address of g_static_ws for the current device (set up once per device).
int static_workspace(float **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_err(RBC_ECUDA, "rbc_model_static: no usable current device");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p) return set_err(RBC_ECUDA, "rbc_model_static: cudaGetSymbolAddress failed");
    g_static_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_static_ptr[dev];
  return RBC_OK;
}

} // namespace

namespace rbc {
// Arm (mode 1) or clear (mode 0) the withheld-copy test fault of the next
// 3-D rbc_model_static call (rbc_inject_fault with a NULL context).
void static_inject_fault(int mode) { g_static_fault.store(mode); }
} // namespace rbc

extern "C" int rbc_model_static(const rbc_grid *g, const float *a_dev, const int *src_host,
                                const float *wavelet_dev, int nrec, const int *rec_host, float *seis_dev,
                                void *stream) {
  if (!g || !a_dev || !src_host || !wavelet_dev || (nrec > 0 && (!rec_host || !seis_dev)) || nrec < 0)
    return set_err(RBC_EINVAL, "rbc_model_static: NULL pointer or negative nrec");
  if ((g->ndim != 2 && g->ndim != 3) || g->nx < 1 || g->nz < 1 || (g->ndim == 3 && g->ny < 1) || g->nb < 2 ||
      g->nt < 1 || !(g->h > 0) || !(g->dt > 0))
    return set_err(RBC_EINVAL, "rbc_model_static: bad grid");
  if (g->free_surface != 0) return set_err(RBC_ENOTSUP, "rbc_model_static: free_surface is not supported");
  // the same layout as a context's fields, extents formed in 64-bit before
  // any 32-bit field is set
  Lay L;
  if (!lay_make(g->ndim, (long long)g->nx + 2LL * g->nb, g->ndim == 3 ? (long long)g->ny + 2LL * g->nb : 1,
                (long long)g->nz + 2LL * g->nb, &L) || L.total > kStaticFloats)
    return set_err(RBC_EINVAL, "rbc_model_static: the grid's fields exceed the static maximum of 4 Mi floats "
                               "(use rbc_create + rbc_model)");
  // A fixed 64-float header holds the shot tables (floats 0..7) and, at
  // floats 16 and 17, the stability maximum and the bounded-wait error word:
  // their place does not depend on the call's sizes, so a call reads the
  // previous call's error word where that call left it.
  const long long o_info = 0;
  const long long o_max = 16;
  const long long o_rec = 64;
  const long long o_wav = o_rec + align64(nrec > 0 ? nrec : 1);
  const long long o_a = o_wav + align64(g->nt);
  const long long o_p0 = o_a + L.total;
  const long long o_p1 = o_p0 + L.total;
  const long long o_seis = o_p1 + L.total;
  const long long need = o_seis + align64((long long)(g->nt + 1) * (nrec > 0 ? nrec : 1));
  if (need > kStaticFloats) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "rbc_model_static: grid and record need %lld floats of workspace; the static maximum is %lld "
             "(use rbc_create + rbc_model)", need, kStaticFloats);
    return set_err(RBC_EINVAL, msg);
  }
  auto node_ok = [&](const int *r) {
    if (r[0] < 0 || r[0] >= L.NX || r[2] < 0 || r[2] >= L.NZ) return false;
    return L.ndim == 2 ? r[1] == 0 : (r[1] >= 0 && r[1] < L.NY);
  };
  if (!node_ok(src_host)) return set_err(RBC_EINVAL, "rbc_model_static: source node outside the padded grid");
  for (int r = 0; r < nrec; ++r)
    if (!node_ok(rec_host + 3 * r)) return set_err(RBC_EINVAL, "rbc_model_static: receiver outside the padded grid");

  float *ws = nullptr;
  int rc = static_workspace(&ws);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  ShotInfo *info = reinterpret_cast<ShotInfo *>(ws + o_info);
  int *rec_off = reinterpret_cast<int *>(ws + o_rec);
  float *wav = ws + o_wav;
  unsigned int *amax = reinterpret_cast<unsigned int *>(ws + o_max);
  float *a = ws + o_a, *p[2] = {ws + o_p0, ws + o_p1}, *seis_t = ws + o_seis;

  // Word 0 of the max slot receives max(a); word 1 is the bounded-wait error
  // word of the 3-D kernels.  The previous call's error word is read back
  // before both are cleared, together with this call's stability check (as
  // rbc_create checks it).
  unsigned int words[2] = {0u, 0u};  // [0]: max(a) bits, [1]: the previous call's error word
  if (cudaMemcpyAsync(&words[1], amax + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned int), s) != cudaSuccess)
    return set_err(RBC_ECUDA, "rbc_model_static: workspace words could not be read or cleared");
  launch_max(a_dev, (long long)L.NX * L.NY * L.NZ, amax, s);
  if (cudaMemcpyAsync(&words[0], amax, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_err(RBC_ECUDA, "rbc_model_static: stability check failed");
  if (words[1] != 0u)
    return set_err(RBC_ETIMEOUT, "rbc_model_static: a bounded wait of the previous call gave up (data in flight "
                                 "did not arrive); that call's record is invalid; this call did no work");
  float am;
  memcpy(&am, &words[0], sizeof am);
  if (!(am * g->ndim * kSymbolMax < 4.0)) return set_err(RBC_ECFL, "rbc_model_static: unstable (v dt/h)^2");

  // tables of this shot
  const double ps = (L.ndim == 3) ? 1.0 / g->h : 1.0;
  ShotInfo hi{};
  hi.src_off = lay_off(L, src_host[0], src_host[1], src_host[2]);
  hi.nrec = nrec;
  hi.src_fwd = (float)ps;
  hi.src_rev = (float)ps;
  hi.rec_scale = (float)ps;
  hi.fault = (L.ndim == 3) ? g_static_fault.exchange(0) : 0;
  std::vector<int> off(nrec > 0 ? nrec : 1);
  for (int r = 0; r < nrec; ++r) off[r] = lay_off(L, rec_host[3 * r], rec_host[3 * r + 1], rec_host[3 * r + 2]);
  // the workspace keeps the last call's contents: clear the three fields
  // (halos included) before this call uses them
  if (cudaMemcpyAsync(info, &hi, sizeof hi, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (nrec > 0 && cudaMemcpyAsync(rec_off, off.data(), sizeof(int) * nrec, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemcpyAsync(wav, wavelet_dev, sizeof(float) * g->nt, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(a, 0, sizeof(float) * 3 * L.total, s) != cudaSuccess)
    return set_err(RBC_ECUDA, "rbc_model_static: copy into the workspace failed");
  launch_copy_in(L, a_dev, a, s);
  StepArgs A{};
  A.L = L;
  A.a = a;
  A.info = info;
  A.wav = wav;
  A.rec_off = rec_off;
  A.seis_t = seis_t;
  A.sample = nrec > 0 ? 1 : 0;
  A.zc = k3dZC;
  A.err = reinterpret_cast<int *>(amax) + 1;  // bounded-wait error word, reported by the next call
  for (int n = 0; n < g->nt; ++n) {
    A.cur = p[n & 1];
    A.nxt = p[(n + 1) & 1];
    A.n = n;
    if (!launch_fwd(A, s)) return set_err(RBC_ECUDA, "rbc_model_static: tensor map encoding failed");
  }
  if (nrec > 0) {
    k_static_sample<<<(nrec + 255) / 256, 256, 0, s>>>(p[g->nt & 1], rec_off, nrec,
                                                         seis_t + (long long)g->nt * nrec);
    launch_transpose(seis_t, seis_dev, g->nt + 1, nrec, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(RBC_ECUDA, cudaGetErrorString(e));
  return RBC_OK;
}
