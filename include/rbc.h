/*
 * rbc.h -- C ABI of librbc: GB300 (sm_103a) seismic modeling and reverse time
 * migration with random boundary conditions (Barbosa & Coutinho,
 * arXiv:2204.03380).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid.  The velocity model has an interior of nx x ny x nz nodes (ny = 1 for
 * 2-D) padded with nb random-boundary cells on every side (Section 4.3), so
 * the PADDED grid has NX = nx + 2 nb, NY = ny + 2 nb (1 in 2-D), NZ = nz + 2 nb
 * nodes.  Dense arrays are x fastest: element (x, y, z) sits at
 * ((z * NY) + y) * NX + x; interior arrays use (nz, ny, nx) the same way.
 * Node indices passed to the ABI (source, receivers) are in the padded frame;
 * for 2-D grids the y index must be 0.  Beyond the padded grid the pressure is
 * zero (Eq. 1: p = 0 on the domain boundary).
 *
 * Scheme.  Eq. 1 discretised 8th order in space, 2nd order in time (Section
 * 4): p^{n+1} = 2 p^n - p^{n-1} + a L8 p^n - a_s f[n] h^(2-d) delta_s, where
 * a = (v dt / h)^2 and L8 is h^2 times the 8th-order Laplacian.  f[n] drives
 * the step from level n to n+1; records hold levels 0..nt (N_t + 1 samples).
 * Arithmetic is fp32.
 *
 * Memory.  Every pointer named *_dev is device memory on the current CUDA
 * device, owned by the caller, 16-byte aligned (any pointer from cudaMalloc or
 * a PyTorch CUDA tensor).  Pointers named *_host are host memory.  No call
 * allocates memory visible to the caller; an rbc_ctx owns its internal
 * wavefields.  Calls that take a `stream` (a cudaStream_t; NULL = legacy
 * default stream) are asynchronous on it unless stated.
 *
 * Errors.  Every call returns RBC_OK (0) or a positive error code, never
 * throws, and leaves a thread-local message for rbc_last_error().  On an
 * error no work has been queued, except for RBC_ECUDA, which reports a CUDA
 * failure from a launch or a copy.
 */
#ifndef RBC_H_
#define RBC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RBC_OK = 0,
  RBC_EINVAL = 1,   /* bad shape, index outside the grid, NULL pointer      */
  RBC_ECFL = 2,     /* a = (v dt/h)^2 violates the scheme's stability limit  */
  RBC_ENOMEM = 3,   /* device allocation failed                              */
  RBC_ECUDA = 4,    /* CUDA launch / copy failure                            */
  RBC_ETIMEOUT = 5, /* a bounded device wait gave up                         */
  RBC_ENOTSUP = 6   /* option not supported by this build                    */
};

/* Flags of rbc_rtm_shot. */
#define RBC_REINJECT_SOURCE 1 /* reconstruction re-subtracts the source term  */
#define RBC_ZERO_FIRST 2      /* overwrite num/den instead of accumulating    */

/* Padded extents: NX = nx + 2 nb, NY = ny + 2 nb (3-D; 1 in 2-D),
 * NZ = nz + nb + top with top = nb, or 4 with free_surface = 1.  Nodes passed
 * to the calls (sources, receivers) are in this padded frame; interior arrays
 * (num, den, images, stores) cover x in [nb, nb + nx), y in [nb, nb + ny),
 * z in [top, top + nz). */

typedef struct {
  int ndim;         /* 2 or 3                                                 */
  int nx, ny, nz;   /* interior nodes; ny is ignored (taken as 1) for 2-D     */
  int nb;           /* random-boundary cells on each side, >= 2              */
  int free_surface; /* 0: random boundary on every side (padded grid         */
                    /*    nz + 2 nb rows, interior from row nb);             */
                    /* 1: a pressure-release top (Section 5): 4 rows (half   */
                    /*    the stencil length) of zero velocity, a = 0, so    */
                    /*    p = 0 there; nz + nb + 4 rows, interior from row 4 */
  double h;         /* grid spacing dx = dy = dz (m)                          */
  double dt;        /* time step (s)                                          */
  int nt;           /* number of time steps N_t (>= 1)                        */
} rbc_grid;

typedef struct rbc_ctx rbc_ctx;

/*
 * rbc_build_velocity -- pad an interior velocity with a random boundary and
 * form the leapfrog coefficient (Section 4.3, Eqs. 4-5; Algorithm 3 "create
 * a RBC").  With g->free_surface the top 4 rows get v = 0 and a = 0 and the
 * pad distance i is measured from the sides and the bottom only.
 *   v_int_dev: interior velocity (m/s), dense (nz, ny, nx) fp32.
 *   For a pad cell with max-norm distance i (1..nb) into the pad and padded
 *   linear index L, two splitmix64 counter draws U1 = draw(2L+1),
 *   U2 = draw(2L+2) of stream `seed` (each the top 53 bits / 2^53) give
 *     c = lo_i + (hi_i - lo_i) U1,  lo_i/hi_i = min/max(h(i), g(i)) of Eqs. 5/4,
 *     v_rand = v_lo + (v_hi - v_lo) U2,
 *     mode 0 ("blend"):   v = c v_edge + (1 - c) v_rand  (v_edge = nearest
 *                         interior value),
 *     mode 1 ("literal"): v = max(c v_rand, v_lo);
 *   then v = min(v, v_max).  Interior cells keep v_int.  All arithmetic in
 *   fp64, a = (v dt / h)^2 rounded once to fp32.
 *   v_pad_dev (may be NULL): padded velocity, dense (NZ, NY, NX) fp32.
 *   a_dev: padded coefficient, dense (NZ, NY, NX) fp32.
 * Errors: RBC_EINVAL for a bad grid, NULL v_int_dev / a_dev, v_lo > v_hi, or
 * mode not 0/1.
 */
int rbc_build_velocity(const rbc_grid *g, const float *v_int_dev, float v_lo,
                       float v_hi, float v_max, uint64_t seed, int mode,
                       float *v_pad_dev, float *a_dev, void *stream);

/*
 * rbc_create -- make a context for one padded model (Algorithm 4/6 "move data
 * to GPU"): validates the grid, checks stability, allocates the internal
 * wavefields (two panels per wavefield, Algorithm 3) and copies a_dev into
 * the context's aligned, zero-haloed layout.  a_dev (dense (NZ, NY, NX)
 * fp32) is only read during this call.  Synchronous.
 * Stability (the paper requires it of the random velocities, Section 4.3):
 *   max(a) * ndim * 6.5015873 < 4   (6.50... = |symbol of L8| at Nyquist),
 *   else RBC_ECFL.
 * Errors: RBC_EINVAL (bad grid, NULL), RBC_ECFL, RBC_ENOMEM, RBC_ECUDA.
 */
int rbc_create(const rbc_grid *g, const float *a_dev, rbc_ctx **out);

/* rbc_destroy -- free a context (synchronises its device work first).
 * NULL is accepted and ignored. */
int rbc_destroy(rbc_ctx *ctx);

/*
 * rbc_set_coef -- replace the context's coefficient a = (v dt/h)^2 (Eq. 1)
 * with a_dev (dense padded fp32, the layout rbc_create takes), enqueued on
 * `stream`; buffers and captured graphs are kept, so repeated evaluations on
 * one grid (an FWI iteration's updated model) pay no allocation or capture.
 * check = 1 tests stability as rbc_create does (synchronises `stream`; the
 * old coefficient stays on RBC_ECFL); check = 0 skips the test, for an a_dev
 * already checked.  a_dev is read by the copy on `stream` only.
 * Errors: RBC_EINVAL (NULL), RBC_ECFL, RBC_ECUDA.
 */
int rbc_set_coef(rbc_ctx *ctx, const float *a_dev, int check, void *stream);

/*
 * rbc_model -- Algorithm 1 (seismic modeling) for one shot.
 *   src_host: (x, y, z) padded node of the point source.
 *   wavelet_dev: f[0..nt-1] fp32 (f[n] drives step n -> n+1).
 *   rec_host: nrec x (x, y, z) int32 padded receiver nodes (nrec >= 0).
 *   seis_dev: output (nrec, nt + 1) fp32, seis[r][n] = p^n(rec_r).
 * After the call the context holds p^{nt-1} and p^{nt} (the two panels that
 * rbc_rtm_shot would keep), readable with rbc_get_panels.
 * Errors: RBC_EINVAL (NULL, node outside the padded grid), RBC_ENOMEM (the
 * receiver tables could not grow), RBC_ECUDA.
 */
int rbc_model(rbc_ctx *ctx, const int *src_host, const float *wavelet_dev,
              int nrec, const int *rec_host, float *seis_dev, void *stream);

/*
 * rbc_rtm_shot -- Algorithm 3 (RTM with wavefield reconstruction) for one
 * shot, with the imaging condition of Eq. 3 accumulated as two integrals.
 *   Forward: Algorithm 1 without recording; keeps p^{nt-1}, p^{nt}.
 *   Reverse, n = nt .. 0:  num += p^R_n pbar_n,  den += (p^R_n)^2 on the
 *   interior; p^R_{n-1} from Eq. 6 (source re-subtracted when flags has
 *   RBC_REINJECT_SOURCE: the exact inverse of the forward step); pbar_{n-1}
 *   from Eq. 2 with the record injected as + a_r s[r][n] h^(2-d).
 *   seis_dev: (nrec, nt + 1) fp32 record (e.g. from rbc_model).
 *   num_dev, den_dev: interior (nz, ny, nx) fp32, ACCUMULATED (+=), or
 *   overwritten with this shot's integrals when flags has RBC_ZERO_FIRST.
 * Errors: as rbc_model; flags outside RBC_REINJECT_SOURCE | RBC_ZERO_FIRST
 * -> RBC_EINVAL.
 */
int rbc_rtm_shot(rbc_ctx *ctx, const int *src_host, const float *wavelet_dev,
                 int nrec, const int *rec_host, const float *seis_dev,
                 int flags, float *num_dev, float *den_dev, void *stream);

/*
 * rbc_nyquist_stride -- Eq. 7: the source wavefield of RTM with wavefield
 * storage is kept every k = floor(dt_nyq / dt) steps (at least 1), where
 * dt_nyq = 1 / (2 (f_max - f_min)) for the source band [f_min, f_max] in Hz.
 * Returns k >= 1, or 0 when dt <= 0 or not 0 <= f_min < f_max (message in
 * rbc_last_error).  Host only.
 */
int rbc_nyquist_stride(double dt, double f_max, double f_min);

/*
 * rbc_storage_bytes -- size of the store that rbc_rtm_storage needs: the
 * interior box (nz, ny, nx) fp32 of every kept level n = 0, k, 2k, ... <= nt,
 * i.e. 4 nx ny nz (nt / k + 1) bytes.  Returns -1 on a bad grid or k < 1.
 * Host only.
 */
long long rbc_storage_bytes(const rbc_grid *g, int stride);

/*
 * rbc_rtm_storage -- Algorithm 2 (RTM with wavefield storage) for one shot,
 * the baseline that reconstruction (rbc_rtm_shot) replaces; the paper runs
 * it with the Nyquist stride of Eq. 7 and keeps the wavefield on disk, here
 * it stays in device memory.
 *   Forward: Algorithm 1 without recording; level n = j k (j = 0 .. nt / k)
 *   is written to store_dev + j nx ny nz as a dense interior (nz, ny, nx)
 *   fp32 box (the store is an output the caller may read afterwards).
 *   Reverse, n = nt .. 0: at the kept levels num += p^n pbar_n and
 *   den += (p^n)^2 (Eq. 3 integrals sampled every k steps); pbar_{n-1} from
 *   Eq. 2 with the record injected as + a_r s[r][n] h^(2-d).
 *   stride: k >= 1 (rbc_nyquist_stride gives Eq. 7's).
 *   store_dev, store_bytes: caller-owned device memory of at least
 *   rbc_storage_bytes(grid, stride) bytes.
 *   flags: 0 or RBC_ZERO_FIRST; num_dev, den_dev as in rbc_rtm_shot.
 * The context keeps a graph per (store_dev, stride) pair: a call with another
 * pair captures anew.  Afterwards the context holds p^{nt-1}, p^{nt}.
 * Errors: as rbc_rtm_shot; store smaller than needed, stride < 1 or other
 * flags -> RBC_EINVAL.
 */
int rbc_rtm_storage(rbc_ctx *ctx, const int *src_host, const float *wavelet_dev,
                    int nrec, const int *rec_host, const float *seis_dev,
                    int stride, float *store_dev, long long store_bytes,
                    int flags, float *num_dev, float *den_dev, void *stream);

/*
 * rbc_image_stack -- Eq. 3 ratio and Algorithm 3 stacking:
 *   I = num / (den + eps_rel * max(den)) over the shot interior (nz, ny, nx),
 *   image[z][y + off_y][x + off_x] += I[z][y][x]   (survey grid interior),
 * where shot->nz must equal survey->nz and the window must fit.  2-D grids
 * need off_y = 0.  Uses a few bytes of stream-ordered scratch.
 * Errors: RBC_EINVAL (shape, window, NULL), RBC_ECUDA.
 */
int rbc_image_stack(const rbc_grid *shot, const float *num_dev,
                    const float *den_dev, float eps_rel, int off_x, int off_y,
                    const rbc_grid *survey, float *image_dev, void *stream);

/*
 * rbc_fwi_forward -- misfit of one shot for full-waveform inversion (an
 * extension built on Algorithm 1; 2-D grids).
 *   Models the shot like rbc_model, then resid = record - dobs_dev and
 *   misfit_dev += 1/2 sum resid^2 (fp64).  dobs_dev, resid_dev: (nrec, nt + 1)
 *   fp32; misfit_dev: one double; panels_dev (may be NULL): 2 dense padded
 *   fields, p^{nt-1} then p^{nt} -- the only state the gradient needs, since
 *   the random boundary lets rbc_fwi_backward rebuild the wavefield backwards
 *   instead of storing or checkpointing it.
 * Errors: RBC_EINVAL, RBC_ENOTSUP (3-D or free_surface), RBC_ECUDA.
 */
int rbc_fwi_forward(rbc_ctx *ctx, const int *src_host, const float *wavelet_dev,
                    int nrec, const int *rec_host, const float *dobs_dev,
                    float *resid_dev, double *misfit_dev, float *panels_dev,
                    void *stream);

/*
 * rbc_fwi_backward -- gradient of that misfit with respect to the interior
 * velocity (random boundary held fixed), by the exact discrete adjoint of the
 * leapfrog: with mu = a lambda the adjoint is the same recursion run backwards
 * with -a_r resid injected, and
 *   dJ/da_i = -(1/a_i^2) sum_n mu_i^{n+1} (p^{n+1} - 2 p^n + p^{n-1})_i,
 *   dJ/dv_i = dJ/da_i * 2 a_i / v_i,
 * p^n rebuilt backwards from the two panels (Eq. 6 with the source
 * re-subtracted).  resid_dev: from rbc_fwi_forward; panels_dev: the panels
 * it exported, or NULL to use those the context still holds from that call.
 * grad_dev: interior (nz, nx) fp32, ACCUMULATED (+=, by atomic adds, so
 * calls on different contexts and streams may share one grad_dev).
 * Errors: RBC_EINVAL, RBC_ENOTSUP (3-D or free_surface), RBC_ECUDA.
 */
int rbc_fwi_backward(rbc_ctx *ctx, const int *src_host, const float *wavelet_dev,
                     int nrec, const int *rec_host, const float *resid_dev,
                     const float *panels_dev, float *grad_dev, void *stream);

/* ------------------------------------------------------------------------
 * Batched RTM of many 2-D shots of uneven aperture (Algorithm 3's shot loop
 * folded into one launch per time step).
 * ------------------------------------------------------------------------ */
typedef struct rbc_batch rbc_batch;

typedef struct {
  int src[3];            /* source node in the shot's own padded grid (y = 0)  */
  int nrec;              /* receivers of the shot (>= 0)                       */
  const int *rec_host;   /* nrec x (x, 0, z) nodes in the shot's padded grid   */
  const float *seis_dev; /* (nrec, nt + 1) fp32 record                         */
  int off_x;             /* survey image column of the shot's interior x = 0   */
} rbc_shot;

/*
 * rbc_batch_create -- contexts for nshots 2-D shots that share nz, nb, h, dt
 * and nt (taken from g; g->nx is ignored) and have interior widths
 * nx_host[s].  a_dev[s]: the shot's padded (v dt/h)^2, dense (nz + 2nb,
 * nx_host[s] + 2nb) fp32, read during the call.  Checks every shot's
 * stability, lays all fields out in one allocation, and times the candidate
 * tile shapes (rows per warp of the forward and reverse kernels) on the batch
 * to keep the fastest.  Synchronous.
 * Errors: RBC_EINVAL (also for free_surface = 1), RBC_ENOTSUP (3-D), RBC_ECFL,
 * RBC_ENOMEM, RBC_ECUDA.
 */
int rbc_batch_create(const rbc_grid *g, int nshots, const int *nx_host,
                     const float *const *a_dev, rbc_batch **out);

/* rbc_batch_destroy -- free a batch (synchronises first); NULL is ignored. */
int rbc_batch_destroy(rbc_batch *b);

/*
 * rbc_batch_rtm -- Algorithm 3 for every shot of the batch: each time step
 * of the forward phase and of the fused reverse phase is one launch over a
 * work list of (shot, tile) items; then, per shot, I = num / (den + eps_rel
 * max den) (Eq. 3) is stacked into image_dev (nz, survey_nx) at column off_x
 * (+=, shots may overlap).  shots: nshots descriptors (host); flags must be
 * RBC_REINJECT_SOURCE.  The shots run in groups of consecutive shots whose
 * seven fields fit an L2 budget (environment RBC_BATCH_L2MB, megabytes,
 * default 96; 0 = one group), each group's forward then reverse phase, so
 * that a group's fields stay in L2 through its time loops.  Each phase of
 * each group runs as a CUDA graph captured on the first call and replayed
 * afterwards.
 * Errors: RBC_EINVAL (window, nodes, flags), RBC_ENOMEM, RBC_ECUDA.
 */
int rbc_batch_rtm(rbc_batch *b, const rbc_shot *shots, const float *wavelet_dev,
                  int flags, float eps_rel, float *image_dev, int survey_nx,
                  void *stream);

/* rbc_batch_timing -- as rbc_phase_timing, for the forward and reverse
 * phases of every rbc_batch_rtm call while enabled (out[0..4]: forward ms,
 * reverse ms, forward time steps, reverse time steps, calls).  The phases of
 * all shot groups are summed, and a time step counts once however many
 * groups it was launched for, so ms / steps is the time of one step of the
 * whole batch. */
int rbc_batch_timing(rbc_batch *b, int enable, double *out);

/* rbc_batch_info -- out[0..14]: forward and reverse kernels chosen by the
 * autotuner (forward: rows per warp, 0 = the streaming kernel; reverse: 1 or
 * 2 rows per warp, 0 = the streaming kernel, 3 = shared-memory tiles of
 * 8 rows), work items of both kernels, their grids, then the measured
 * per-launch time in microseconds of every candidate on the first shot
 * group: forward streaming / 1 / 2 / 4 rows, reverse 1 / 2 rows / streaming /
 * tiles (0 where a candidate was not timed), then the number of shot groups.
 * Host only. */
int rbc_batch_info(const rbc_batch *b, int *out);

/* ------------------------------------------------------------------------
 * Learned denoiser of random-boundary noise in RTM images (not in the paper:
 * it stands in for stacking K boundary realizations).  Network: five 3x3
 * convolutions 1 -> 32 -> 32 -> 32 -> 32 -> 1 channels, zero padding, ReLU
 * after the first four, the input added to the output.  bf16 operands, fp32
 * accumulation, tensor cores.  Parameters: one fp32 vector of
 * rbc_cnn_param_count() values, [W1 b1 W2 b2 W3 b3 W4 b4 W5 b5], every W
 * stored [tap][out][in] with tap = 3 (dy + 1) + (dx + 1) for the input offset
 * (dy, dx) in {-1, 0, 1}^2.  Images: nimg x H x W fp32, row major.
 * ------------------------------------------------------------------------ */
long long rbc_cnn_param_count(void);

/* Bytes of the caller-owned workspace of rbc_cnn_forward/backward for a
 * batch of nimg H x W images (bf16 activations kept for the backward pass). */
long long rbc_cnn_workspace_bytes(int nimg, int H, int W);

/* y = CNN(x).  ws_dev: workspace of rbc_cnn_workspace_bytes (keeps the
 * activations needed by rbc_cnn_backward).  Errors: RBC_EINVAL, RBC_ECUDA. */
int rbc_cnn_forward(const float *params_dev, int nimg, int H, int W,
                    const float *x_dev, float *y_dev, void *ws_dev,
                    void *stream);

/* y = CNN(x) for inference: the same result as rbc_cnn_forward, without
 * keeping what rbc_cnn_backward needs (the first layer's output is built
 * inside the second layer's kernel and never written to global memory).
 * ws_dev: workspace of rbc_cnn_workspace_bytes, used for the hidden
 * activations.  Errors: RBC_EINVAL, RBC_ECUDA. */
int rbc_cnn_infer(const float *params_dev, int nimg, int H, int W,
                  const float *x_dev, float *y_dev, void *ws_dev,
                  void *stream);

/* grad_dev (param_count fp32) += dL/dparams for the dL/dy in dy_dev, using
 * the activations the preceding rbc_cnn_forward left in ws_dev (same batch,
 * same parameters).  Errors: RBC_EINVAL, RBC_ECUDA. */
int rbc_cnn_backward(const float *params_dev, int nimg, int H, int W,
                     const float *dy_dev, float *grad_dev, void *ws_dev,
                     void *stream);

/* loss_dev (one double) += mean((y - t)^2) over n values; dy_dev (may be
 * NULL) = 2 (y - t) / n.  Errors: RBC_EINVAL, RBC_ECUDA. */
int rbc_cnn_mse(const float *y_dev, const float *t_dev, long long n,
                float *dy_dev, double *loss_dev, void *stream);

/* One Adam step (Kingma & Ba 2015, bias-corrected; step >= 1) on the
 * parameter vector with moment vectors m_dev, v_dev. */
int rbc_cnn_adam(float *params_dev, const float *grad_dev, float *m_dev,
                 float *v_dev, float lr, float b1, float b2, float eps,
                 int step, void *stream);

/*
 * rbc_set_snapshots -- ask the next rbc_model / rbc_rtm_shot on this context
 * to copy wavefields at chosen time levels (Figure 1's propagation and
 * reconstruction panels).  levels_host[k] in [0, nt]; pf_dev / pr_dev / pb_dev
 * (each may be NULL) receive nsnap dense padded (NZ, NY, NX) fp32 fields:
 * pf = forward p^n (both calls), pr = reconstructed p^R_n and pb = receiver
 * pbar_n (rbc_rtm_shot only).  nsnap = 0 clears the request.  The request
 * stays until cleared.  Errors: RBC_EINVAL.
 */
int rbc_set_snapshots(rbc_ctx *ctx, int nsnap, const int *levels_host,
                      float *pf_dev, float *pr_dev, float *pb_dev);

/*
 * rbc_get_panels -- copy the two forward panels kept after the last
 * rbc_model / forward phase (p^{nt-1} -> prev_dev, p^{nt} -> last_dev; dense
 * padded (NZ, NY, NX) fp32; either may be NULL).  Lets a caller checkpoint the
 * reconstruction's initial state (Algorithm 3 "store p_{N-1}, p_N").
 */
int rbc_get_panels(rbc_ctx *ctx, float *prev_dev, float *last_dev,
                   void *stream);

/*
 * rbc_phase_timing -- per-phase device timing with CUDA events recorded on
 * the caller's stream.  enable = 1 clears the record and starts timing the
 * forward and reverse phases of every following rbc_rtm_shot on this
 * context; enable = 0 stops, synchronises and writes out[0] = forward ms,
 * out[1] = reverse ms, out[2] = forward stencil launches, out[3] = reverse
 * stencil launches, out[4] = shots timed (out may be NULL).  The phase times
 * include the few memsets that clear the fields.  Errors: RBC_EINVAL,
 * RBC_ECUDA.
 */
int rbc_phase_timing(rbc_ctx *ctx, int enable, double *out);

/*
 * rbc_model_static -- the same seismic modeling as rbc_model (one shot), for
 * callers that cannot allocate device memory.  The paper has no counterpart:
 * it is an interface addition.
 *   Some callers cannot call cudaMalloc: code that runs while a caching
 *   allocator owns (or has exhausted) the device heap, plugins whose host
 *   runtime forbids allocation on its worker threads, and real-time loops
 *   where an allocation's implicit synchronisation or failure is not
 *   acceptable.  This call needs no context and calls no allocator: its
 *   scratch (coefficient in the zero-haloed layout, two wavefield panels, the
 *   time-major record, the shot tables) lives in one file-scope device array
 *   of 16 MiB (4 Mi floats) inside the library.
 *   Placement of that array: CUDA loads the library's modules lazily by
 *   default, so the array is placed on a device when the first call on that
 *   device looks up its address (with that device current).  A caller whose
 *   heap may be exhausted later should make one small call early (or run with
 *   CUDA_MODULE_LOADING=EAGER, which places it when the CUDA context is
 *   created).  Once placed, it stays until the process exits.  Make the first
 *   call on a device before any stream capture starts.
 *   Arguments are those of rbc_create (grid, a_dev) and rbc_model (source,
 *   wavelet, receivers, seis_dev [nrec][nt + 1] output), all caller-owned.
 *   Grids and records whose scratch exceeds the 16 MiB maximum return
 *   RBC_EINVAL with the needed size in the message; nothing is queued.
 *   All calls on a device share the array and it keeps the previous call's
 *   contents; each call clears its fields itself.  Calls whose work overlaps
 *   on the GPU (other streams or host threads) race on the array: serialise
 *   them.  The stability check of rbc_create runs first and waits on
 *   `stream`.
 *   Failure reporting is deferred, as for contexts: a bounded device wait of
 *   the 3-D kernels that gives up is recorded in the array, and the NEXT call
 *   on that device returns RBC_ETIMEOUT (that earlier record is invalid; the
 *   reporting call does no work and clears the record).
 * Errors: RBC_EINVAL, RBC_ECFL, RBC_ETIMEOUT, RBC_ENOTSUP (free_surface),
 * RBC_ECUDA.
 */
int rbc_model_static(const rbc_grid *g, const float *a_dev,
                     const int *src_host, const float *wavelet_dev, int nrec,
                     const int *rec_host, float *seis_dev, void *stream);

/*
 * rbc_inject_fault -- failure-detection test hook.  mode 1 (3-D contexts):
 * in the next rbc_model / rbc_rtm_shot call, block 0 of the first forward
 * launch never issues one of its TMA plane copies, so that block's bounded
 * mbarrier wait runs out after about a second; the block records the
 * timeout in the context's error word, drains its other copies and leaves,
 * and the next call on the context returns RBC_ETIMEOUT (the results of the
 * faulted call are invalid).  Nothing faults, traps or hangs.  mode 0
 * clears a pending request.  With ctx = NULL the request applies to the next
 * 3-D rbc_model_static call instead (reported by the call after it).
 * Errors: RBC_EINVAL, RBC_ENOTSUP (2-D context).
 */
int rbc_inject_fault(rbc_ctx *ctx, int mode);

/* Thread-local message of the last error on this thread ("" if none). */
const char *rbc_last_error(void);

/* Kernel launches queued by this thread's calls since the counter was last
 * reset (diagnostics for launch accounting); reset=1 zeroes it. */
long long rbc_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* RBC_H_ */
