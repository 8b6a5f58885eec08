/*
 * rbc_oracle.c -- plain, slow FP64 CPU oracle for seismic modeling and reverse
 * time migration with random boundary conditions (Barbosa & Coutinho,
 * arXiv:2204.03380).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm do.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every routine restates the paper's definitions in the paper's order:
 *   - Eq. 1 (acoustic wave equation, source f at r_s, p = dp/dt = 0 at t = 0,
 *     p = 0 on the domain boundary) discretised as Section 4 says: 8th order
 *     in space, 2nd order in time (explicit leapfrog).
 *   - Algorithm 1 (seismic modeling: time loop, record the seismogram near
 *     the surface, N_t + 1 samples per receiver).
 *   - Eqs. 4-5 (linear taper g and Gaussian taper h) and the random boundary
 *     of Section 4.3 (velocities in an N_a-cell pad, coefficients h <= c <= g).
 *   - Eq. 6 (homogeneous reconstruction equation for p^R started from the
 *     last two panels p_{N-1}, p_N), Eq. 2 (receiver back-propagation with
 *     the seismogram as source in reversed time) and Eq. 3 (source-normalised
 *     cross-correlation imaging condition), combined as Algorithm 3 (RTM with
 *     wavefield reconstruction); shot stacking as Algorithm 3's last step.
 *   - Algorithm 2 (RTM with wavefield storage): the forward wavefield kept
 *     every k steps, k from the Nyquist step of Eq. 7, and the Eq. 3
 *     integrals accumulated at the kept levels.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - Stencil weights are the standard 8th-order central second-derivative
 *     weights c0..c4 (the paper prints none).
 *   - Point source of strength f[n] on one node: the discrete delta is
 *     1/dV, dV = h^d, so the step adds -a_s f[n] h^(2-d) (sign from Eq. 1,
 *     where f sits on the right of  lap p - p_tt / v^2).
 *   - Receiver back-propagation injects the data with sign `rec_sign`
 *     (+1 by default; Eq. 3's claim that the image carries the sign of the
 *     reflection coefficient fixes it, checked by the flat-reflector pin).
 *   - Eq. 3 is a ratio of two time integrals: num and den are accumulated
 *     separately and divided once, I = num / (den + eps * max den).
 *   - Reconstruction re-subtracts the source term (the exact discrete
 *     inverse of the forward step); reinject = 0 gives Eq. 6 literally.
 *   - Random boundary: v = c v_edge + (1 - c) v_rand, c ~ U[h_i, g_i],
 *     v_rand ~ U[v_lo, v_hi], i = max-norm cell distance into the pad,
 *     v_edge = nearest interior value, capped at v_max ("blend", mode 0);
 *     mode 1 ("literal") is v = max(c v_rand, v_lo).  Random numbers come
 *     from splitmix64 (Steele, Lea & Flood, OOPSLA 2014) used as a counter
 *     generator: draw j of seed s is mix(s + j * 0x9E3779B97F4A7C15).
 *
 * Arrays are dense, x fastest: index ((z * NY) + y) * NX + x.  For 2-D
 * grids NY = 1 and the y axis carries no stencil.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* 8th-order central weights for d^2/dx^2 times h^2 (Section 4). */
static const double C8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0,
                             8.0 / 315.0, -1.0 / 560.0};

void orc_stencil_weights(double *out) {
  for (int k = 0; k < 5; ++k) out[k] = C8[k];
}

typedef struct {
  int ndim;
  long NX, NY, NZ;
} dims_t;

static dims_t mkdims(int ndim, int NX, int NY, int NZ) {
  dims_t g;
  g.ndim = ndim;
  g.NX = NX;
  g.NY = (ndim == 3) ? NY : 1;
  g.NZ = NZ;
  return g;
}

static long npts(const dims_t *g) { return g->NX * g->NY * g->NZ; }

static long idx(const dims_t *g, long x, long y, long z) {
  return (z * g->NY + y) * g->NX + x;
}

/* p = 0 on and beyond the boundary of the padded grid (Eq. 1). */
static double at(const double *p, const dims_t *g, long x, long y, long z) {
  if (x < 0 || x >= g->NX || y < 0 || y >= g->NY || z < 0 || z >= g->NZ)
    return 0.0;
  return p[idx(g, x, y, z)];
}

/* h^2 * discrete Laplacian at one node: sum over axes of sum_k c_|k| p_{i+k}. */
static double lap8(const double *p, const dims_t *g, long x, long y, long z) {
  double s = 0.0;
  for (int k = -4; k <= 4; ++k) {
    double c = C8[k < 0 ? -k : k];
    s += c * at(p, g, x + k, y, z);
    s += c * at(p, g, x, y, z + k);
    if (g->ndim == 3) s += c * at(p, g, x, y + k, z);
  }
  return s;
}

double orc_lap8_point(int ndim, int NX, int NY, int NZ, const double *p,
                      int x, int y, int z) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  return lap8(p, &g, x, y, z);
}

/* One leapfrog step of Eq. 1 without source:
 *   p_next = 2 p_cur - p_prev + a * L8 p_cur,  a = (v dt / h)^2. */
static void leapfrog(const dims_t *g, const double *a, const double *p_prev,
                     const double *p_cur, double *p_next) {
#pragma omp parallel for schedule(static)
  for (long z = 0; z < g->NZ; ++z)
    for (long y = 0; y < g->NY; ++y)
      for (long x = 0; x < g->NX; ++x) {
        long i = idx(g, x, y, z);
        p_next[i] = 2.0 * p_cur[i] - p_prev[i] + a[i] * lap8(p_cur, g, x, y, z);
      }
}

void orc_leapfrog(int ndim, int NX, int NY, int NZ, const double *a,
                  const double *p_prev, const double *p_cur, double *p_next) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  leapfrog(&g, a, p_prev, p_cur, p_next);
}

/* Point-source scale h^(2-d): the delta of strength 1 on one node is 1/h^d,
 * and a carries dt^2 v^2 / h^2. */
static double point_scale(int ndim, double h) {
  return ndim == 3 ? 1.0 / h : 1.0;
}

static int inside(const dims_t *g, const int *r) {
  long y = (g->ndim == 3) ? r[1] : 0;
  return r[0] >= 0 && r[0] < g->NX && y >= 0 && y < g->NY && r[2] >= 0 &&
         r[2] < g->NZ;
}

static long ridx(const dims_t *g, const int *r) {
  long y = (g->ndim == 3) ? r[1] : 0;
  return idx(g, r[0], y, r[2]);
}

static int in_list(int n, int nlist, const int *list) {
  for (int k = 0; k < nlist; ++k)
    if (list[k] == n) return k;
  return -1;
}

/*
 * Algorithm 1 (seismic modeling) for one shot.
 *   p^{-1} = p^0 = 0;  for n = 0..nt-1:
 *     p^{n+1} = 2 p^n - p^{n-1} + a L8 p^n - a_s f[n] h^(2-d) delta_s
 *   seis[r][n] = p^n(rec_r) for n = 0..nt (N_t + 1 samples, Section 4).
 * Outputs (each may be NULL): seis [nrec][nt+1]; p_prev/p_last = p^{nt-1},
 * p^{nt}; snaps [nsnap][N] = p^{snap_n[k]}.
 * Returns 0, or -1 on a bad argument.
 */
int orc_model(int ndim, int NX, int NY, int NZ, const double *a, double h,
              int nt, const int *src, const double *wavelet, int nrec,
              const int *rec, double *seis, double *p_prev_out,
              double *p_last_out, int nsnap, const int *snap_n,
              double *snaps) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  long N = npts(&g);
  if (nt < 1 || !inside(&g, src)) return -1;
  for (int r = 0; r < nrec; ++r)
    if (!inside(&g, rec + 3 * r)) return -1;
  double *pm = calloc(N, sizeof(double)); /* p^{n-1} */
  double *pc = calloc(N, sizeof(double)); /* p^n     */
  double *pn = calloc(N, sizeof(double)); /* p^{n+1} */
  if (!pm || !pc || !pn) { free(pm); free(pc); free(pn); return -1; }
  long s = ridx(&g, src);
  double ps = point_scale(ndim, h);
  for (int n = 0; n <= nt; ++n) {
    /* record p^n */
    if (seis)
      for (int r = 0; r < nrec; ++r)
        seis[(long)r * (nt + 1) + n] = pc[ridx(&g, rec + 3 * r)];
    int k = in_list(n, nsnap, snap_n);
    if (k >= 0 && snaps) memcpy(snaps + (long)k * N, pc, N * sizeof(double));
    if (n == nt) break;
    leapfrog(&g, a, pm, pc, pn);
    pn[s] -= a[s] * wavelet[n] * ps;
    double *t = pm; pm = pc; pc = pn; pn = t;
  }
  if (p_prev_out) memcpy(p_prev_out, pm, N * sizeof(double));
  if (p_last_out) memcpy(p_last_out, pc, N * sizeof(double));
  free(pm); free(pc); free(pn);
  return 0;
}

/*
 * Algorithm 3 (RTM with wavefield reconstruction) for one shot.
 * Forward: Algorithm 1 without recording, keeping p^{N-1}, p^N.
 * Reverse, for n = N down to 0 (tau = T - t):
 *   image:   num += p^R_n pbar_n,  den += (p^R_n)^2   (Eq. 3, interior only)
 *   Eq. 6:   p^R_{n-1} = 2 p^R_n - p^R_{n+1} + a L8 p^R_n
 *                        - reinject * a_s f[n] h^(2-d) delta_s   (n <= N-1;
 *            p^R_N = p^N, p^R_{N-1} = p^{N-1} are the stored panels)
 *   Eq. 2:   pbar_{n-1} = 2 pbar_n - pbar_{n+1} + a L8 pbar_n
 *                        + rec_sign * sum_r a_r s[r][n] h^(2-d) delta_r
 *            with pbar_{N+1} = pbar_N = 0.
 * num, den: interior boxes [nz][ny][nx] starting at padded node
 * (x, y, z) = (nb, nb, top) (y ignored in 2-D; top = nb, or 4 with a free
 * surface), accumulated (+=).  Snapshots (each may be NULL):
 * pr_snaps/pb_snaps [nsnap][N] = p^R_n, pbar_n for n = snap_n[k].
 */
int orc_rtm_shot(int ndim, int NX, int NY, int NZ, const double *a, double h,
                 int nt, const int *src, const double *wavelet, int nrec,
                 const int *rec, const double *seis, int reinject,
                 double rec_sign, int nb, int top, int nx, int ny, int nz, double *num,
                 double *den, int nsnap, const int *snap_n, double *pr_snaps,
                 double *pb_snaps) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  long N = npts(&g);
  if (ndim == 2) ny = 1;
  long yoff = (ndim == 3) ? nb : 0;
  if (nb + nx > NX || top + nz > NZ || (ndim == 3 && nb + ny > NY)) return -1;
  if (!inside(&g, src)) return -1;
  for (int r = 0; r < nrec; ++r)
    if (!inside(&g, rec + 3 * r)) return -1;
  double *A = malloc(N * sizeof(double));
  double *B = malloc(N * sizeof(double));
  double *C = calloc(N, sizeof(double));
  double *pb_prev = calloc(N, sizeof(double)); /* pbar_{n+1} */
  double *pb_cur = calloc(N, sizeof(double));  /* pbar_n     */
  double *pb_next = calloc(N, sizeof(double)); /* pbar_{n-1} */
  int rc = -1;
  if (!A || !B || !C || !pb_prev || !pb_cur || !pb_next) goto done;
  /* forward: keep the last two panels (Algorithm 3: store p_{N-1}, p_N) */
  rc = orc_model(ndim, NX, NY, NZ, a, h, nt, src, wavelet, 0, NULL, NULL, A, B,
                 0, NULL, NULL);
  if (rc) goto done;
  {
    long s = ridx(&g, src);
    double ps = point_scale(ndim, h);
    double *pr_cur = B;  /* p^R_n     (starts at p^N)       */
    double *pr_next = A; /* p^R_{n-1} (starts at p^{N-1})   */
    double *pr_prev = C; /* p^R_{n+1} (unused at n = N)     */
    for (int n = nt; n >= 0; --n) {
      /* Eq. 3 accumulation at time level n */
      for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
          for (long x = 0; x < nx; ++x) {
            long i = idx(&g, x + nb, y + yoff, z + top);
            long o = (z * ny + y) * nx + x;
            num[o] += pr_cur[i] * pb_cur[i];
            den[o] += pr_cur[i] * pr_cur[i];
          }
      int k = in_list(n, nsnap, snap_n);
      if (k >= 0 && pr_snaps)
        memcpy(pr_snaps + (long)k * N, pr_cur, N * sizeof(double));
      if (k >= 0 && pb_snaps)
        memcpy(pb_snaps + (long)k * N, pb_cur, N * sizeof(double));
      if (n == 0) break;
      /* Eq. 6: reconstruction (p^R_{N-1} is the stored panel) */
      if (n < nt) {
        leapfrog(&g, a, pr_prev, pr_cur, pr_next);
        pr_next[s] -= reinject * a[s] * wavelet[n] * ps;
      }
      /* Eq. 2: receiver wavefield, data injected in reversed time */
      leapfrog(&g, a, pb_prev, pb_cur, pb_next);
      for (int r = 0; r < nrec; ++r) {
        long j = ridx(&g, rec + 3 * r);
        pb_next[j] += rec_sign * a[j] * seis[(long)r * (nt + 1) + n] * ps;
      }
      /* advance one level back in time: (n+1, n, n-1) <- (n, n-1, free) */
      double *t1 = pr_prev; pr_prev = pr_cur; pr_cur = pr_next; pr_next = t1;
      double *t2 = pb_prev; pb_prev = pb_cur; pb_cur = pb_next; pb_next = t2;
    }
  }
done:
  free(A); free(B); free(C);
  free(pb_prev); free(pb_cur); free(pb_next);
  return rc;
}

/*
 * Eq. 7: the Nyquist time step of a source band [f_min, f_max] is
 * dt_nyq = 1 / (2 (f_max - f_min)); the source wavefield is kept every
 * k = floor(dt_nyq / dt) finite-difference steps (at least 1).  The small
 * guard absorbs a ratio such as 9.999999999 that is an integer in exact
 * arithmetic.  Returns 0 on a bad argument.
 */
int orc_nyquist_stride(double dt, double f_max, double f_min) {
  if (!(dt > 0.0) || !(f_max > f_min) || !(f_min >= 0.0)) return 0;
  double dt_nyq = 1.0 / (2.0 * (f_max - f_min));
  double k = floor(dt_nyq / dt + 1e-9);
  return k < 1.0 ? 1 : (int)k;
}

/*
 * Algorithm 2 (RTM with wavefield storage) for one shot, with the source
 * wavefield stored only at the levels n = 0, k, 2k, ... <= N (k = stride,
 * from Eq. 7 in the paper's experiments).
 * Forward: Algorithm 1 (no recording); at every kept level the interior box
 *   of p^n is written to store[n / k] ([nz][ny][nx], the box at padded node
 *   (nb, nb, top)).
 * Reverse, n = N .. 0:
 *   image at kept levels only:  num += p^n pbar_n,  den += (p^n)^2  (Eq. 3
 *     integrals sampled every k steps);
 *   Eq. 2:  pbar_{n-1} = 2 pbar_n - pbar_{n+1} + a L8 pbar_n
 *                        + rec_sign * sum_r a_r s[r][n] h^(2-d) delta_r,
 *   with pbar_{N+1} = pbar_N = 0.
 * store: NULL or (N / k + 1) interior boxes (written).  num, den accumulated.
 * Returns 0, or -1 on a bad argument.
 */
int orc_rtm_storage(int ndim, int NX, int NY, int NZ, const double *a, double h,
                    int nt, const int *src, const double *wavelet, int nrec,
                    const int *rec, const double *seis, double rec_sign,
                    int stride, int nb, int top, int nx, int ny, int nz, double *num,
                    double *den, double *store) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  long N = npts(&g);
  if (ndim == 2) ny = 1;
  long yoff = (ndim == 3) ? nb : 0;
  if (stride < 1 || nt < 1) return -1;
  if (nb + nx > NX || top + nz > NZ || (ndim == 3 && nb + ny > NY)) return -1;
  if (!inside(&g, src)) return -1;
  for (int r = 0; r < nrec; ++r)
    if (!inside(&g, rec + 3 * r)) return -1;
  long nbox = (long)nx * ny * nz;
  long nkeep = nt / stride + 1;
  double *S = store ? store : malloc(nkeep * nbox * sizeof(double));
  double *pm = calloc(N, sizeof(double)); /* p^{n-1} */
  double *pc = calloc(N, sizeof(double)); /* p^n     */
  double *pn = calloc(N, sizeof(double)); /* p^{n+1} */
  int rc = -1;
  if (!S || !pm || !pc || !pn) goto done;
  /* forward (Algorithm 2, first loop): solve Eq. 1, keep every k-th level */
  {
    long s = ridx(&g, src);
    double ps = point_scale(ndim, h);
    for (int n = 0; n <= nt; ++n) {
      if (n % stride == 0) {
        double *box = S + (long)(n / stride) * nbox;
        for (long z = 0; z < nz; ++z)
          for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x)
              box[(z * ny + y) * nx + x] = pc[idx(&g, x + nb, y + yoff, z + top)];
      }
      if (n == nt) break;
      leapfrog(&g, a, pm, pc, pn);
      pn[s] -= a[s] * wavelet[n] * ps;
      double *t = pm; pm = pc; pc = pn; pn = t;
    }
  }
  /* reverse (second loop): receiver wavefield, imaging at the kept levels */
  memset(pm, 0, N * sizeof(double)); /* pbar_{n+1} */
  memset(pc, 0, N * sizeof(double)); /* pbar_n     */
  {
    double ps = point_scale(ndim, h);
    for (int n = nt; n >= 0; --n) {
      if (n % stride == 0) {
        const double *box = S + (long)(n / stride) * nbox;
        for (long z = 0; z < nz; ++z)
          for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
              long o = (z * ny + y) * nx + x;
              double p = box[o];
              num[o] += p * pc[idx(&g, x + nb, y + yoff, z + top)];
              den[o] += p * p;
            }
      }
      if (n == 0) break;
      leapfrog(&g, a, pm, pc, pn);
      for (int r = 0; r < nrec; ++r) {
        long j = ridx(&g, rec + 3 * r);
        pn[j] += rec_sign * a[j] * seis[(long)r * (nt + 1) + n] * ps;
      }
      double *t = pm; pm = pc; pc = pn; pn = t;
    }
  }
  rc = 0;
done:
  if (!store) free(S);
  free(pm); free(pc); free(pn);
  return rc;
}

/* Eq. 3 ratio, formed once: I = num / (den + eps_rel * max(den)). */
void orc_image(long n, const double *num, const double *den, double eps_rel,
               double *img) {
  double m = 0.0;
  for (long i = 0; i < n; ++i) m = den[i] > m ? den[i] : m;
  double e = eps_rel * m;
  for (long i = 0; i < n; ++i) img[i] = num[i] / (den[i] + e);
}

/* Algorithm 3 stacking: survey[z][y+off_y][x+off_x] += shot[z][y][x]. */
void orc_stack(int nx, int ny, int nz, const double *shot, int off_x,
               int off_y, int sx, int sy, double *survey) {
  for (long z = 0; z < nz; ++z)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x)
        survey[(z * sy + y + off_y) * (long)sx + x + off_x] +=
            shot[(z * ny + y) * (long)nx + x];
}

/* Discrete energy of the undamped leapfrog between levels n and n+1:
 *   E = (p1 - p0)^T W (p1 - p0) - p1^T L8 p0,  W = diag(1/a).
 * It is exactly conserved by the source-free recursion (L8 is symmetric). */
double orc_energy(int ndim, int NX, int NY, int NZ, const double *a,
                  const double *p0, const double *p1) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  double e = 0.0;
#pragma omp parallel for reduction(+ : e) schedule(static)
  for (long z = 0; z < g.NZ; ++z)
    for (long y = 0; y < g.NY; ++y)
      for (long x = 0; x < g.NX; ++x) {
        long i = idx(&g, x, y, z);
        double d = p1[i] - p0[i];
        e += d * d / a[i] - p1[i] * lap8(p0, &g, x, y, z);
      }
  return e;
}

/* ---------------- random boundary (Section 4.3, Eqs. 4-5) ---------------- */

/* splitmix64 finaliser (Steele, Lea & Flood 2014). */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The j-th output (j >= 1) of a splitmix64 stream seeded with `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t j) {
  return mix64(seed + j * 0x9E3779B97F4A7C15ULL);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static double unif(uint64_t seed, uint64_t j) {
  return (double)(orc_splitmix64(seed, j) >> 11) * (1.0 / 9007199254740992.0);
}

/* Eq. 4: linear taper g(x) = (Na - x) / (Na - 1), x in [1, Na]. */
double orc_taper_g(double x, int na) { return (na - x) / (double)(na - 1); }

/* Eq. 5: Gaussian taper h(x) = exp(-120 (x - 1)^2 / (Na - 1)^2). */
double orc_taper_h(double x, int na) {
  double u = (x - 1.0) / (double)(na - 1);
  return exp(-120.0 * u * u);
}

static long clampl(long v, long lo, long hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

/* distance (1-based) of padded coordinate q outside the interior [nb, nb+n) */
static long pad_dist(long q, int nb, int n) {
  if (q < nb) return nb - q;
  if (q >= nb + n) return q - (nb + n - 1);
  return 0;
}

/*
 * Pad the interior velocity v_int [nz][ny][nx] with an nb-cell random
 * boundary on every side (Section 4.3) or, with free_surface, on every side
 * but the top, which gets 4 rows (half the stencil length) of v = 0: there
 * a = 0 and p stays 0, the pressure-release surface of Section 5.  The
 * padded grid then has nz + nb + 4 rows and the interior starts at row 4.
 * For a pad cell with max-norm distance i (1..nb) into the pad (measured
 * from the sides and the bottom only when free_surface) and linear index L
 * in the padded grid:
 *   c  = h_i + (g_i - h_i) U_{2L+1},   v_rand = v_lo + (v_hi - v_lo) U_{2L+2}
 *   mode 0: v = min(c v_edge + (1 - c) v_rand, v_max)
 *   mode 1: v = min(max(c v_rand, v_lo), v_max)
 * Optional outputs c_out, vr_out (NaN in the interior) expose the draws.
 */
int orc_rbc_velocity(int ndim, int nx, int ny, int nz, int nb, int free_surface,
                     const double *v_int, double v_lo, double v_hi,
                     double v_max, uint64_t seed, int mode, double *v_pad,
                     double *c_out, double *vr_out) {
  if (nb < 2 || nx < 1 || nz < 1 || (ndim == 3 && ny < 1)) return -1;
  if (ndim == 2) ny = 1;
  long top = free_surface ? 4 : nb;
  long NX = nx + 2L * nb, NZ = nz + nb + top;
  long NY = (ndim == 3) ? ny + 2L * nb : 1;
  for (long z = 0; z < NZ; ++z)
    for (long y = 0; y < NY; ++y)
      for (long x = 0; x < NX; ++x) {
        long L = (z * NY + y) * NX + x;
        if (free_surface && z < top) { /* the zero-pressure rows */
          v_pad[L] = 0.0;
          if (c_out) c_out[L] = NAN;
          if (vr_out) vr_out[L] = NAN;
          continue;
        }
        long dx = pad_dist(x, nb, nx), dz = pad_dist(z, (int)top, nz);
        long dy = (ndim == 3) ? pad_dist(y, nb, ny) : 0;
        long i = dx > dz ? dx : dz;
        i = dy > i ? dy : i;
        long ex = clampl(x - nb, 0, nx - 1), ez = clampl(z - top, 0, nz - 1);
        long ey = (ndim == 3) ? clampl(y - nb, 0, ny - 1) : 0;
        double v_edge = v_int[(ez * ny + ey) * (long)nx + ex];
        if (i == 0) {
          v_pad[L] = v_edge;
          if (c_out) c_out[L] = NAN;
          if (vr_out) vr_out[L] = NAN;
          continue;
        }
        double gi = orc_taper_g((double)i, nb), hi = orc_taper_h((double)i, nb);
        double lo = hi < gi ? hi : gi, up = hi < gi ? gi : hi;
        double c = lo + (up - lo) * unif(seed, 2 * (uint64_t)L + 1);
        double vr = v_lo + (v_hi - v_lo) * unif(seed, 2 * (uint64_t)L + 2);
        double v;
        if (mode == 0) {
          v = c * v_edge + (1.0 - c) * vr;
        } else {
          v = c * vr;
          if (v < v_lo) v = v_lo;
        }
        if (v > v_max) v = v_max;
        v_pad[L] = v;
        if (c_out) c_out[L] = c;
        if (vr_out) vr_out[L] = vr;
      }
  return 0;
}

/* Coefficient of the leapfrog: a = (v dt / h)^2, in fp64 and rounded to fp32. */
void orc_coef(long n, const double *v, double dt, double h, double *a64,
              float *a32) {
  for (long i = 0; i < n; ++i) {
    double c = v[i] * dt / h;
    double a = c * c;
    if (a64) a64[i] = a;
    if (a32) a32[i] = (float)a;
  }
}

/* ------------------- FWI velocity gradient (exact discrete adjoint) -------------------
 * Not in the paper: the gradient of the least-squares misfit of Algorithm 1's
 * record, J = 1/2 sum_n sum_r (p^n(rec_r) - d_obs[r][n])^2, with respect to the
 * interior velocity, the random boundary held fixed.  Written from the
 * Lagrangian of the recursion C_{n+1} = p^{n+1} - 2p^n + p^{n-1} - A L8 p^n - s_n
 * (A = diag(a), s_n = -a_s f[n] h^(2-d) e_s), n = 0..N-1:
 *   adjoint:  lambda^n = 2 lambda^{n+1} - lambda^{n+2} + L8(a lambda^{n+1}) - R^T r_n,
 *             n = N..1, lambda^{N+1} = lambda^{N+2} = 0, r_n = R p^n - d_obs[.][n];
 *   gradient: dJ/da_i = sum_{n=0}^{N-1} lambda_i^{n+1} (-(L8 p^n)_i + delta_is f[n] h^(2-d));
 *             dJ/dv_i = dJ/da_i * 2 a_i / v_i,  v_i = sqrt(a_i) h / dt.
 * p^n is rebuilt backwards from p^{N-1}, p^N (the random boundary keeps the
 * recursion reversible).  grad_v: interior (nz, ny, nx), written.  Returns J.
 */
double orc_fwi_grad(int ndim, int NX, int NY, int NZ, const double *a, double h, double dt, int nt,
                    const int *src, const double *wavelet, int nrec, const int *rec,
                    const double *d_obs, int nb, int nx, int ny, int nz, double *grad_v) {
  dims_t g = mkdims(ndim, NX, NY, NZ);
  long N = npts(&g);
  if (ndim == 2) ny = 1;
  long yoff = (ndim == 3) ? nb : 0;
  double *seis = malloc((size_t)nrec * (nt + 1) * sizeof(double));
  double *pA = malloc(N * sizeof(double)), *pB = malloc(N * sizeof(double)), *pC = calloc(N, sizeof(double));
  double *l0 = calloc(N, sizeof(double)), *l1 = calloc(N, sizeof(double)), *l2 = calloc(N, sizeof(double));
  double *al = calloc(N, sizeof(double)), *ga = calloc(N, sizeof(double));
  double J = 0.0;
  orc_model(ndim, NX, NY, NZ, a, h, nt, src, wavelet, nrec, rec, seis, pA, pB, 0, NULL, NULL);
  for (long k = 0; k < (long)nrec * (nt + 1); ++k) {
    seis[k] -= d_obs[k]; /* residual */
    J += 0.5 * seis[k] * seis[k];
  }
  long s = ridx(&g, src);
  double ps = point_scale(ndim, h);
  double *p_next = pC;  /* p^{n+1} (unused at n = N) */
  double *p_cur = pB;   /* p^n                       */
  double *p_prev = pA;  /* p^{n-1}                   */
  double *lam1 = l1;    /* lambda^{n+1}              */
  double *lam2 = l2;    /* lambda^{n+2}              */
  double *lam0 = l0;    /* lambda^n (being formed)   */
  for (int n = nt; n >= 0; --n) {
    /* gradient term of constraint C_{n+1} */
    if (n <= nt - 1) {
      for (long z = 0; z < g.NZ; ++z)
        for (long y = 0; y < g.NY; ++y)
          for (long x = 0; x < g.NX; ++x) {
            long i = idx(&g, x, y, z);
            double t = -lap8(p_cur, &g, x, y, z);
            if (i == s) t += wavelet[n] * ps;
            ga[i] += lam1[i] * t;
          }
    }
    if (n == 0) break;
    /* adjoint step: lambda^n */
    for (long i = 0; i < N; ++i) al[i] = a[i] * lam1[i];
    for (long z = 0; z < g.NZ; ++z)
      for (long y = 0; y < g.NY; ++y)
        for (long x = 0; x < g.NX; ++x) {
          long i = idx(&g, x, y, z);
          lam0[i] = 2.0 * lam1[i] - lam2[i] + lap8(al, &g, x, y, z);
        }
    for (int r = 0; r < nrec; ++r) lam0[ridx(&g, rec + 3 * r)] -= seis[(long)r * (nt + 1) + n];
    /* rebuild p^{n-1} (stored panel at n = N) */
    if (n < nt) {
      leapfrog(&g, a, p_next, p_cur, p_prev);
      p_prev[s] -= a[s] * wavelet[n] * ps;
    }
    double *t1 = p_next; p_next = p_cur; p_cur = p_prev; p_prev = t1;
    double *t2 = lam2; lam2 = lam1; lam1 = lam0; lam0 = t2;
  }
  for (long z = 0; z < nz; ++z)
    for (long y = 0; y < ny; ++y)
      for (long x = 0; x < nx; ++x) {
        long i = idx(&g, x + nb, y + yoff, z + nb);
        double v = sqrt(a[i]) * h / dt;
        grad_v[(z * ny + y) * (long)nx + x] = ga[i] * 2.0 * a[i] / v;
      }
  free(seis); free(pA); free(pB); free(pC); free(l0); free(l1); free(l2); free(al); free(ga);
  return J;
}

/* J alone (for finite differences): 1/2 sum (record - d_obs)^2. */
double orc_misfit(int ndim, int NX, int NY, int NZ, const double *a, double h, int nt, const int *src,
                  const double *wavelet, int nrec, const int *rec, const double *d_obs) {
  double *seis = malloc((size_t)nrec * (nt + 1) * sizeof(double));
  orc_model(ndim, NX, NY, NZ, a, h, nt, src, wavelet, nrec, rec, seis, NULL, NULL, 0, NULL, NULL);
  double J = 0.0;
  for (long k = 0; k < (long)nrec * (nt + 1); ++k) {
    double r = seis[k] - d_obs[k];
    J += 0.5 * r * r;
  }
  free(seis);
  return J;
}
