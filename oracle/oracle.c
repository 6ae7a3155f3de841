/*
 * HEALPix RING spherical harmonic transform oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU statement of what the GPU library
 * computes.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product path never does.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Paper: "cuHPX: GPU-Accelerated Differentiable Spherical Harmonic Transforms
 * on HEALPix Grids" (arXiv 2510.01785).
 *   - Grid structure: Sec. III-A (Nside a power of two, Npix = 12 Nside^2,
 *     4 Nside - 1 iso-latitude rings, 4 Nside pixels on the equatorial rings
 *     down to 4 next to the poles, pixels evenly spaced in phi).  The pixel
 *     centres themselves follow Gorski et al. 2005, the grid's definition,
 *     which the paper cites for HEALPix.
 *   - Spherical harmonics and lambda_lm: Eq. 8 (orthonormal Y_lm, lambda is
 *     the normalised prefactor times P_l^m), Eq. 15 (Condon-Shortley (-1)^m
 *     folded into the normalised P_n^m), Eq. 16 (three-term recurrence in l).
 *   - Synthesis operator p = Y a: Eq. 24-25 (ring form, phi_{0,y} offset).
 *   - Analysis operator a = Y^dagger W p: Eq. 26-27, with equal weights
 *     4 pi / Npix from Eq. 1.
 *   - Adjoints: Sec. III-F ("Adjoint Operators"): adjoint of synthesis is
 *     Y^dagger, adjoint of analysis is W Y.
 *
 * Real fields: coefficients are stored for m >= 0 only; a_{l,-m} =
 * (-1)^m conj(a_lm) is implied, so a synthesis reads Re(a_l0) only.
 * Storage: alm[b][idx(l,m)][re,im], idx(l,m) = m(2 lmax + 1 - m)/2 + l;
 * map[b][pixel] in RING order.
 *
 * Two tiers compute the same sums in different groupings, so that each
 * checks the other:
 *   Tier A (direct): every coefficient is the literal double sum over all
 *     pixels of Eq. 26 (resp. every pixel the literal double sum of Eq. 24).
 *   Tier B (separable, Sec. III-D Eq. 13-14): per ring a naive DFT at each
 *     needed m (no FFT), then a Legendre sum over all rings (no north/south
 *     parity trick).  Tier B also evaluates chosen subsets of outputs, which
 *     is how large configurations are checked.
 *
 * lambda_lm is carried as (mantissa, binary exponent) renormalised with
 * frexp after every step, so it is exact to FP64 rounding at any magnitude;
 * it becomes a double (and may underflow to zero) only when it is used.
 * All sums use Neumaier-compensated accumulation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* compensated summation                                                     */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } acc_t;

static inline void acc_add(acc_t *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static inline double acc_val(const acc_t *a) { return a->s + a->c; }

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */
int64_t or_nalm(int lmax, int mmax) {
  return (int64_t)(mmax + 1) * (lmax + 1) - (int64_t)mmax * (mmax + 1) / 2;
}

static inline int64_t alm_index(int lmax, int l, int m) {
  return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

/* Ring y (0-based, north to south).  i = y + 1 is the 1-based ring index.
 * North cap (i < Nside): 4i pixels, z = 1 - i^2/(3 Nside^2), first pixel at
 *   phi = pi/(4i), i.e. phi_x = pi (2x + 1) / N.
 * Belt (Nside <= i <= 3 Nside): 4 Nside pixels, z = (2 Nside - i) 2/(3 Nside),
 *   phi_x = pi (2x + s) / N with s = (i - Nside + 1) mod 2.
 * South cap: mirror of the north cap.
 * sin(theta) is formed from exact integer expressions for (1-z)(1+z). */
static void ring_info(int nside, int y, int64_t *start, int *nphi, double *z,
                      double *sinth, int *sigma) {
  const int64_t ns = nside, npix = 12 * ns * ns;
  const int64_t i = (int64_t)y + 1;
  const int south = i > 2 * ns;
  const int64_t ii = south ? 4 * ns - i : i; /* mirrored into the north */
  if (ii < ns) {
    const double den = 3.0 * (double)(ns * ns);
    *nphi = (int)(4 * ii);
    *sigma = 1;
    *z = 1.0 - (double)(ii * ii) / den;
    *sinth = (double)ii * sqrt((double)(6 * ns * ns - ii * ii)) / den;
    *start = south ? npix - 2 * ii * (ii + 1) : 2 * ii * (ii - 1);
  } else {
    *nphi = (int)(4 * ns);
    *sigma = (int)((i - ns + 1) & 1);
    *z = (double)(2 * (2 * ns - ii)) / (double)(3 * ns);
    *sinth = sqrt((double)((2 * ii - ns) * (7 * ns - 2 * ii))) / (double)(3 * ns);
    *start = 2 * ns * (ns - 1) + 4 * ns * (i - ns);
  }
  if (south) *z = -*z;
}

void or_ring_geometry(int nside, int64_t *start, int32_t *nphi, double *z,
                      double *sinth, int32_t *sigma) {
  const int nring = 4 * nside - 1;
  for (int y = 0; y < nring; y++) {
    int n, s;
    ring_info(nside, y, &start[y], &n, &z[y], &sinth[y], &s);
    nphi[y] = n;
    sigma[y] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* lambda_lm (Eq. 8, 15, 16)                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { double mant; int ex; } sval; /* value = mant * 2^ex */

static inline sval snorm(double v, int ex) {
  sval r;
  int e2 = 0;
  r.mant = frexp(v, &e2);
  r.ex = (r.mant == 0.0) ? 0 : ex + e2;
  return r;
}

/* lambda_mm = (-1)^m sqrt( (1/4pi) prod_{k=1..m} (2k+1)/(2k) ) sin^m(theta) */
static sval lambda_mm(int m, double sinth) {
  sval v = snorm(sqrt(1.0 / (4.0 * M_PI)), 0);
  for (int k = 1; k <= m; k++)
    v = snorm(-v.mant * sqrt((2.0 * k + 1.0) / (2.0 * k)) * sinth, v.ex);
  return v;
}

/* alpha_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)), l > m */
static inline double alpha_lm(int l, int m) {
  const double ld = l, md = m;
  return sqrt((4.0 * ld * ld - 1.0) / (ld * ld - md * md));
}

/* Fill out[l - m] = lambda_lm(z) for l = m..lmax (as doubles; magnitudes
 * below the double range become 0).  If lg2 is non-NULL it also receives
 * log2|lambda| (-inf for an exact zero) and sgn the sign, without
 * underflow.  Recurrence: lambda_lm = alpha_lm (z lambda_{l-1,m}
 * - lambda_{l-2,m} / alpha_{l-1,m}), lambda_{m-1,m} = 0. */
static void lambda_chain_full(int lmax, int m, double z, double sinth,
                              double *out, double *lg2, double *sgn) {
  sval p1 = lambda_mm(m, sinth), p2 = {0.0, 0};
  for (int l = m; l <= lmax; l++) {
    if (l > m) {
      const double a = alpha_lm(l, m);
      const double ainv_prev = (l - 1 > m) ? 1.0 / alpha_lm(l - 1, m) : 0.0;
      int e;
      if (p1.mant == 0.0) e = p2.ex;
      else if (p2.mant == 0.0) e = p1.ex;
      else e = p1.ex > p2.ex ? p1.ex : p2.ex;
      const double t = z * ldexp(p1.mant, p1.ex - e) -
                       ainv_prev * ldexp(p2.mant, p2.ex - e);
      const sval nv = snorm(a * t, e);
      p2 = p1;
      p1 = nv;
    }
    if (out) out[l - m] = ldexp(p1.mant, p1.ex);
    if (lg2) lg2[l - m] = (p1.mant == 0.0) ? -INFINITY
                                           : log2(fabs(p1.mant)) + (double)p1.ex;
    if (sgn) sgn[l - m] = (p1.mant < 0.0) ? -1.0 : (p1.mant > 0.0 ? 1.0 : 0.0);
  }
}

void or_lambda_chain(int lmax, int m, double z, double sinth, double *out) {
  lambda_chain_full(lmax, m, z, sinth, out, NULL, NULL);
}

void or_lambda_chain_log2(int lmax, int m, double z, double sinth, double *lg2,
                          double *sgn) {
  lambda_chain_full(lmax, m, z, sinth, NULL, lg2, sgn);
}

/* ------------------------------------------------------------------------ */
/* ring DFT at chosen frequencies (Sec. III-D Eq. 13, Eq. 26 inner sum)       */
/* ------------------------------------------------------------------------ */
/* G[j] = sum_x p_x exp(-i m_j phi_x), phi_x = pi (2x + sigma) / N.  The angle
 * m phi_x = pi r / N with r = m (2x + sigma) mod 2N reduced exactly in
 * integers; cos/sin of pi r / N come from a per-ring table of 2N entries. */
static void ring_modes(int n, int sigma, const double *p, int nm, const int *ms,
                       double *G /* [nm][2] */) {
  double *cs = (double *)malloc(sizeof(double) * 4 * (size_t)n);
  for (int r = 0; r < 2 * n; r++) {
    const double ang = M_PI * (double)r / (double)n;
    cs[2 * r] = cos(ang);
    cs[2 * r + 1] = sin(ang);
  }
  for (int j = 0; j < nm; j++) {
    const int64_t m = ms[j];
    acc_t re = {0, 0}, im = {0, 0};
    for (int x = 0; x < n; x++) {
      const int64_t r = (m * (2 * (int64_t)x + sigma)) % (2 * (int64_t)n);
      acc_add(&re, p[x] * cs[2 * r]);
      acc_add(&im, -p[x] * cs[2 * r + 1]);
    }
    G[2 * j] = acc_val(&re);
    G[2 * j + 1] = acc_val(&im);
  }
  free(cs);
}

void or_ring_modes(int nphi, int sigma, const double *ring_values, int nm,
                   const int32_t *ms, double *G) {
  ring_modes(nphi, sigma, ring_values, nm, (const int *)ms, G);
}

/* ------------------------------------------------------------------------ */
/* Tier A: direct double sums                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nside, nring;
  int64_t *start;
  int *nphi, *sigma;
  double *z, *sinth;
} geom_t;

static void geom_make(geom_t *g, int nside) {
  g->nside = nside;
  g->nring = 4 * nside - 1;
  g->start = (int64_t *)malloc(sizeof(int64_t) * g->nring);
  g->nphi = (int *)malloc(sizeof(int) * g->nring);
  g->sigma = (int *)malloc(sizeof(int) * g->nring);
  g->z = (double *)malloc(sizeof(double) * g->nring);
  g->sinth = (double *)malloc(sizeof(double) * g->nring);
  for (int y = 0; y < g->nring; y++)
    ring_info(nside, y, &g->start[y], &g->nphi[y], &g->z[y], &g->sinth[y],
              &g->sigma[y]);
}

static void geom_free(geom_t *g) {
  free(g->start); free(g->nphi); free(g->sigma); free(g->z); free(g->sinth);
}

/* lam[(m * nring + y) * (lmax+1) + l] = lambda_lm(z_y), 0 for l < m */
static double *lambda_table(const geom_t *g, int lmax, int mmax) {
  const size_t L = (size_t)lmax + 1;
  double *lam = (double *)calloc((size_t)(mmax + 1) * g->nring * L, sizeof(double));
#pragma omp parallel for schedule(dynamic)
  for (int job = 0; job < (mmax + 1) * g->nring; job++) {
    const int m = job / g->nring, y = job % g->nring;
    lambda_chain_full(lmax, m, g->z[y], g->sinth[y],
                      lam + ((size_t)m * g->nring + y) * L + m, NULL, NULL);
  }
  return lam;
}

/* a_lm[b] = sum_y sum_x map[b][start_y + x] w_y lambda_lm(z_y)
 *           exp(-i m (phi_{0,y} + 2 pi x / N_y))                      (Eq. 26)
 * w = per-ring weights (NULL: all ones). */
void or_map2alm_direct(int nside, int lmax, int mmax, int nbatch,
                       const double *map, const double *w, double *alm,
                       int nthreads) {
  set_threads(nthreads);
  geom_t g;
  geom_make(&g, nside);
  const int64_t npix = 12 * (int64_t)nside * nside, nalm = or_nalm(lmax, mmax);
  const size_t L = (size_t)lmax + 1;
  double *lam = lambda_table(&g, lmax, mmax);
#pragma omp parallel for schedule(dynamic)
  for (int64_t job = 0; job < nalm * nbatch; job++) {
    const int b = (int)(job / nalm);
    const int64_t idx = job % nalm;
    int m = 0;
    while (alm_index(lmax, lmax, m) < idx) m++; /* idx(lmax, m) is the last of column m */
    const int l = (int)(idx - alm_index(lmax, 0, m));
    acc_t re = {0, 0}, im = {0, 0};
    for (int y = 0; y < g.nring; y++) {
      const double lw = lam[((size_t)m * g.nring + y) * L + l] * (w ? w[y] : 1.0);
      const int n = g.nphi[y];
      for (int x = 0; x < n; x++) {
        const int64_t r = ((int64_t)m * (2 * (int64_t)x + g.sigma[y])) % (2 * (int64_t)n);
        const double ang = M_PI * (double)r / (double)n;
        const double v = map[(size_t)b * npix + g.start[y] + x] * lw;
        acc_add(&re, v * cos(ang));
        acc_add(&im, -v * sin(ang));
      }
    }
    alm[2 * ((size_t)b * nalm + idx)] = acc_val(&re);
    alm[2 * ((size_t)b * nalm + idx) + 1] = acc_val(&im);
  }
  free(lam);
  geom_free(&g);
}

/* p_xy[b] = sum_l lambda_l0 Re a_l0 + 2 sum_{m>=1} sum_l lambda_lm
 *           Re(a_lm exp(i m phi_xy))  ( = Eq. 24 summed over +-m ), times
 * scale[y] (NULL: 1). */
void or_alm2map_direct(int nside, int lmax, int mmax, int nbatch,
                       const double *alm, const double *scale, double *map,
                       int nthreads) {
  set_threads(nthreads);
  geom_t g;
  geom_make(&g, nside);
  const int64_t npix = 12 * (int64_t)nside * nside, nalm = or_nalm(lmax, mmax);
  const size_t L = (size_t)lmax + 1;
  double *lam = lambda_table(&g, lmax, mmax);
#pragma omp parallel for schedule(dynamic)
  for (int64_t job = 0; job < npix * nbatch; job++) {
    const int b = (int)(job / npix);
    const int64_t pix = job % npix;
    int y = 0;
    while (y + 1 < g.nring && g.start[y + 1] <= pix) y++;
    const int n = g.nphi[y], x = (int)(pix - g.start[y]);
    acc_t s = {0, 0};
    for (int m = 0; m <= mmax; m++) {
      const int64_t r = ((int64_t)m * (2 * (int64_t)x + g.sigma[y])) % (2 * (int64_t)n);
      const double ang = M_PI * (double)r / (double)n;
      const double c = cos(ang), sn = sin(ang);
      for (int l = m; l <= lmax; l++) {
        const double lam_v = lam[((size_t)m * g.nring + y) * L + l];
        const double *a = alm + 2 * ((size_t)b * nalm + alm_index(lmax, l, m));
        if (m == 0) acc_add(&s, lam_v * a[0]);
        else acc_add(&s, 2.0 * lam_v * (a[0] * c - a[1] * sn));
      }
    }
    map[(size_t)b * npix + pix] = acc_val(&s) * (scale ? scale[y] : 1.0);
  }
  free(lam);
  geom_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Tier B: separable form on chosen outputs                                  */
/* ------------------------------------------------------------------------ */
/* out[b][s] = a_{ls[s], ms[s]}[b] of Eq. 26 with per-ring weights w (NULL: 1).
 * Step 1: per ring, naive DFT at every distinct m in the request.
 * Step 2: per distinct m, lambda chains on every ring, Legendre sums over all
 * rings (Eq. 14). */
void or_map2alm_sep(int nside, int lmax, int nbatch, const double *map,
                    const double *w, int nsamp, const int32_t *ls,
                    const int32_t *ms, double *out, int nthreads) {
  set_threads(nthreads);
  geom_t g;
  geom_make(&g, nside);
  const int64_t npix = 12 * (int64_t)nside * nside;
  /* distinct m values, and the largest l needed for each */
  int mmax = 0;
  for (int s = 0; s < nsamp; s++) if (ms[s] > mmax) mmax = ms[s];
  int *lneed = (int *)malloc(sizeof(int) * (mmax + 1));
  for (int m = 0; m <= mmax; m++) lneed[m] = -1;
  for (int s = 0; s < nsamp; s++) if (ls[s] > lneed[ms[s]]) lneed[ms[s]] = ls[s];
  int nm = 0;
  int *mlist = (int *)malloc(sizeof(int) * (mmax + 1));
  int *mslot = (int *)malloc(sizeof(int) * (mmax + 1));
  for (int m = 0; m <= mmax; m++) {
    mslot[m] = -1;
    if (lneed[m] >= 0) { mslot[m] = nm; mlist[nm++] = m; }
  }
  /* G[((j * nring) + y) * nbatch + b][2] */
  double *G = (double *)malloc(sizeof(double) * 2 * (size_t)nm * g.nring * nbatch);
#pragma omp parallel for schedule(dynamic)
  for (int job = 0; job < g.nring * nbatch; job++) {
    const int y = job / nbatch, b = job % nbatch;
    double *tmp = (double *)malloc(sizeof(double) * 2 * nm);
    ring_modes(g.nphi[y], g.sigma[y], map + (size_t)b * npix + g.start[y], nm,
               mlist, tmp);
    for (int j = 0; j < nm; j++) {
      double *dst = G + 2 * (((size_t)j * g.nring + y) * nbatch + b);
      dst[0] = tmp[2 * j];
      dst[1] = tmp[2 * j + 1];
    }
    free(tmp);
  }
#pragma omp parallel for schedule(dynamic)
  for (int j = 0; j < nm; j++) {
    const int m = mlist[j], lm = lneed[m];
    double *lam = (double *)malloc(sizeof(double) * (size_t)g.nring * (lm - m + 1));
    for (int y = 0; y < g.nring; y++)
      lambda_chain_full(lm, m, g.z[y], g.sinth[y], lam + (size_t)y * (lm - m + 1),
                        NULL, NULL);
    for (int s = 0; s < nsamp; s++) {
      if (ms[s] != m) continue;
      const int l = ls[s];
      for (int b = 0; b < nbatch; b++) {
        acc_t re = {0, 0}, im = {0, 0};
        for (int y = 0; y < g.nring; y++) {
          const double lw = lam[(size_t)y * (lm - m + 1) + (l - m)] * (w ? w[y] : 1.0);
          const double *gv = G + 2 * (((size_t)j * g.nring + y) * nbatch + b);
          acc_add(&re, lw * gv[0]);
          acc_add(&im, lw * gv[1]);
        }
        out[2 * ((size_t)b * nsamp + s)] = acc_val(&re);
        out[2 * ((size_t)b * nsamp + s) + 1] = acc_val(&im);
      }
    }
    free(lam);
  }
  free(G); free(mlist); free(mslot); free(lneed);
  geom_free(&g);
}

/* Synthesis of the chosen rings: out holds, for each b, the pixels of
 * rings[0], rings[1], ... back to back.
 * Step 1: F_m(y)[b] = sum_l a_lm lambda_lm(z_y)  (Re a_l0 for m = 0).
 * Step 2: p_xy = F_0 + 2 sum_{m>=1} Re(F_m exp(i m phi_xy)) by a naive sum,
 * times scale[y] (NULL: 1). */
void or_alm2map_sep(int nside, int lmax, int mmax, int nbatch, const double *alm,
                    const double *scale, int nrings, const int32_t *rings,
                    double *out, int nthreads) {
  set_threads(nthreads);
  geom_t g;
  geom_make(&g, nside);
  const int64_t nalm = or_nalm(lmax, mmax);
  int64_t *ooff = (int64_t *)malloc(sizeof(int64_t) * (nrings + 1));
  ooff[0] = 0;
  for (int k = 0; k < nrings; k++) ooff[k + 1] = ooff[k] + g.nphi[rings[k]];
  const int64_t nout = ooff[nrings];
#pragma omp parallel for schedule(dynamic)
  for (int job = 0; job < nrings * nbatch; job++) {
    const int k = job / nbatch, b = job % nbatch;
    const int y = rings[k], n = g.nphi[y];
    double *F = (double *)malloc(sizeof(double) * 2 * (mmax + 1));
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
    for (int m = 0; m <= mmax; m++) {
      lambda_chain_full(lmax, m, g.z[y], g.sinth[y], lam, NULL, NULL);
      acc_t re = {0, 0}, im = {0, 0};
      for (int l = m; l <= lmax; l++) {
        const double *a = alm + 2 * ((size_t)b * nalm + alm_index(lmax, l, m));
        acc_add(&re, lam[l - m] * a[0]);
        if (m > 0) acc_add(&im, lam[l - m] * a[1]);
      }
      F[2 * m] = acc_val(&re);
      F[2 * m + 1] = acc_val(&im);
    }
    double *cs = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    for (int r = 0; r < 2 * n; r++) {
      const double ang = M_PI * (double)r / (double)n;
      cs[2 * r] = cos(ang);
      cs[2 * r + 1] = sin(ang);
    }
    for (int x = 0; x < n; x++) {
      acc_t s = {0, 0};
      acc_add(&s, F[0]);
      for (int m = 1; m <= mmax; m++) {
        const int64_t r = ((int64_t)m * (2 * (int64_t)x + g.sigma[y])) % (2 * (int64_t)n);
        acc_add(&s, 2.0 * (F[2 * m] * cs[2 * r] - F[2 * m + 1] * cs[2 * r + 1]));
      }
      out[(size_t)b * nout + ooff[k] + x] = acc_val(&s) * (scale ? scale[y] : 1.0);
    }
    free(cs); free(lam); free(F);
  }
  free(ooff);
  geom_free(&g);
}
