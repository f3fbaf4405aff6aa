/*
 * crash_oracle.c -- plain sequential FP64 CPU oracle of one CRASH2-style
 * Monte-Carlo radiative-transfer step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and
 * the benchmark's CPU-baseline leg; never by the product path.  It shares no
 * source with the CUDA library.  Compile with -ffp-contract=off so that every
 * product and sum is rounded on its own, which the bit-exact transport
 * comparison relies on.
 *
 * One step (the step-synchronous scheme of the build):
 *   1. freeze the absorber densities n_HI, n_HeI, n_HeII from the state at the
 *      start of the step (Sec. 2: the cell optical depth sums these species);
 *   2. for each source s, for each of its N_p/N_t packets p (Sec. 3.2) in
 *      index order: draw a direction (Sec. 2: angular emission PDF, isotropic
 *      here), give the packet its share of the source's photons in every
 *      frequency bin (Sec. 2: coloured packets), walk it cell by cell, and in
 *      every crossed cell absorb N_T (1 - exp(-tau)) photons per bin (Eq. 1),
 *      split among H I / He I / He II by their share of tau (Sec. 2), until
 *      the packet is empty or leaves the box (Sec. 2, non-periodic);
 *   3. per cell, integrate the ionisation network and the temperature over
 *      the step with the absorbed photons as the photo-ionisation source,
 *      sub-sampled where the step exceeds the local time-scales (Sec. 3.2).
 *
 * Deposits are integers in units of a per-step photon quantum q = 2^E, so
 * the photon budget closes exactly: emitted = absorbed + escaped.
 * Parity with the paper's own outputs is unpinned (its figures hold no
 * values); the pins are closed forms, invariants and textbook values.
 */
#include "crash_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_BINS 16

/* physical constants (cgs) */
static const double K_B = 1.380649e-16;        /* erg/K */
static const double EV = 1.602176634e-12;      /* erg */
static const double SIGMA_T = 6.6524587321e-25;
static const double A_RAD = 7.565723e-15;      /* erg cm^-3 K^-4 */
static const double M_E = 9.1093837015e-28;
static const double C_LIGHT = 2.99792458e10;

/* ionisation thresholds (eV) of H I, He I, He II */
static const double E_TH[3] = {13.6, 24.6, 54.4};

struct or_ctx {
  int nx, ny, nz;
  int64_t ncell;
  double dl;                 /* cell edge, cm */
  double he_over_h;
  int isothermal, caseB;
  double T_cmb;
  uint64_t seed;
  double f_rec;                               /* > 0: diffuse recombination field */
  int coupling;                               /* 1: photon-conserving chemistry coupling */
  int periodic;                               /* 1: periodic box, light-travel stop */
  double uv_rate[3], uv_heat[3];              /* uniform background: s^-1 per atom, erg */
  double path_limit;                          /* periodic: c dt / dl of this step (cells) */
  uint32_t chem_stride;                       /* timing sample of the per-cell update */
  double dep_scale;
  int chem_pending;                           /* last step ran without chemistry */
  double last_dt;
  double *rec[3];                             /* ground-state recombination photons */
  double *nH, *xHII, *xHeII, *xHeIII, *T;
  double *aHI, *aHeI, *aHeII;                 /* frozen absorber densities */
  int64_t *dHI, *dHeI, *dHeII, *dE;           /* per-step deposits */
  int n_src, n_bins;
  double *pos, *ndot, *binE, *binFrac;
  double sigma[3][OR_MAX_BINS];               /* cm^2 per species and bin */
  double wheat[3][OR_MAX_BINS];               /* excess energy / 2^F per species and bin */
  int heatF;
  int chemistry;
  uint32_t pkt_begin, pkt_end;
  double chem_eps;
  int chem_max_sub, cool_mask;
  uint64_t step;
  int64_t budget[8];
  char err[256];
};

static int fail(or_ctx* c, const char* msg) {
  if (c) snprintf(c->err, sizeof c->err, "%s", msg);
  return -1;
}

/* ------------------------------------------------------------------ RNG */
/* Philox-4x32 with 10 rounds (Salmon et al. 2011): each round multiplies
   counter words 0 and 2 by fixed 32-bit constants, mixes the high halves
   with words 1 and 3 and the key, and the key is bumped by the Weyl
   constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform double in [0,1) from the top 53 bits of a 64-bit word */
static double u01(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)(w >> 11) * 0x1.0p-53;
}

/* Isotropic direction by Marsaglia's (1972) rejection method: draw (v1, v2)
   uniform in the square [-1,1)^2 until s = v1^2 + v2^2 lies in (0, 1), then
   d = (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2 s).  Attempt k uses the Philox
   counter (pkt, src, step, k) under key = seed.  Returns the attempts used,
   or -1 after 64 rejections. */
int or_direction(uint64_t seed, uint32_t step, uint32_t src, uint32_t pkt, double d[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t ctr[4] = {pkt, src, step, k}, r[4];
    or_philox4x32_10(ctr, key, r);
    double v1 = 2.0 * u01(r[0], r[1]) - 1.0;
    double v2 = 2.0 * u01(r[2], r[3]) - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s >= 1.0 || s == 0.0) continue;
    double t = sqrt(1.0 - s);
    d[0] = (2.0 * v1) * t;
    d[1] = (2.0 * v2) * t;
    d[2] = 1.0 - 2.0 * s;
    return (int)k + 1;
  }
  return -1;
}

/* Start of the re-emission packet of a cell (the diffuse recombination
   field of Sec. 2): a point drawn uniformly in the cell and an isotropic
   direction.  The Philox counters are those of a source with index
   0x80000000 | (cell >> 32) and packet cell & 0xffffffff, so no point source
   shares them: the direction takes attempts 0..63 as for a source packet,
   the offsets in the cell take attempts 64 (x, y) and 65 (z), each the top
   31 bits of a 64-bit word times 2^-31, so that cell + offset is exact and
   stays inside the cell. */
static double u31(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)(w >> 33) * 0x1.0p-31;
}

int or_rec_start(uint64_t seed, uint32_t step, int64_t cell, int nx, int ny, double pos[3],
                 double dir[3]) {
  const uint32_t src = 0x80000000u | (uint32_t)((uint64_t)cell >> 32), pkt = (uint32_t)cell;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t c0[4] = {pkt, src, step, 64u}, c1[4] = {pkt, src, step, 65u}, r0[4], r1[4];
  or_philox4x32_10(c0, key, r0);
  or_philox4x32_10(c1, key, r1);
  const int64_t ix = cell % nx, iy = (cell / nx) % ny, iz = cell / ((int64_t)nx * ny);
  pos[0] = (double)ix + u31(r0[0], r0[1]);
  pos[1] = (double)iy + u31(r0[2], r0[3]);
  pos[2] = (double)iz + u31(r1[0], r1[1]);
  return or_direction(seed, step, src, pkt, dir);
}

/* ------------------------------------------------------------ exp(-tau) */
/* exp(-tau) for tau >= 0 by Cody-Waite range reduction and a Taylor
   polynomial: k = rint(x / ln 2), r = (x - k ln2_hi) - k ln2_lo with
   |r| <= ln2/2, e^r = sum_{n<=13} r^n / n! in Horner form, result = 2^k e^r.
   ln2_hi is ln 2 cut to 40 significant bits so that k*ln2_hi is exact.
   tau > 50 returns 0: then N*exp(-tau) < 0.5 for every N < 2^63, so the
   rounded transmitted count is 0 either way. */
double or_exp_neg(double tau) {
  if (!(tau <= 50.0)) return 0.0;
  const double inv_ln2 = 0x1.71547652b82fep+0;
  const double ln2_hi = 0x1.62e42fefa2000p-1;
  const double ln2_lo = 0x1.9ef35793c7673p-41;
  static const double c[14] = {
      0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1,
      0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
      0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
      0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
      0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
  double x = -tau;
  double k = rint(x * inv_ln2);
  double r = (x - k * ln2_hi) - k * ln2_lo;
  double p = c[13];
  for (int n = 12; n >= 0; --n) p = p * r + c[n];
  return ldexp(p, (int)k);
}

/* ------------------------------------------------------- cross sections */
/* Photo-ionisation cross sections at the bin energies (Sec. 2 names the
   three absorbers; the fits are the build's reading): H I and He II
   hydrogenic, sigma_0 (E_th/E)^3 with sigma_0 = 6.30e-18 and 1.58e-18 cm^2;
   He I the Osterbrock (1989) fit 7.83e-18 [1.66 (E/E_th)^-2.05 - 0.66
   (E/E_th)^-3.05] cm^2.  Zero below threshold. */
void or_cross_sections(int n_bins, const double* E, double* sigma) {
  for (int j = 0; j < n_bins; ++j) {
    double e = E[j];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (e >= E_TH[0]) { double r = E_TH[0] / e; s0 = 6.30e-18 * ((r * r) * r); }
    if (e >= E_TH[1]) {
      double y = e / E_TH[1];
      s1 = 7.83e-18 * (1.66 * pow(y, -2.05) + (1.0 - 1.66) * pow(y, -3.05));
    }
    if (e >= E_TH[2]) { double r = E_TH[2] / e; s2 = 1.58e-18 * ((r * r) * r); }
    sigma[0 * n_bins + j] = s0;
    sigma[1 * n_bins + j] = s1;
    sigma[2 * n_bins + j] = s2;
  }
}

/* ceil(log2(x)) for x > 0, exactly, from the binary exponent */
static int ceil_log2(double x) {
  int e;
  double m = frexp(x, &e);          /* x = m 2^e, m in [0.5, 1) */
  return (m == 0.5) ? e - 1 : e;
}

/* ------------------------------------------------------------ context */
or_ctx* oracle_init_grid(const or_grid_desc* d) {
  if (!d || d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || !(d->box_cm > 0)) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  if (!c) return NULL;
  c->nx = d->nx; c->ny = d->ny; c->nz = d->nz;
  c->ncell = (int64_t)d->nx * d->ny * d->nz;
  c->dl = d->box_cm / d->nx;
  c->he_over_h = d->he_over_h;
  c->isothermal = d->isothermal; c->caseB = d->caseB;
  c->T_cmb = d->z_compton >= 0 ? 2.725 * (1.0 + d->z_compton) : 0.0;
  c->seed = d->seed;
  c->f_rec = d->f_rec > 0 ? d->f_rec : 0.0;
  c->coupling = d->coupling ? 1 : 0;
  c->periodic = d->periodic ? 1 : 0;
  for (int s = 0; s < 3; ++s) {
    if (!(d->uv_rate[s] >= 0.0) || !isfinite(d->uv_rate[s]) || !(d->uv_heat_eV[s] >= 0.0) ||
        !isfinite(d->uv_heat_eV[s])) {
      free(c);
      return NULL;
    }
    c->uv_rate[s] = d->uv_rate[s];
    c->uv_heat[s] = d->uv_heat_eV[s] * EV;
  }
  c->path_limit = INFINITY;
  c->chem_stride = 1;
  c->dep_scale = 1.0;
  size_t n = (size_t)c->ncell;
  c->nH = malloc(n * 8); c->xHII = malloc(n * 8); c->xHeII = malloc(n * 8);
  c->xHeIII = malloc(n * 8); c->T = malloc(n * 8);
  c->aHI = calloc(n, 8); c->aHeI = calloc(n, 8); c->aHeII = calloc(n, 8);
  c->dHI = calloc(n, 8); c->dHeI = calloc(n, 8); c->dHeII = calloc(n, 8); c->dE = calloc(n, 8);
  if (c->f_rec > 0)   /* counts of the diffuse field, only when it is on */
    for (int a = 0; a < 3; ++a) c->rec[a] = calloc(n, 8);
  if (!c->nH || !c->xHII || !c->xHeII || !c->xHeIII || !c->T || !c->aHI || !c->aHeI ||
      !c->aHeII || !c->dHI || !c->dHeI || !c->dHeII || !c->dE ||
      (c->f_rec > 0 && (!c->rec[0] || !c->rec[1] || !c->rec[2]))) {
    oracle_free(c);
    return NULL;
  }
  for (size_t i = 0; i < n; ++i) {
    /* densities are single-precision inputs; a uniform value is rounded the same way */
    c->nH[i] = d->n_H ? (double)d->n_H[i] : (double)(float)d->n_H0;
    c->xHII[i] = d->x_HII ? d->x_HII[i] : d->x_HII0;
    c->xHeII[i] = d->x_HeII ? d->x_HeII[i] : d->x_HeII0;
    c->xHeIII[i] = d->x_HeIII ? d->x_HeIII[i] : d->x_HeIII0;
    c->T[i] = d->T ? d->T[i] : d->T0;
  }
  c->chemistry = 1;
  c->pkt_begin = 0; c->pkt_end = 0xFFFFFFFFu;
  c->chem_eps = 0.1; c->chem_max_sub = 10000; c->cool_mask = OR_C_ALL;
  return c;
}

void oracle_free(or_ctx* c) {
  if (!c) return;
  free(c->nH); free(c->xHII); free(c->xHeII); free(c->xHeIII); free(c->T);
  free(c->aHI); free(c->aHeI); free(c->aHeII);
  free(c->dHI); free(c->dHeI); free(c->dHeII); free(c->dE);
  free(c->rec[0]); free(c->rec[1]); free(c->rec[2]);
  free(c->pos); free(c->ndot); free(c->binE); free(c->binFrac);
  free(c);
}

const char* oracle_last_error(or_ctx* c) { return c ? c->err : "null context"; }

int oracle_set_options(or_ctx* c, int chemistry, uint32_t pkt_begin, uint32_t pkt_end,
                       double chem_eps, int chem_max_sub, int cool_mask) {
  if (!c) return -1;
  if (pkt_end < pkt_begin || !(chem_eps > 0) || chem_max_sub < 1)
    return fail(c, "bad options");
  c->chemistry = chemistry; c->pkt_begin = pkt_begin; c->pkt_end = pkt_end;
  c->chem_eps = chem_eps; c->chem_max_sub = chem_max_sub; c->cool_mask = cool_mask;
  return 0;
}

int oracle_set_step_index(or_ctx* c, uint64_t step) {
  if (!c) return -1;
  c->step = step;
  return 0;
}

int oracle_set_chem_sample(or_ctx* c, uint32_t chem_stride, double dep_scale) {
  if (!c) return -1;
  if (chem_stride < 1 || !(dep_scale > 0)) return fail(c, "bad chemistry sample");
  c->chem_stride = chem_stride;
  c->dep_scale = dep_scale;
  return 0;
}

int oracle_add_sources(or_ctx* c, int n_src, const double* pos, const double* ndot,
                       int n_bins, const double* bin_eV, const double* bin_frac) {
  if (!c) return -1;
  if (n_src <= 0 || n_bins <= 0 || n_bins > OR_MAX_BINS) return fail(c, "bad source/bin count");
  for (int s = 0; s < n_src; ++s) {
    if (!(pos[3 * s] >= 0 && pos[3 * s] < c->nx && pos[3 * s + 1] >= 0 &&
          pos[3 * s + 1] < c->ny && pos[3 * s + 2] >= 0 && pos[3 * s + 2] < c->nz))
      return fail(c, "source outside the grid");
    if (!(ndot[s] >= 0)) return fail(c, "negative luminosity");
    for (int j = 0; j < n_bins; ++j)
      if (!(bin_frac[s * n_bins + j] >= 0)) return fail(c, "negative bin fraction");
  }
  for (int j = 0; j < n_bins; ++j)
    if (!(bin_eV[j] > 0)) return fail(c, "non-positive bin energy");
  free(c->pos); free(c->ndot); free(c->binE); free(c->binFrac);
  c->n_src = n_src; c->n_bins = n_bins;
  c->pos = malloc(sizeof(double) * 3 * n_src);
  c->ndot = malloc(sizeof(double) * n_src);
  c->binE = malloc(sizeof(double) * n_bins);
  c->binFrac = malloc(sizeof(double) * n_src * n_bins);
  memcpy(c->pos, pos, sizeof(double) * 3 * n_src);
  memcpy(c->ndot, ndot, sizeof(double) * n_src);
  memcpy(c->binE, bin_eV, sizeof(double) * n_bins);
  memcpy(c->binFrac, bin_frac, sizeof(double) * n_src * n_bins);
  double sig[3 * OR_MAX_BINS];
  or_cross_sections(n_bins, bin_eV, sig);
  /* heating unit 2^F eV with 2^F >= the largest excess energy */
  double emax = 0.0;
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j < n_bins; ++j) {
      c->sigma[s][j] = sig[s * n_bins + j];
      if (bin_eV[j] >= E_TH[s] && bin_eV[j] - E_TH[s] > emax) emax = bin_eV[j] - E_TH[s];
    }
  c->heatF = emax > 1.0 ? ceil_log2(emax) : 0;
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j < n_bins; ++j)
      c->wheat[s][j] = bin_eV[j] >= E_TH[s] ? ldexp(bin_eV[j] - E_TH[s], -c->heatF) : 0.0;
  return 0;
}

int or_freeze_absorbers(or_ctx* c) {
  double y = c->he_over_h;
  for (int64_t i = 0; i < c->ncell; ++i) {
    double nH = c->nH[i];
    double nHe = nH * y;
    c->aHI[i] = nH * (1.0 - c->xHII[i]);
    c->aHeI[i] = nHe * ((1.0 - c->xHeII[i]) - c->xHeIII[i]);
    c->aHeII[i] = nHe * c->xHeII[i];
    c->dHI[i] = 0; c->dHeI[i] = 0; c->dHeII[i] = 0; c->dE[i] = 0;
  }
  return 0;
}

/* ------------------------------------------------------------ transport */
/* Walk one packet cell by cell (Amanatides & Woo 1987 in grid units; ties
   step x before y before z).  In a periodic box (Sec. 2) a packet that
   crosses a face re-enters through the opposite one, and its walk ends
   after the path c dt (the step's path_limit, in cells): the last segment is
   cut there and what the packet still holds is counted with the escaped
   photons (it leaves the step).  In each cell with path l > 0: per bin j,
   tau_j = l * sum_s n_s sigma_s,j; N' = rint(N exp(-tau_j)) (Eq. 1 in
   integer quanta); the absorbed A = N - N' goes to He I and He II by
   rint(A kappa_s / kappa) and the rest to H I (Sec. 2 species split);
   the excess energy sum_s A_s (E_j - E_th,s) / 2^F is rounded once per
   cell.  Stops when every bin is empty or the packet leaves the grid. */
int64_t or_trace_packet(or_ctx* c, const double pos[3], const double dir[3],
                        int64_t* N, int64_t* escaped, int64_t* absorbed,
                        int max_log, int64_t* log_cell, double* log_len, int* n_log) {
  const int nb = c->n_bins;
  const int n[3] = {c->nx, c->ny, c->nz};
  int idx[3], step[3];
  double tMax[3], tDelta[3];
  int64_t crossings = 0;
  if (n_log) *n_log = 0;
  for (int a = 0; a < 3; ++a) {
    idx[a] = (int)floor(pos[a]);
    if (dir[a] > 0) {
      step[a] = 1; tMax[a] = ((double)(idx[a] + 1) - pos[a]) / dir[a]; tDelta[a] = 1.0 / dir[a];
    } else if (dir[a] < 0) {
      step[a] = -1; tMax[a] = ((double)idx[a] - pos[a]) / dir[a]; tDelta[a] = -1.0 / dir[a];
    } else {
      step[a] = 0; tMax[a] = INFINITY; tDelta[a] = INFINITY;
    }
  }
  for (int a = 0; a < 3; ++a)
    if (idx[a] < 0 || idx[a] >= n[a]) {
      for (int j = 0; j < nb; ++j) *escaped += N[j];
      return 0;
    }
  double t = 0.0;
  /* a path of length L crosses at most (|d_x| + |d_y| + |d_z|) L + 3 < 2 L + 3 faces */
  const double tlim = c->periodic ? c->path_limit : INFINITY;
  const int64_t max_iter = c->periodic ? (int64_t)(2.0 * tlim) + 4 : (int64_t)c->nx + c->ny + c->nz + 3;
  for (int64_t it = 0; it < max_iter; ++it) {
    int a = 0;
    if (tMax[1] < tMax[a]) a = 1;
    if (tMax[2] < tMax[a]) a = 2;
    double tn = tMax[a];
    const int stop = tn >= tlim;
    if (stop) tn = tlim;
    double seg = tn - t;
    if (seg > 0) {
      int64_t cell = (int64_t)idx[0] + (int64_t)c->nx * ((int64_t)idx[1] + (int64_t)c->ny * idx[2]);
      double l = seg * c->dl;
      double nHI = c->aHI[cell], nHeI = c->aHeI[cell], nHeII = c->aHeII[cell];
      int64_t aHI = 0, aHeI = 0, aHeII = 0;
      double heat = 0.0;
      int64_t left = 0;
      for (int j = 0; j < nb; ++j) {
        double kHI = nHI * c->sigma[0][j];
        double kHeI = nHeI * c->sigma[1][j];
        double kHeII = nHeII * c->sigma[2][j];
        double kap = (kHI + kHeI) + kHeII;
        double f = or_exp_neg(l * kap);
        int64_t Nj = N[j];
        int64_t Np = llrint((double)Nj * f);
        if (Np > Nj) Np = Nj;
        int64_t A = Nj - Np;
        N[j] = Np;
        left |= Np;
        if (A > 0) {
          int64_t A1 = llrint((double)A * (kHeI / kap));
          if (A1 > A) A1 = A;
          int64_t A2 = llrint((double)A * (kHeII / kap));
          if (A2 > A - A1) A2 = A - A1;
          int64_t A0 = A - A1 - A2;
          aHI += A0; aHeI += A1; aHeII += A2;
          heat += ((double)A0 * c->wheat[0][j] + (double)A1 * c->wheat[1][j]) +
                  (double)A2 * c->wheat[2][j];
        }
      }
      c->dHI[cell] += aHI; c->dHeI[cell] += aHeI; c->dHeII[cell] += aHeII;
      if (!c->isothermal) c->dE[cell] += llrint(heat);
      *absorbed += aHI + aHeI + aHeII;
      ++crossings;
      if (log_cell && *n_log < max_log) {
        log_cell[*n_log] = cell; log_len[*n_log] = seg; ++*n_log;
      }
      if (left == 0) return crossings;
    }
    if (stop) {
      for (int j = 0; j < nb; ++j) *escaped += N[j];
      return crossings;
    }
    t = tn;
    tMax[a] += tDelta[a];
    idx[a] += step[a];
    if (c->periodic) {
      if (idx[a] < 0) idx[a] = n[a] - 1;
      else if (idx[a] >= n[a]) idx[a] = 0;
    } else if (idx[a] < 0 || idx[a] >= n[a]) {
      for (int j = 0; j < nb; ++j) *escaped += N[j];
      return crossings;
    }
  }
  fail(c, "DDA iteration limit");
  return -1;
}

/* ------------------------------------------------------------ chemistry */
/* Rate coefficients.  Recombination: Hui & Gnedin (1997) case A/B fits for
   H II, He II, He III (He III by hydrogenic scaling of H II), dielectronic
   He II recombination of Aldrovandi & Pequignot as used by Cen (1992).
   Collisional ionisation and collisional-excitation cooling: Cen (1992).
   Recombination cooling: Hui & Gnedin (1997).  Bremsstrahlung: 1.42e-27
   g_ff sqrt(T) Z^2 with the Cen (1992) Gaunt factor. */
void or_rates(double T, int caseB, double o[17]) {
  double lHI = 315614.0 / T, lHeI = 570670.0 / T, lHeII = 1263030.0 / T;
  double sq = 1.0 / (1.0 + sqrt(T / 1e5));
  double aHII, aHeII, aHeIII, rcHII, rcHeIII;
  if (caseB) {
    aHII = 2.753e-14 * pow(lHI, 1.5) / pow(1.0 + pow(lHI / 2.740, 0.407), 2.242);
    aHeII = 1.26e-14 * pow(lHeI, 0.750);
    aHeIII = 2.0 * 2.753e-14 * pow(lHeII, 1.5) / pow(1.0 + pow(lHeII / 2.740, 0.407), 2.242);
    rcHII = 3.435e-30 * T * pow(lHI, 1.970) / pow(1.0 + pow(lHI / 2.250, 0.376), 3.720);
    rcHeIII = 8.0 * 3.435e-30 * (0.25 * T) * pow(lHeII, 1.970) /
              pow(1.0 + pow(lHeII / 2.250, 0.376), 3.720);
  } else {
    aHII = 1.269e-13 * pow(lHI, 1.503) / pow(1.0 + pow(lHI / 0.522, 0.470), 1.923);
    aHeII = 3.0e-14 * pow(lHeI, 0.654);
    aHeIII = 2.0 * 1.269e-13 * pow(lHeII, 1.503) / pow(1.0 + pow(lHeII / 0.522, 0.470), 1.923);
    rcHII = 1.778e-29 * T * pow(lHI, 1.965) / pow(1.0 + pow(lHI / 0.541, 0.502), 2.697);
    rcHeIII = 8.0 * 1.778e-29 * (0.25 * T) * pow(lHeII, 1.965) /
              pow(1.0 + pow(lHeII / 0.541, 0.502), 2.697);
  }
  double adiel = 1.90e-3 * pow(T, -1.5) * exp(-470000.0 / T) * (1.0 + 0.3 * exp(-94000.0 / T));
  double bHI = 5.85e-11 * sqrt(T) * exp(-157809.1 / T) * sq;
  double bHeI = 2.38e-11 * sqrt(T) * exp(-285335.4 / T) * sq;
  double bHeII = 5.68e-12 * sqrt(T) * exp(-631515.0 / T) * sq;
  double lg = log10(T);
  double gff = 1.1 + 0.34 * exp(-(5.5 - lg) * (5.5 - lg) / 3.0);
  o[0] = aHII; o[1] = aHeII; o[2] = aHeIII; o[3] = adiel;
  o[4] = bHI; o[5] = bHeI; o[6] = bHeII;
  o[7] = 7.50e-19 * exp(-118348.0 / T) * sq;                        /* exc HI */
  o[8] = 5.54e-17 * pow(T, -0.397) * exp(-473638.0 / T) * sq;       /* exc HeII */
  o[9] = E_TH[0] * EV * bHI;                                        /* ion HI */
  o[10] = E_TH[1] * EV * bHeI;                                      /* ion HeI */
  o[11] = E_TH[2] * EV * bHeII;                                     /* ion HeII */
  o[12] = rcHII;                                                    /* rec HII */
  o[13] = K_B * T * aHeII;                                          /* rec HeII */
  o[14] = rcHeIII;                                                  /* rec HeIII */
  o[15] = 6.526e-11 * adiel;                                        /* dielectronic */
  o[16] = 1.42e-27 * gff * sqrt(T);                                 /* brems per Z^2 */
}

/* Compton exchange with the CMB per electron: 4 sigma_T a T_cmb^4 k / (m_e c)
   times (T - T_cmb). */
double or_compton_coef(double T_cmb) {
  double t2 = T_cmb * T_cmb;
  return 4.0 * SIGMA_T * A_RAD * (t2 * t2) * K_B / (M_E * C_LIGHT);
}

/* cooling rate (erg cm^-3 s^-1) excluding Compton */
static double cooling(const double* r, int mask, double ne, double nHI, double nHII,
                      double nHeI, double nHeII, double nHeIII) {
  double L = 0.0;
  if (mask & OR_C_COLL_EXC) L += ne * (r[7] * nHI + r[8] * nHeII);
  if (mask & OR_C_COLL_ION) L += ne * (r[9] * nHI + r[10] * nHeI + r[11] * nHeII);
  if (mask & OR_C_RECOMB) L += ne * (r[12] * nHII + r[13] * nHeII + r[14] * nHeIII);
  if (mask & OR_C_DIELEC) L += ne * r[15] * nHeII;
  if (mask & OR_C_BREMS) L += ne * r[16] * (nHII + nHeII + 4.0 * nHeIII);
  return L;
}

/* Ionisation network + temperature of one cell over dt (Sec. 2 lists the
   network and the continuous processes; Sec. 3.2 sub-samples it when dt
   exceeds the local time-scales).  Each sub-step h:
     * h = min(remaining, eps max(v, 1e-3) / |dv/dt|) over the ionic
       fractions v (and eps T / |dT/dt|), the last allowed sub-step taking
       the remainder;
     * backward Euler for the H (2-state) and He (3-state) chains at fixed
       T, with n_e taken at the end of the sub-step by at most 4 fixed-point
       passes (fewer once n_e changes by less than 1e-12 relative);
     * temperature from the energy balance 1.5 k (n_tot T)' = H - Lambda,
       cooling linear in the new T (semi-implicit), photo-heating = mean
       excess energy per absorbed photon times the photo-ionisations of the
       new absorbers.
   Returns the number of sub-steps. */
int or_chem_cell(or_chem_t* c, double dt) {
  const double nH = c->nH, nHe = c->nHe;
  const int mask = c->cool_mask;
  const int use_coll = (mask & OR_C_COLL_ION) != 0;
  const int use_rec = (mask & OR_C_RECOMB) != 0;
  const double ccomp = (c->T_cmb > 0 && (mask & OR_C_COMPTON)) ? or_compton_coef(c->T_cmb) : 0.0;
  double x = c->xHII, y2 = c->xHeII, y3 = c->xHeIII, T = c->T;
  double rem = dt;
  int nsub = 0;
  double r[17], rB[17];
  while (rem > 0) {
    or_rates(T, c->caseB, r);
    if (c->count_rec) or_rates(T, 1, rB);     /* case B at the same temperature */
    double aH = use_rec ? r[0] : 0.0, aHe2 = use_rec ? r[1] + ((mask & OR_C_DIELEC) ? r[3] : 0.0) : 0.0;
    double aHe3 = use_rec ? r[2] : 0.0;
    double bH = use_coll ? r[4] : 0.0, bHe1 = use_coll ? r[5] : 0.0, bHe2 = use_coll ? r[6] : 0.0;
    double y1 = (1.0 - y2) - y3;
    double ne = nH * x + nHe * (y2 + 2.0 * y3);
    /* derivatives at the start of the sub-step */
    /* photo-ionisation by the deposits and by the uniform background */
    const double GH = c->G_HI + c->U_HI, G1 = c->G_HeI + c->U_HeI, G2 = c->G_HeII + c->U_HeII;
    double IH = GH + bH * ne, RH = aH * ne;
    double I1 = G1 + bHe1 * ne, R2 = aHe2 * ne, I2 = G2 + bHe2 * ne, R3 = aHe3 * ne;
    /* constant-count photo-ionisation sources (photon-conserving coupling),
       for the step size at most what the atoms present can take over the
       time left (a used-up species does not shorten the sub-steps) */
    double sH = fmin(c->S_HI, (1.0 - x) / rem);
    double s1 = fmin(c->S_HeI, y1 / rem);
    double s2 = fmin(c->S_HeII, y2 / rem);
    double dx = (sH + IH * (1.0 - x)) - RH * x;
    double dy1 = (-I1 * y1 + R2 * y2) - s1;
    double dy3 = (s2 + I2 * y2) - R3 * y3;
    double dy2 = -dy1 - dy3;
    double h = rem;
    double v[5] = {1.0 - x, x, y1, y2, y3};
    double dv[5] = {-dx, dx, dy1, dy2, dy3};
    int nv = nHe > 0 ? 5 : 2;
    for (int i = 0; i < nv; ++i) {
      double fl = v[i] > 1e-3 ? v[i] : 1e-3;
      double ad = fabs(dv[i]);
      if (ad * h > c->eps * fl) h = c->eps * fl / ad;
    }
    double ntot = nH + nHe + ne;
    if (!c->isothermal) {
      double nHI = nH * (1.0 - x), nHII = nH * x;
      double heat = c->heat_per_ion * (c->G_HI * nHI + c->G_HeI * nHe * y1 + c->G_HeII * nHe * y2) +
                    c->heat_rate +
                    ((c->U_HI * c->Ue_HI) * nHI + (c->U_HeI * c->Ue_HeI) * (nHe * y1) +
                     (c->U_HeII * c->Ue_HeII) * (nHe * y2));
      double L = cooling(r, mask, ne, nHI, nHII, nHe * y1, nHe * y2, nHe * y3) +
                 ccomp * ne * (T - c->T_cmb);
      double dne = nH * dx + nHe * (dy2 + 2.0 * dy3);
      double dT = ((heat - L) / (1.5 * K_B) - T * dne) / ntot;
      double adT = fabs(dT);
      if (adT * h > c->eps * T) h = c->eps * T / adT;
    }
    if (nsub == c->max_sub - 1 || !(h < rem)) h = rem;
    /* the sources of the sub-step ionise at most the atoms present (He II
       also what He I gives it): the photons beyond are lost */
    sH = fmin(c->S_HI, (1.0 - x) / h);
    s1 = fmin(c->S_HeI, y1 / h);
    s2 = fmin(c->S_HeII, y2 / h + s1);
    /* backward Euler with n_e from the end of the sub-step */
    double xn = x, y1n = y1, y2n = y2, y3n = y3, nen = ne;
    for (int it = 0; it < 4; ++it) {
      double IHn = GH + bH * nen, RHn = aH * nen;
      xn = (x + h * (sH + IHn)) / (1.0 + h * (IHn + RHn));
      if (nHe > 0) {
        double i1 = G1 + bHe1 * nen, r2 = aHe2 * nen;
        double i2 = G2 + bHe2 * nen, r3 = aHe3 * nen;
        double a11 = 1.0 + h * i1, a12 = -h * r2;
        double a21 = -h * i1, a22 = 1.0 + h * (r2 + i2), a23 = -h * r3;
        double a32 = -h * i2, a33 = 1.0 + h * r3;
        /* right-hand side: the old fractions plus the constant sources */
        double b1 = y1 - h * s1, b2 = y2 + h * (s1 - s2), b3 = y3 + h * s2;
        double c1 = a12 / a11, d1 = b1 / a11;
        double m2 = a22 - a21 * c1;
        double c2 = a23 / m2, d2 = (b2 - a21 * d1) / m2;
        double m3 = a33 - a32 * c2;
        y3n = (b3 - a32 * d2) / m3;
        y2n = d2 - c2 * y3n;
        y1n = d1 - c1 * y2n;
      }
      double ne_it = nH * xn + nHe * (y2n + 2.0 * y3n);
      int converged = fabs(ne_it - nen) <= 1e-12 * ne_it;
      nen = ne_it;
      if (converged) break;
    }
    if (xn < 0.0) xn = 0.0;
    if (xn > 1.0) xn = 1.0;
    if (nHe > 0) {
      if (y1n < 0.0) y1n = 0.0;
      if (y2n < 0.0) y2n = 0.0;
      if (y3n < 0.0) y3n = 0.0;
      double s = (y1n + y2n) + y3n;
      y2n = y2n / s;
      y3n = y3n / s;
      y1n = (1.0 - y2n) - y3n;
    }
    double nen2 = nH * xn + nHe * (y2n + 2.0 * y3n);
    if (!c->isothermal) {
      double nHI = nH * (1.0 - xn), nHII = nH * xn;
      double heat = c->heat_per_ion * (c->G_HI * nHI + c->G_HeI * nHe * y1n + c->G_HeII * nHe * y2n) +
                    c->heat_rate +
                    ((c->U_HI * c->Ue_HI) * nHI + (c->U_HeI * c->Ue_HeI) * (nHe * y1n) +
                     (c->U_HeII * c->Ue_HeII) * (nHe * y2n));
      double L = cooling(r, mask, nen2, nHI, nHII, nHe * y1n, nHe * y2n, nHe * y3n);
      double L1 = L / T;
      double C = ccomp * nen2;
      double ntot2 = nH + nHe + nen2;
      T = (1.5 * K_B * ntot * T + h * (heat + C * c->T_cmb)) / (1.5 * K_B * ntot2 + h * (L1 + C));
    }
    if (c->count_rec && use_rec) {
      /* recombinations straight to the ground state, alpha_A - alpha_B of
         each ion (at least 0) at the sub-step's starting temperature, with
         n_e and the ions at the end of the sub-step as in the backward-Euler
         update */
      double gH = r[0] - rB[0], g2 = r[1] - rB[1], g3 = r[2] - rB[2];
      if (gH < 0.0) gH = 0.0;
      if (g2 < 0.0) g2 = 0.0;
      if (g3 < 0.0) g3 = 0.0;
      c->rec[0] += h * gH * nen2 * (nH * xn);
      if (nHe > 0) {
        c->rec[1] += h * g2 * nen2 * (nHe * y2n);
        c->rec[2] += h * g3 * nen2 * (nHe * y3n);
      }
    }
    x = xn; y2 = y2n; y3 = y3n;
    rem = (h == rem) ? 0.0 : rem - h;
    ++nsub;
  }
  c->xHII = x; c->xHeII = y2; c->xHeIII = y3; c->T = T;
  return nsub;
}

/* The per-cell update of a step (Sec. 2 network and continuous processes,
   sub-sampled as in Sec. 3.2) from the deposits the context holds, with the
   step's photon quantum 2^E. */
static void or_step_chemistry(or_ctx* c, double dt, int E) {
  const double V = (c->dl * c->dl) * c->dl;
  const double q = ldexp(1.0, E);
  const double qE = ldexp(1.0, E + c->heatF) * EV;   /* erg per heat unit */
  int64_t subs = 0;
  for (int64_t i = 0; i < c->ncell; ++i) {
    if (c->chem_stride > 1 && (uint64_t)i % c->chem_stride != 0) continue;   /* timing sample */
    or_chem_t ch;
    ch.nH = c->nH[i];
    ch.nHe = c->nH[i] * c->he_over_h;
    ch.xHII = c->xHII[i]; ch.xHeII = c->xHeII[i]; ch.xHeIII = c->xHeIII[i]; ch.T = c->T[i];
    const double dHI = (double)c->dHI[i] * c->dep_scale, dHeI = (double)c->dHeI[i] * c->dep_scale;
    const double dHeII = (double)c->dHeII[i] * c->dep_scale, dE = (double)c->dE[i] * c->dep_scale;
    ch.S_HI = ch.S_HeI = ch.S_HeII = 0.0;
    ch.heat_rate = 0.0;
    /* the uniform background acts in every cell, whatever the deposits */
    ch.U_HI = c->uv_rate[0]; ch.U_HeI = c->uv_rate[1]; ch.U_HeII = c->uv_rate[2];
    ch.Ue_HI = c->uv_heat[0]; ch.Ue_HeI = c->uv_heat[1]; ch.Ue_HeII = c->uv_heat[2];
    if (!c->coupling) {
      /* photo-ionisation rate per absorber frozen at the start of the step */
      double NHI = c->aHI[i] * V, NHeI = c->aHeI[i] * V, NHeII = c->aHeII[i] * V;
      ch.G_HI = NHI > 0 ? (dHI * q) / (dt * NHI) : 0.0;
      ch.G_HeI = NHeI > 0 ? (dHeI * q) / (dt * NHeI) : 0.0;
      ch.G_HeII = NHeII > 0 ? (dHeII * q) / (dt * NHeII) : 0.0;
      int64_t nabs = (c->dHI[i] + c->dHeI[i]) + c->dHeII[i];
      ch.heat_per_ion = nabs > 0 ? (dE * qE) / (((double)nabs * c->dep_scale) * q) : 0.0;
    } else {
      /* photon-conserving: every absorbed photon ionises one atom of its
         species, at a constant rate over the step (per atom of the element:
         H for H I, He for He I and He II); the excess energy heats at a
         constant rate */
      double NH = ch.nH * V, NHe = ch.nHe * V;
      ch.G_HI = ch.G_HeI = ch.G_HeII = 0.0;
      ch.heat_per_ion = 0.0;
      ch.S_HI = NH > 0 ? (dHI * q) / (dt * NH) : 0.0;
      ch.S_HeI = NHe > 0 ? (dHeI * q) / (dt * NHe) : 0.0;
      ch.S_HeII = NHe > 0 ? (dHeII * q) / (dt * NHe) : 0.0;
      ch.heat_rate = (dE * qE) / (dt * V);
    }
    /* with the diffuse field on, recombinations to the ground state are
       no longer absorbed on the spot: case A, and they are counted */
    ch.isothermal = c->isothermal; ch.caseB = c->f_rec > 0 ? 0 : c->caseB; ch.T_cmb = c->T_cmb;
    ch.eps = c->chem_eps; ch.max_sub = c->chem_max_sub; ch.cool_mask = c->cool_mask;
    ch.count_rec = c->f_rec > 0;
    ch.rec[0] = ch.rec[1] = ch.rec[2] = 0.0;
    subs += or_chem_cell(&ch, dt);
    c->xHII[i] = ch.xHII; c->xHeII[i] = ch.xHeII; c->xHeIII[i] = ch.xHeIII; c->T[i] = ch.T;
    if (ch.count_rec)
      for (int a = 0; a < 3; ++a) c->rec[a][i] += ch.rec[a] * V;
  }
  c->budget[7] = subs;
}

/* ------------------------------------------------------------ one step */
int oracle_step(or_ctx* c, double dt, uint64_t P) {
  if (!c) return -1;
  if (c->n_src <= 0) return fail(c, "no sources");
  if (!(dt > 0)) return fail(c, "dt must be positive");
  if (P == 0 || P % (uint64_t)c->n_src) return fail(c, "packets_per_step must be a positive multiple of n_src");
  uint64_t Ns = P / (uint64_t)c->n_src;
  if (Ns > 0xFFFFFFFFull) return fail(c, "too many packets per source");
  const int nb = c->n_bins;
  or_freeze_absorbers(c);
  memset(c->budget, 0, sizeof c->budget);
  /* periodic box: a packet travels at most c dt in the step (in cells) */
  c->path_limit = c->periodic ? (C_LIGHT * dt) / c->dl : INFINITY;
  if (c->periodic && !(c->path_limit <= 536870912.0))
    return fail(c, "periodic box: the light-travel distance of the step exceeds 2^29 cells");

  /* photon quantum q = 2^E with the step's photons of all sources,
     (sum_s ndot_s) dt / q, at most 2^62 (the sum taken in source order) */
  double tot = 0.0;
  for (int s = 0; s < c->n_src; ++s) tot += c->ndot[s];
  double X = tot * dt;
  int E = X > 0 ? ceil_log2(X) - 62 : 0;
  if (c->f_rec > 0) {
    /* the diffuse field re-emits this step at most ncell times the largest
       count over its threshold: the quantum also keeps that below 2^62, and
       one more bit keeps sources plus re-emission below 2^62 */
    const double V = (c->dl * c->dl) * c->dl;
    double rmax = 0.0;
    for (int64_t i = 0; i < c->ncell; ++i) {
      const double atoms[3] = {c->nH[i] * V, c->nH[i] * c->he_over_h * V,
                               c->nH[i] * c->he_over_h * V};
      for (int a = 0; a < 3; ++a) {
        const double v = c->rec[a][i];
        if (atoms[a] > 0 && v > 0 && v >= c->f_rec * atoms[a] && v > rmax) rmax = v;
      }
    }
    if (rmax > 0) {
      const int Er = ceil_log2(rmax * (double)c->ncell) - 62;
      if (Er > E) E = Er;
    }
    E += 1;
  }
  c->budget[5] = E;
  c->budget[6] = c->heatF;

  uint32_t pb = c->pkt_begin, pe = c->pkt_end;
  if ((uint64_t)pe > Ns) pe = (uint32_t)Ns;
  int64_t emitted = 0, escaped = 0, absorbed = 0, crossings = 0, traced = 0;
  int64_t Bj[OR_MAX_BINS], N[OR_MAX_BINS];
  for (int s = 0; s < c->n_src; ++s) {
    /* the source's photons this step in quanta, split over bins by the
     cumulative SED fractions, the last bin taking the remainder */
    int64_t B = llrint(ldexp(c->ndot[s] * dt, -E));
    double F = 0.0;
    int64_t prev = 0;
    for (int j = 0; j < nb; ++j) {
      int64_t Cj;
      if (j == nb - 1) {
        Cj = B;
      } else {
        F = F + c->binFrac[s * nb + j];
        Cj = (int64_t)floor((double)B * F);
        if (Cj > B) Cj = B;
        if (Cj < prev) Cj = prev;
      }
      Bj[j] = Cj - prev;
      prev = Cj;
    }
    for (uint32_t p = pb; p < pe; ++p) {
      double d[3];
      if (or_direction(c->seed, (uint32_t)c->step, (uint32_t)s, p, d) < 0)
      return fail(c, "direction sampling exceeded 64 attempts");
      for (int j = 0; j < nb; ++j) {
        int64_t base = Bj[j] / (int64_t)Ns, rmd = Bj[j] % (int64_t)Ns;
        N[j] = base + ((int64_t)p < rmd ? 1 : 0);
        emitted += N[j];
      }
      int64_t cr = or_trace_packet(c, &c->pos[3 * s], d, N, &escaped, &absorbed, 0, NULL, NULL, NULL);
      if (cr < 0) return -1;
      crossings += cr;
      ++traced;
    }
  }
  if (c->f_rec > 0) {
    /* diffuse recombination radiation (Sec. 2): every cell where the
     recombinations to the ground state of some species reach f_rec times
     that element's atoms in the cell re-emits them as one packet, and the
     species' count restarts from zero.  The photons of a species go to the
     lowest bin at or above its ionisation threshold (its Milne spectrum
     lies within a few kT of the threshold); in quanta q of this step. */
    const double V = (c->dl * c->dl) * c->dl;
    const double q = ldexp(1.0, E);
    int rec_bin[3];
    for (int a = 0; a < 3; ++a) {
      rec_bin[a] = -1;
      for (int j = 0; j < nb; ++j)
      if (c->binE[j] >= E_TH[a] && (rec_bin[a] < 0 || c->binE[j] < c->binE[rec_bin[a]]))
        rec_bin[a] = j;
    }
    for (int64_t i = 0; i < c->ncell; ++i) {
      const double atoms[3] = {c->nH[i] * V, c->nH[i] * c->he_over_h * V,
                             c->nH[i] * c->he_over_h * V};
      int64_t Nq[3] = {0, 0, 0};
      int any = 0;
      for (int a = 0; a < 3; ++a)
      if (atoms[a] > 0 && c->rec[a][i] > 0 && c->rec[a][i] >= c->f_rec * atoms[a]) {
        Nq[a] = llrint(c->rec[a][i] / q);
        c->rec[a][i] = 0.0;
        any = 1;
      }
      if (!any) continue;
      for (int j = 0; j < nb; ++j) N[j] = 0;
      int64_t tot = 0;
      for (int a = 0; a < 3; ++a)
      if (rec_bin[a] >= 0 && Nq[a] > 0) { N[rec_bin[a]] += Nq[a]; tot += Nq[a]; }
      if (tot == 0) continue;
      double pos[3], d[3];
      if (or_rec_start(c->seed, (uint32_t)c->step, i, c->nx, c->ny, pos, d) < 0)
      return fail(c, "direction sampling exceeded 64 attempts");
      emitted += tot;
      int64_t cr = or_trace_packet(c, pos, d, N, &escaped, &absorbed, 0, NULL, NULL, NULL);
      if (cr < 0) return -1;
      crossings += cr;
      ++traced;
    }
  }
  c->budget[0] = emitted; c->budget[1] = absorbed; c->budget[2] = escaped;
  c->budget[3] = crossings; c->budget[4] = traced;

  c->chem_pending = !c->chemistry;
  c->last_dt = dt;
  if (c->chemistry) or_step_chemistry(c, dt, E);
  c->step += 1;
  return 0;
}

int oracle_read_fields(or_ctx* c, int f, void* out) {
  if (!c || !out) return -1;
  size_t n = (size_t)c->ncell;
  switch (f) {
    case OR_F_XHII: memcpy(out, c->xHII, n * 8); return 0;
    case OR_F_XHEII: memcpy(out, c->xHeII, n * 8); return 0;
    case OR_F_XHEIII: memcpy(out, c->xHeIII, n * 8); return 0;
    case OR_F_T: memcpy(out, c->T, n * 8); return 0;
    case OR_F_DEP_HI: memcpy(out, c->dHI, n * 8); return 0;
    case OR_F_DEP_HEI: memcpy(out, c->dHeI, n * 8); return 0;
    case OR_F_DEP_HEII: memcpy(out, c->dHeII, n * 8); return 0;
    case OR_F_DEP_E: memcpy(out, c->dE, n * 8); return 0;
    case OR_F_BUDGET: memcpy(out, c->budget, sizeof c->budget); return 0;
    case OR_F_NH: memcpy(out, c->nH, n * 8); return 0;
    case OR_F_REC_HI: case OR_F_REC_HEI: case OR_F_REC_HEII:
      if (!c->rec[f - OR_F_REC_HI]) return fail(c, "the diffuse recombination field is off");
      memcpy(out, c->rec[f - OR_F_REC_HI], n * 8);
      return 0;
    default: return fail(c, "unknown field id");
  }
}

int oracle_write_fields(or_ctx* c, int f, const void* in) {
  if (!c || !in) return -1;
  size_t n = (size_t)c->ncell;
  switch (f) {
    case OR_F_XHII: memcpy(c->xHII, in, n * 8); return 0;
    case OR_F_XHEII: memcpy(c->xHeII, in, n * 8); return 0;
    case OR_F_XHEIII: memcpy(c->xHeIII, in, n * 8); return 0;
    case OR_F_T: memcpy(c->T, in, n * 8); return 0;
    case OR_F_REC_HI: case OR_F_REC_HEI: case OR_F_REC_HEII:
      if (!c->rec[f - OR_F_REC_HI]) return fail(c, "the diffuse recombination field is off");
      memcpy(c->rec[f - OR_F_REC_HI], in, n * 8);
      return 0;
    default: return fail(c, "field is not writable");
  }
}

/* The exchange of a step split over processes: overwrite the deposits
   (int64[cells][4]: H I, He I, He II, heat) with those summed over the
   processes, then run the per-cell update of the last step, which must have
   run without chemistry (same shapes as the library's crash_write_deposits
   and crash_chemistry). */
int oracle_write_deposits(or_ctx* c, const int64_t* in) {
  if (!c || !in) return -1;
  for (int64_t i = 0; i < c->ncell; ++i) {
    c->dHI[i] = in[4 * i]; c->dHeI[i] = in[4 * i + 1];
    c->dHeII[i] = in[4 * i + 2]; c->dE[i] = in[4 * i + 3];
  }
  return 0;
}

int oracle_chemistry(or_ctx* c, double dt) {
  if (!c) return -1;
  if (!c->chem_pending) return fail(c, "the last step ran its chemistry already");
  if (!(dt == c->last_dt)) return fail(c, "chemistry needs the dt of its step");
  or_step_chemistry(c, dt, (int)c->budget[5]);
  c->chem_pending = 0;
  return 0;
}
