/*
 * hff_oracle.c -- plain FP64 CPU oracle of the hybrid force-free / PIC time
 * step (Soudais, Cerutti & Contopoulos 2024).  TEST INFRASTRUCTURE ONLY: the
 * product path never includes, links or calls this file.
 *
 * Every function below is a direct, unblocked, unfused transcription of one
 * step of the scheme as the paper defines it (sections and equation numbers
 * cited next to each), plus the readings written down where the paper is
 * silent.  Loops are plain, geometry is recomputed from its exact-integral
 * definition at every use, and everything is double precision.
 *
 * Step order (Fig. 1 is not available; the order follows Sect. 3).  E and B
 * are both stored at integer times; B is advanced in two half steps.
 *   1. node pass A : psi^n (Eq. 27); collocated E^n, B^n; rho = div E / 4 pi;
 *                    J_perp (first term of Eq. 24)
 *   2. particles   : modified Boris push with radiation reaction (Eqs. 15-17),
 *                    u_perp removal near the star (Sect. 5.1), move,
 *                    charge-conserving deposit of J_PIC
 *   3. Faraday     : B^n -> B^{n+1/2}  (Eq. 18)
 *   4. Ampere      : E^n -> E^{n+1} with J = (1-f) J_PIC + f J_FFE (Eqs. 19, 28)
 *                    then the corotating star (Sect. 4) and the absorber
 *   5. correction  : node pass B renormalises the collocated E^{n+1} against
 *                    B^{n+1/2} (Eqs. 25-26); the mesh E moves to f <E''>
 *                    (default reading), or takes E += f <Delta E> (readings 1
 *                    and 2; reading 2 returns E'' on the stellar radial edges)
 *   6. Faraday     : B^{n+1/2} -> B^{n+1} from the corrected E, absorber on B
 *   7. injection   : top-up of the surface pair density (Sects. 4, 5.1),
 *                    then the pairs of the threshold pair creation (Sect. 5.1)
 *   8. sort        : stable sort by tile key with compaction, every k steps
 *
 * Parity pins for each part live in tests/test_oracle_*.py.  Parity unpinned:
 * the exact absorber profile (the paper only cites an earlier work for it);
 * its purpose is pinned (an outgoing pulse passes r_abs undamped, decays
 * monotonically in the layer and is not sent back).
 */
#include "hff_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define B2_MIN 1e-30

typedef struct {
  or_config c;
  int nr, nt;
  double dlog, dth, dt, omega, psi_unit, xi_abs;
  double *f[19]; /* fields, J, node arrays, initial B (see or_get_field) */
  int64_t cap, n[4];
  int32_t *cell[4];
  double *p[4][6]; /* xo yo ur ut up w */
  int32_t *surf, *target;
  int64_t step;
  double rr_k[4];
  double injected, killed, radiated, nonfinite, created, clamps;
  /* pair-creation events of the current step, in push order (species 0 by
   * particle index, then species 1): new cell, offsets, momentum, weight   */
  int64_t n_ev, cap_ev;
  int32_t *ev_cell;
  double *ev[6];
} ost;

/* ------------------------------------------------------------------ sizes */
static int64_t fsize(const ost *s, int which) {
  int64_t nr = s->nr, nt = s->nt;
  switch (which) {
  case 0: case 6: return nr * (nt + 1);          /* E_r, J_r  */
  case 1: case 7: return (nr + 1) * nt;          /* E_th, J_th */
  case 2: case 8: return (nr + 1) * (nt + 1);    /* E_ph, J_ph */
  case 3: case 16: return (nr + 1) * nt;         /* B_r */
  case 4: case 17: return nr * (nt + 1);         /* B_th */
  case 5: case 18: return nr * nt;               /* B_ph */
  default: return (nr + 1) * (nt + 1);           /* node scalars 9..15 */
  }
}

#define ER(i, j) s->f[0][(int64_t)(i) * (s->nt + 1) + (j)]
#define ET(i, j) s->f[1][(int64_t)(i) * s->nt + (j)]
#define EP(i, j) s->f[2][(int64_t)(i) * (s->nt + 1) + (j)]
#define BR(i, j) s->f[3][(int64_t)(i) * s->nt + (j)]
#define BT(i, j) s->f[4][(int64_t)(i) * (s->nt + 1) + (j)]
#define BP(i, j) s->f[5][(int64_t)(i) * s->nt + (j)]
#define JR(i, j) s->f[6][(int64_t)(i) * (s->nt + 1) + (j)]
#define JT(i, j) s->f[7][(int64_t)(i) * s->nt + (j)]
#define JP(i, j) s->f[8][(int64_t)(i) * (s->nt + 1) + (j)]
#define PSI(i, j) s->f[9][(int64_t)(i) * (s->nt + 1) + (j)]
#define NODE(k, i, j) s->f[(k)][(int64_t)(i) * (s->nt + 1) + (j)]
#define BR0(i, j) s->f[16][(int64_t)(i) * s->nt + (j)]
#define BT0(i, j) s->f[17][(int64_t)(i) * (s->nt + 1) + (j)]
#define BP0(i, j) s->f[18][(int64_t)(i) * s->nt + (j)]

/* --------------------------------------------------------------- geometry
 * Grid (Sect. 4): r_i = r_min exp(i D), D = ln(r_max/r_min)/nr; theta_j = j pi/nt.
 * Half nodes are geometric, r_{i+1/2} = r_min exp((i+1/2) D).  Every length,
 * area and volume is the exact integral over its edge, face or cell, which
 * makes div B = 0 and the charge-conservation / Gauss identity exact.      */
static double rn(const ost *s, int i) { return s->c.r_min * exp(i * s->dlog); }
static double rh(const ost *s, int i) { return s->c.r_min * exp((i + 0.5) * s->dlog); }
static double tn(const ost *s, int j) { return j * s->dth; }
static double th(const ost *s, int j) { return (j + 0.5) * s->dth; }
/* dual-cell bounds around node (i, j), clipped at r_min, r_max and the axis */
static double rlo(const ost *s, int i) { return i == 0 ? s->c.r_min : rh(s, i - 1); }
static double rhi(const ost *s, int i) { return i == s->nr ? s->c.r_max : rh(s, i); }
static double tlo(const ost *s, int j) { return j == 0 ? 0.0 : th(s, j - 1); }
static double thi(const ost *s, int j) { return j == s->nt ? PI : th(s, j); }
static double dch(const ost *s, int j) { return cos(tlo(s, j)) - cos(thi(s, j)); }
static double dcp(const ost *s, int j) { return cos(tn(s, j)) - cos(tn(s, j + 1)); }

/* primary faces (B locations) */
static double a_br(const ost *s, int i, int j) { return 2 * PI * rn(s, i) * rn(s, i) * dcp(s, j); }
static double a_bt(const ost *s, int i, int j) {
  return PI * sin(tn(s, j)) * (rn(s, i + 1) * rn(s, i + 1) - rn(s, i) * rn(s, i));
}
static double a_bp(const ost *s, int i) {
  return 0.5 * (rn(s, i + 1) * rn(s, i + 1) - rn(s, i) * rn(s, i)) * s->dth;
}
/* dual faces (E and J locations) and node dual volume */
static double a_er(const ost *s, int i, int j) { return 2 * PI * rh(s, i) * rh(s, i) * dch(s, j); }
static double a_et(const ost *s, int i, int j) {
  return PI * sin(th(s, j)) * (rhi(s, i) * rhi(s, i) - rlo(s, i) * rlo(s, i));
}
static double a_ep(const ost *s, int i, int j) {
  return 0.5 * (rhi(s, i) * rhi(s, i) - rlo(s, i) * rlo(s, i)) * (thi(s, j) - tlo(s, j));
}
static double vnode(const ost *s, int i, int j) {
  double a = rlo(s, i), b = rhi(s, i);
  return 2.0 * PI / 3.0 * (b * b * b - a * a * a) * dch(s, j);
}

/* --------------------------------------------------------- blend function
 * Eqs. 29-31, generalised to a piecewise-linear table (psi_k, f_k) so that the
 * two-layer dipole of Table 1 and the sharp monopole cut of Sect. 4 are both
 * expressible.  Below the first break f = f_0, above the last f = f_last; at a
 * jump (two equal breaks) the right-hand value applies.                     */
static double blend(const ost *s, double psi) {
  int n = s->c.n_breaks;
  if (n <= 0) return 0.0;
  const double *x = s->c.psi_break, *y = s->c.f_break;
  double u = s->psi_unit;
  if (psi < x[0] * u) return y[0];
  for (int k = 1; k < n; ++k) {
    double x0 = x[k - 1] * u, x1 = x[k] * u;
    if (psi < x1) return y[k - 1] + (y[k] - y[k - 1]) * (psi - x0) / (x1 - x0);
  }
  return y[n - 1];
}
double or_blend(void *st, double psi) { return blend((ost *)st, psi); }

/* ------------------------------------------------------- initial fields
 * Analytic flux functions: dipole Psi_D = mu sin^2(theta) / r (Eq. 37),
 * monopole Psi_M = Psi_star (1 - cos theta) (Eq. 32).  B is built from Psi by
 * differences over exact face areas, B = grad Psi x phi / (r sin theta).    */
static double psi_analytic(const ost *s, double r, double t) {
  double mu = s->c.b_star * pow(s->c.r_min, 3), pst = s->c.b_star * s->c.r_min * s->c.r_min;
  double sn = sin(t), cs = cos(t);
  switch (s->c.geom) {
  case OR_DIPOLE: return mu * sn * sn / r;
  case OR_MONOPOLE: case OR_MICHEL: return pst * (1.0 - cs);
  case OR_UNIFORM: return 0.5 * s->c.b_star * r * r * sn * sn;
  case OR_SYNTH: {
    /* dipole inside R_LC, split monopole outside (synthetic workload) */
    double w = 0.5 * (1.0 - tanh((r - s->c.r_lc) / (0.2 * s->c.r_lc)));
    double popen = s->c.synth_psi_open * s->psi_unit;
    return w * mu * sn * sn / r + (1.0 - w) * popen * (1.0 - fabs(cs));
  }
  }
  return 0.0;
}

static void init_fields(ost *s) {
  int nr = s->nr, nt = s->nt;
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j)
      BR(i, j) = (psi_analytic(s, rn(s, i), tn(s, j + 1)) - psi_analytic(s, rn(s, i), tn(s, j))) *
                 2 * PI / a_br(s, i, j);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      double a = a_bt(s, i, j);
      BT(i, j) = (j == 0 || j == nt)
                     ? 0.0
                     : -(psi_analytic(s, rn(s, i + 1), tn(s, j)) - psi_analytic(s, rn(s, i), tn(s, j))) *
                           2 * PI / a;
    }
  if (s->c.geom == OR_MICHEL) {
    /* Michel monopole, Eq. 33 and E_theta = B_phi (Sect. 4) */
    double pst = s->c.b_star * s->c.r_min * s->c.r_min;
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nt; ++j) BP(i, j) = -(pst / s->c.r_lc) * sin(th(s, j)) / rh(s, i);
    for (int i = 0; i <= nr; ++i)
      for (int j = 0; j < nt; ++j) ET(i, j) = -(pst / s->c.r_lc) * sin(th(s, j)) / rn(s, i);
  }
  memcpy(s->f[16], s->f[3], sizeof(double) * fsize(s, 3));
  memcpy(s->f[17], s->f[4], sizeof(double) * fsize(s, 4));
  memcpy(s->f[18], s->f[5], sizeof(double) * fsize(s, 5));
}

/* Corotating star (Sect. 4): the tangential field at r_star is the ideal
 * E = -(Omega x r) x B / c, i.e. E_theta = -Omega r sin(theta) B_r / c and
 * E_phi = 0; the normal E_r is left to Ampere's law.  The outer wall is a
 * conductor (tangential E = 0) hidden behind the absorber; E_phi = 0 on the
 * axis by symmetry.                                                          */
static void field_bc(ost *s) {
  int nr = s->nr, nt = s->nt;
  double r0 = rn(s, 0);
  for (int j = 0; j < nt; ++j) {
    ET(0, j) = -s->omega * r0 * sin(th(s, j)) * BR(0, j);
    ET(nr, j) = 0.0;
  }
  for (int j = 0; j <= nt; ++j) { EP(0, j) = 0.0; EP(nr, j) = 0.0; }
  for (int i = 0; i <= nr; ++i) { EP(i, 0) = 0.0; EP(i, nt) = 0.0; }
}

/* Absorbing layer (Sect. 4 gives only its start, r_abs = 3 R_LC, and its
 * purpose).  Reading: damping coefficient sigma(r) = sigma_0 x^3 with
 * x = (r - r_abs)/(r_max - r_abs); E -> (1 - sigma) E, B -> B - sigma (B - B_0). */
static double sigma_abs(const ost *s, double r) {
  if (r <= s->c.r_abs) return 0.0;
  double x = (r - s->c.r_abs) / (s->c.r_max - s->c.r_abs);
  return s->c.absorb_strength * x * x * x;
}

/* ----------------------------------------------------------- Philox4x32-10
 * Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11), written
 * from its published definition: 10 rounds of two 32x32->64 multiplies with
 * a Weyl-sequence key schedule.                                             */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------ create */
/* Courant: dt = C min_i [1/sqrt(1/dr_i^2 + 1/(r_i dtheta)^2)] / c.  C = 0.5
 * agrees with Table 1 (c dt = 129 cm against a 255 cm 2D limit at r_star). */
double or_config_dt(const or_config *cfg) {
  double dlog = log(cfg->r_max / cfg->r_min) / cfg->nr, dth = PI / cfg->nt, best = 1e300;
  for (int i = 0; i < cfg->nr; ++i) {
    double r0 = cfg->r_min * exp(i * dlog), r1 = cfg->r_min * exp((i + 1) * dlog);
    double dr = r1 - r0, rt = r0 * dth;
    double l = 1.0 / sqrt(1.0 / (dr * dr) + 1.0 / (rt * rt));
    if (l < best) best = l;
  }
  return cfg->courant * best;
}

static int64_t ncells_theta_tiles(const ost *s) { return (s->nt + s->c.tile_t - 1) / s->c.tile_t; }

void *or_create(const or_config *cfg) {
  if (cfg->nr < 4 || cfg->nt < 4 || cfg->n_species < 1 || cfg->n_species > 4) return NULL;
  ost *s = (ost *)calloc(1, sizeof(ost));
  s->c = *cfg;
  if (s->c.tile_r <= 0) s->c.tile_r = 16;
  if (s->c.tile_t <= 0) s->c.tile_t = 16;
  s->nr = cfg->nr;
  s->nt = cfg->nt;
  s->dlog = log(cfg->r_max / cfg->r_min) / cfg->nr;
  s->dth = PI / cfg->nt;
  s->omega = 1.0 / cfg->r_lc; /* Omega = c / R_LC (Eq. 1) */
  s->xi_abs = log(cfg->r_abs / cfg->r_min) / s->dlog;
  /* psi unit: Psi_pc = mu / R_LC for dipolar fields (Sect. 5.1),
   * Psi_star = B_star r_star^2 for the monopole (Sect. 4).                   */
  if (cfg->geom == OR_MONOPOLE || cfg->geom == OR_MICHEL)
    s->psi_unit = cfg->b_star * cfg->r_min * cfg->r_min;
  else
    s->psi_unit = cfg->b_star * pow(cfg->r_min, 3) / cfg->r_lc;
  s->dt = or_config_dt(cfg);
  for (int k = 0; k < 19; ++k) s->f[k] = (double *)calloc(fsize(s, k), sizeof(double));
  s->cap = cfg->capacity;
  for (int sp = 0; sp < cfg->n_species; ++sp) {
    s->cell[sp] = (int32_t *)calloc(s->cap > 0 ? s->cap : 1, sizeof(int32_t));
    for (int k = 0; k < 6; ++k) s->p[sp][k] = (double *)calloc(s->cap > 0 ? s->cap : 1, sizeof(double));
  }
  /* Radiation-reaction coefficient per species.  Eq. 16 is a force; it enters
   * du/dt as g / (m c).  Its strength is fixed by gamma_rad: for species 0 the
   * drag (2/3) r_e^2 gamma^2 B^2 balances |q| E at E = B_perp = b_ref
   * (Sect. 2), so (2/3) r_0^2 = |q_0| / (gamma_rad^2 b_ref); other species
   * scale with their classical radius r_s = q_s^2 / m_s.                     */
  for (int sp = 0; sp < cfg->n_species; ++sp) {
    if (cfg->gamma_rad <= 0) { s->rr_k[sp] = 0; continue; }
    double r0c = cfg->q[0] * cfg->q[0] / cfg->m[0], rsc = cfg->q[sp] * cfg->q[sp] / cfg->m[sp];
    double two3_r0sq = fabs(cfg->q[0]) / (cfg->gamma_rad * cfg->gamma_rad * cfg->b_ref);
    s->rr_k[sp] = two3_r0sq * (rsc / r0c) * (rsc / r0c) / cfg->m[sp];
  }
  init_fields(s);
  field_bc(s);
  /* Injection targets per surface cell (Sects. 4 and 5.1).  The surface
   * decomposition is frozen at the star (Sect. 3), so eligibility f < 1 and
   * the target kappa n_GJ V / w (n_GJ = Omega |B_r| / (2 pi e c), Sect. 2) are
   * fixed once.                                                               */
  s->surf = (int32_t *)calloc(s->nt, sizeof(int32_t));
  s->target = (int32_t *)calloc(s->nt, sizeof(int32_t));
  s->cap_ev = s->cap > 0 ? s->cap : 1;
  s->ev_cell = (int32_t *)calloc(s->cap_ev, sizeof(int32_t));
  for (int k = 0; k < 6; ++k) s->ev[k] = (double *)calloc(s->cap_ev, sizeof(double));
  {
    double pacc = 0.0, r0 = rn(s, 0);
    for (int j = 0; j < s->nt; ++j) {
      double p0 = pacc;
      pacc += BR(0, j) * r0 * r0 * dcp(s, j);
      double fs = blend(s, 0.5 * (p0 + pacc));
      int32_t tgt = 0;
      if (cfg->inject == OR_INJ_ON && fs < 1.0 && cfg->w_inj > 0) {
        double ngj = s->omega * fabs(BR(0, j)) / (2 * PI * fabs(cfg->q[0]));
        double r1 = rn(s, 1);
        double v = 2.0 * PI / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0) * dcp(s, j);
        tgt = (int32_t)floor(cfg->kappa_inj * ngj * v / cfg->w_inj + 0.5);
      }
      s->target[j] = tgt;
    }
  }
  return s;
}

void or_destroy(void *st) {
  ost *s = (ost *)st;
  if (!s) return;
  for (int k = 0; k < 19; ++k) free(s->f[k]);
  for (int sp = 0; sp < s->c.n_species; ++sp) {
    free(s->cell[sp]);
    for (int k = 0; k < 6; ++k) free(s->p[sp][k]);
  }
  free(s->surf);
  free(s->target);
  free(s->ev_cell);
  for (int k = 0; k < 6; ++k) free(s->ev[k]);
  free(s);
}

double or_dt(void *st) { return ((ost *)st)->dt; }
double or_psi_unit(void *st) { return ((ost *)st)->psi_unit; }
int64_t or_step_index(void *st) { return ((ost *)st)->step; }
/* Sets the step counter (the injection generator's key and the sort cadence);
 * a caller that splits one step into several stage groups uses it so that the
 * step counts once (tests only). */
void or_set_step_index(void *st, int64_t step) { ((ost *)st)->step = step; }
int64_t or_field_size(void *st, int which) { return fsize((ost *)st, which); }
int or_get_field(void *st, int which, double *out) {
  ost *s = (ost *)st;
  if (which < 0 || which > 18) return -1;
  memcpy(out, s->f[which], sizeof(double) * fsize(s, which));
  return 0;
}
int or_set_field(void *st, int which, const double *in) {
  ost *s = (ost *)st;
  if (which < 0 || which > 18) return -1;
  memcpy(s->f[which], in, sizeof(double) * fsize(s, which));
  return 0;
}
int64_t or_count(void *st, int sp) { return ((ost *)st)->n[sp]; }
int or_set_particles(void *st, int sp, int64_t n, const int32_t *cell, const double *xo,
                     const double *yo, const double *ur, const double *ut, const double *up,
                     const double *w) {
  ost *s = (ost *)st;
  if (sp < 0 || sp >= s->c.n_species || n > s->cap) return -1;
  const double *src[6] = {xo, yo, ur, ut, up, w};
  memcpy(s->cell[sp], cell, sizeof(int32_t) * n);
  for (int k = 0; k < 6; ++k) memcpy(s->p[sp][k], src[k], sizeof(double) * n);
  s->n[sp] = n;
  return 0;
}
int or_get_particles(void *st, int sp, int32_t *cell, double *xo, double *yo, double *ur,
                     double *ut, double *up, double *w) {
  ost *s = (ost *)st;
  if (sp < 0 || sp >= s->c.n_species) return -1;
  double *dst[6] = {xo, yo, ur, ut, up, w};
  memcpy(cell, s->cell[sp], sizeof(int32_t) * s->n[sp]);
  for (int k = 0; k < 6; ++k) memcpy(dst[k], s->p[sp][k], sizeof(double) * s->n[sp]);
  return 0;
}
int32_t or_surface_count(void *st, int j) { return ((ost *)st)->surf[j]; }
void or_set_surface_count(void *st, int j, int32_t v) { ((ost *)st)->surf[j] = v; }
int32_t or_inject_target(void *st, int j) { return ((ost *)st)->target[j]; }
void or_set_rr_scale(void *st, double v) { ((ost *)st)->c.rr_scale = v; }

/* ------------------------------------------------------- collocation
 * Force-free quantities are collocated at the nodes by arithmetic means of the
 * neighbouring staggered values (Sect. 3); on the axis the transverse
 * components vanish by symmetry.  Interior rows 1 .. nr-1 only.             */
static void collocate(const ost *s, int i, int j, double e[3], double b[3]) {
  int nt = s->nt, axis = (j == 0 || j == nt);
  e[0] = 0.5 * (ER(i - 1, j) + ER(i, j));
  e[1] = axis ? 0.0 : 0.5 * (ET(i, j - 1) + ET(i, j));
  e[2] = axis ? 0.0 : EP(i, j);
  b[0] = (j == 0) ? BR(i, 0) : (j == nt) ? BR(i, nt - 1) : 0.5 * (BR(i, j - 1) + BR(i, j));
  b[1] = axis ? 0.0 : 0.5 * (BT(i - 1, j) + BT(i, j));
  b[2] = axis ? 0.0 : 0.25 * (BP(i - 1, j - 1) + BP(i - 1, j) + BP(i, j - 1) + BP(i, j));
}

/* ---------------------------------------------------------------- 1. node pass A
 * Psi (Eq. 27) as a theta-prefix of the radial flux: Psi(i,0) = 0 and
 * Psi(i,j+1) = Psi(i,j) + B_r(i,j+1/2) r_i^2 (cos theta_j - cos theta_{j+1}).
 * At each interior node, from the collocated E^n and B^n:
 *   rho = div E / 4 pi  (finite volume over the node's dual cell)
 *   J_perp = c rho (E x B) / B^2             (first term of Eq. 24)       */
static void node_pass_a(ost *s) {
  int nr = s->nr, nt = s->nt;
  for (int i = 0; i <= nr; ++i) {
    double acc = 0.0, r2 = rn(s, i) * rn(s, i);
    PSI(i, 0) = 0.0;
    for (int j = 0; j < nt; ++j) {
      acc += BR(i, j) * r2 * dcp(s, j);
      PSI(i, j + 1) = acc;
    }
  }
  for (int k = 10; k <= 12; ++k) memset(s->f[k], 0, sizeof(double) * fsize(s, k));
  for (int i = 1; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      double e[3], b[3];
      collocate(s, i, j, e, b);
      double flux = ER(i, j) * a_er(s, i, j) - ER(i - 1, j) * a_er(s, i - 1, j);
      if (j < nt) flux += ET(i, j) * a_et(s, i, j);
      if (j > 0) flux -= ET(i, j - 1) * a_et(s, i, j - 1);
      double rho = flux / (4 * PI * vnode(s, i, j));
      double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
      if (!(b2 > B2_MIN)) continue;
      double exb[3] = {e[1] * b[2] - e[2] * b[1], e[2] * b[0] - e[0] * b[2], e[0] * b[1] - e[1] * b[0]};
      for (int k = 0; k < 3; ++k) NODE(10 + k, i, j) = rho * exb[k] / b2; /* c = 1 */
    }
}

/* ---------------------------------------------------------------- node pass B
 * Renormalisation of E at the nodes (Sect. 3), from the collocated E^{n+1}
 * and the latest B (B^{n+1/2}):
 *   E' = E - (E.B) B / B^2                   (Eq. 25)
 *   E'' = sqrt(B^2/E'^2) E' if E'^2 > B^2     (Eq. 26)
 *   Delta E = E'' - E.                                                      */
static void node_pass_b(ost *s) {
  int nr = s->nr, nt = s->nt;
  for (int k = 13; k <= 15; ++k) memset(s->f[k], 0, sizeof(double) * fsize(s, k));
  for (int i = 1; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      double e[3], b[3];
      collocate(s, i, j, e, b);
      double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
      if (!(b2 > B2_MIN)) continue;
      double edb = e[0] * b[0] + e[1] * b[1] + e[2] * b[2];
      double ep[3], ep2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        ep[k] = e[k] - edb * b[k] / b2;
        ep2 += ep[k] * ep[k];
      }
      double sc = (ep2 > b2) ? sqrt(b2 / ep2) : 1.0;
      if (ep2 > b2) s->clamps += 1; /* Eq. 26 applied at this node */
      for (int k = 0; k < 3; ++k) NODE(13 + k, i, j) = sc * ep[k] - e[k];
    }
  /* reading "interpolate these back" literally: the corrected node field
   * E'' = E + Delta E itself returns to the edges                         */
  if (!s->c.ff_delta_only)
    for (int i = 1; i < nr; ++i)
      for (int j = 0; j <= nt; ++j) {
        double e[3], b[3];
        collocate(s, i, j, e, b);
        for (int k = 0; k < 3; ++k) NODE(13 + k, i, j) += e[k];
      }
}

/* Mean of a node quantity over the two nodes of a radial edge, using only
 * interior nodes (rows 0 and nr carry the boundary conditions). */
static double edge_r_mean(const ost *s, int k, int i, int j) {
  int lo = (i >= 1), hi = (i + 1 <= s->nr - 1);
  double v = 0.0;
  if (lo) v += NODE(k, i, j);
  if (hi) v += NODE(k, i + 1, j);
  return (lo && hi) ? 0.5 * v : v;
}

/* ---------------------------------------------------------- 5. correction
 * Delta E (node pass B) is interpolated back onto the staggered mesh by
 * arithmetic means (Sect. 3) and applied with the blend weight f(Psi^n) of
 * Eqs. 29-31: full in the force-free domain, absent in pure PIC, linear
 * across the layer.  Psi on an edge is the mean of its nodes.               */
/* Fourth differences of E_r along r and of E_th along theta at the edges
 * (zero where the five-point stencil does not fit), from the field as it is
 * before the correction.  The two-point means of the collocation (Sect. 3)
 * do not see the odd-even component of E_r along r or of E_th along theta,
 * so the node corrections cannot act on it; the filter E -= f sigma/16 D4 E
 * (reading, optional) removes that component (sigma = 1) and changes a
 * smooth field by O(h^4) per step.                                          */
static double d4_er(const ost *s, int i, int j) {
  if (i < 2 || i > s->nr - 3) return 0.0;
  return ER(i - 2, j) - 4 * ER(i - 1, j) + 6 * ER(i, j) - 4 * ER(i + 1, j) + ER(i + 2, j);
}
static double d4_et(const ost *s, int i, int j) {
  if (j < 2 || j > s->nt - 3) return 0.0;
  return ET(i, j - 2) - 4 * ET(i, j - 1) + 6 * ET(i, j) - 4 * ET(i, j + 1) + ET(i, j + 2);
}

static void correct_e(ost *s) {
  int nr = s->nr, nt = s->nt, lit = s->c.ff_delta_only == 0;
  double sg = s->c.ff_filter / 16.0;
  double *fr = NULL, *ft = NULL;
  if (sg != 0.0) { /* the filter terms from the uncorrected E */
    fr = (double *)calloc(fsize(s, 0), sizeof(double));
    ft = (double *)calloc(fsize(s, 1), sizeof(double));
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j <= nt; ++j) fr[(int64_t)i * (nt + 1) + j] = sg * d4_er(s, i, j);
    for (int i = 1; i < nr; ++i)
      for (int j = 0; j < nt; ++j) ft[(int64_t)i * nt + j] = sg * d4_et(s, i, j);
  }
  node_pass_b(s);
  /* with the literal reading the edge value moves toward the mean of the
   * corrected node fields, E <- E + f (<E''> - E); otherwise E += f <dE>;
   * the optional filter term is subtracted with the same weight f.
   * Reading 2 returns the corrections alone except on the radial edges that
   * end on the star (i = 0): their one interior node is node row 1, and
   * there the corrected node field itself returns, E_r <- E_r + f (E''(1) -
   * E_r), with E''(1) = Delta E(1) + the collocated E of row 1.  Row 0 is
   * processed first, so that collocated E is still the uncorrected one.    */
  int star_lit = s->c.ff_delta_only == 2;
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      double f = blend(s, 0.5 * (PSI(i, j) + PSI(i + 1, j)));
      double m = edge_r_mean(s, 13, i, j);
      if (fr) m -= fr[(int64_t)i * (nt + 1) + j];
      int star = star_lit && i == 0 && nr > 1;
      if (star) m += 0.5 * (ER(0, j) + ER(1, j));
      int l = lit || star;
      if (f != 0.0) ER(i, j) += f * (l ? m - ER(i, j) : m);
    }
  for (int i = 1; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double f = blend(s, 0.5 * (PSI(i, j) + PSI(i, j + 1)));
      double m = 0.5 * (NODE(14, i, j) + NODE(14, i, j + 1));
      if (ft) m -= ft[(int64_t)i * nt + j];
      if (f != 0.0) ET(i, j) += f * (lit ? m - ET(i, j) : m);
    }
  free(fr);
  free(ft);
  for (int i = 1; i < nr; ++i)
    for (int j = 1; j < nt; ++j) {
      double f = blend(s, PSI(i, j));
      double m = NODE(15, i, j);
      if (f != 0.0) EP(i, j) += f * (lit ? m - EP(i, j) : m);
    }
}

/* ----------------------------------------------------------------- 3. push */
static void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Modified Boris pusher (Sect. 3, Eqs. 15-17), code units c = 1:
 *   du/dt = (q/m)(E + u x B / gamma) + K F_RR,
 *   F_RR  = (E + beta x B) x B + (beta.E) E - gamma^2 Bperp^2 beta,
 *   Bperp^2 = (E + beta x B)^2 - (beta.E)^2                      (Eq. 17)
 * Reading of "modified": a textbook Boris step for the Lorentz force gives
 * u_L; the radiation-reaction kick is then evaluated at the time-centred
 * momentum (u^{n-1/2} + u_L)/2 and added explicitly.                        */
void or_push_local(double qm, double krr, double dt, const double u[3], const double e[3],
                   const double b[3], double out[3], double *radiated_dgamma) {
  double a = 0.5 * qm * dt, um[3], t[3], sv[3], up[3], tmp[3], ul[3];
  for (int k = 0; k < 3; ++k) um[k] = u[k] + a * e[k];
  double gm = sqrt(1.0 + dot(um, um));
  for (int k = 0; k < 3; ++k) t[k] = a * b[k] / gm;
  double t2 = dot(t, t);
  for (int k = 0; k < 3; ++k) sv[k] = 2.0 * t[k] / (1.0 + t2);
  cross(um, t, tmp);
  for (int k = 0; k < 3; ++k) up[k] = um[k] + tmp[k];
  cross(up, sv, tmp);
  for (int k = 0; k < 3; ++k) ul[k] = um[k] + tmp[k] + a * e[k];
  if (krr != 0.0) {
    double ub[3], beta[3], epb[3], bxb[3], f[3];
    for (int k = 0; k < 3; ++k) ub[k] = 0.5 * (u[k] + ul[k]);
    double gb = sqrt(1.0 + dot(ub, ub));
    for (int k = 0; k < 3; ++k) beta[k] = ub[k] / gb;
    cross(beta, b, bxb);
    for (int k = 0; k < 3; ++k) epb[k] = e[k] + bxb[k];
    double be = dot(beta, e);
    double bp2 = dot(epb, epb) - be * be;
    if (bp2 < 0.0) bp2 = 0.0;
    cross(epb, b, f);
    double du[3];
    for (int k = 0; k < 3; ++k) du[k] = dt * krr * (f[k] + be * e[k] - gb * gb * bp2 * beta[k]);
    /* Reading: the explicit kick may remove at most half of |u_L| in one
     * step.  This is a no-op whenever the cooling time exceeds ~2 dt (Table 1
     * quotes t_syn ~ 85 dt) and keeps unresolved cooling from reversing u.   */
    double dn2 = dot(du, du), ul2 = dot(ul, ul);
    double lim = (dn2 > 0.25 * ul2) ? 0.5 * sqrt(ul2 / dn2) : 1.0;
    for (int k = 0; k < 3; ++k) out[k] = ul[k] + lim * du[k];
  } else {
    for (int k = 0; k < 3; ++k) out[k] = ul[k];
  }
  if (radiated_dgamma) *radiated_dgamma = sqrt(1.0 + dot(ul, ul)) - sqrt(1.0 + dot(out, out));
}

/* Move (the paper is silent on the particle mover of its spherical code).
 * Reading: the particle moves on a straight line x' = x + (u/gamma) c dt in
 * the local Cartesian frame (r_hat, theta_hat, phi_hat) at azimuth 0; the
 * azimuthal part of the motion is then rotated away (axisymmetry), and u is
 * re-expressed in the local basis of the new point.  All increments are
 * formed without subtracting large absolute radii.                          */
void or_move_local(double r, double t, double dt, const double u[3], double *dr, double *dth,
                   double *dphi, double uo[3]) {
  double g = sqrt(1.0 + dot(u, u));
  double d0 = u[0] * dt / g, d1 = u[1] * dt / g, d2 = u[2] * dt / g;
  double sn = sin(t), cs = cos(t);
  double x = (r + d0) * sn + d1 * cs;             /* cylindrical radius before phi motion */
  double rc = sqrt(x * x + d2 * d2);
  double dR = (x > 0.0) ? d2 * d2 / (rc + x) : rc - x; /* growth of cylindrical radius */
  double pa = d0 + dR * sn;                      /* new point in the old (r, theta) plane */
  double a = r + pa, b = d1 + dR * cs;
  double rnew = sqrt(a * a + b * b);
  *dr = (pa * (2.0 * r + pa) + b * b) / (rnew + r);
  double al = atan2(b, a);
  double ph = atan2(d2, x);
  *dth = al;
  *dphi = ph;
  double uR = u[0] * sn + u[1] * cs;
  double sp = sin(ph), h = sin(0.5 * ph);
  double duR = uR * (-2.0 * h * h) + u[2] * sp;
  double t1 = t + al, s1 = sin(t1), c1 = cos(t1), ca = cos(al), sa = sin(al);
  uo[0] = u[0] * ca + u[1] * sa + duR * s1;
  uo[1] = -u[0] * sa + u[1] * ca + duR * c1;
  uo[2] = -uR * sp + u[2] * cos(ph);
}

/* 1D linear-weight index for a staggered component: positions k + a with
 * a in {0, 1/2}, k = 0 .. n-1; constant extrapolation beyond the ends.      */
static void stag(int c, double o, int half, int n, int *k0, double *w) {
  if (!half) { *k0 = c; *w = o; }
  else if (o >= 0.5) { *k0 = c; *w = o - 0.5; }
  else { *k0 = c - 1; *w = o + 0.5; }
  if (*k0 < 0) { *k0 = 0; *w = 0.0; }
  if (*k0 > n - 2) { *k0 = n - 2; *w = 1.0; }
}

static double interp(const double *a, int ld, int i0, double wx, int j0, double wy) {
  return (1 - wx) * (1 - wy) * a[(int64_t)i0 * ld + j0] + wx * (1 - wy) * a[(int64_t)(i0 + 1) * ld + j0] +
         (1 - wx) * wy * a[(int64_t)i0 * ld + j0 + 1] + wx * wy * a[(int64_t)(i0 + 1) * ld + j0 + 1];
}

/* Linear (cloud-in-cell) gather in logical coordinates from the staggered
 * mesh; returns E and B in the local spherical basis at the particle.       */
static void gather(const ost *s, int i, int j, double xo, double yo, double e[3], double b[3]) {
  int nr = s->nr, nt = s->nt, ki, kj;
  double wi, wj;
  stag(i, xo, 1, nr, &ki, &wi); stag(j, yo, 0, nt + 1, &kj, &wj); e[0] = interp(s->f[0], nt + 1, ki, wi, kj, wj);
  stag(i, xo, 0, nr + 1, &ki, &wi); stag(j, yo, 1, nt, &kj, &wj); e[1] = interp(s->f[1], nt, ki, wi, kj, wj);
  stag(i, xo, 0, nr + 1, &ki, &wi); stag(j, yo, 0, nt + 1, &kj, &wj); e[2] = interp(s->f[2], nt + 1, ki, wi, kj, wj);
  stag(i, xo, 0, nr + 1, &ki, &wi); stag(j, yo, 1, nt, &kj, &wj); b[0] = interp(s->f[3], nt, ki, wi, kj, wj);
  stag(i, xo, 1, nr, &ki, &wi); stag(j, yo, 0, nt + 1, &kj, &wj); b[1] = interp(s->f[4], nt + 1, ki, wi, kj, wj);
  stag(i, xo, 1, nr, &ki, &wi); stag(j, yo, 1, nt, &kj, &wj); b[2] = interp(s->f[5], nt, ki, wi, kj, wj);
}

/* Linear shape on the 4 nodes c-1 .. c+2 around a start cell c, for a point
 * at x relative to node c (x in (-1, 2)). */
static void shape4(double x, double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  int k = (int)floor(x);
  double fr = x - k;
  out[k + 1] = 1.0 - fr;
  out[k + 2] = fr;
}

/* Charge-conserving deposit (Esirkepov's decomposition for linear shapes in
 * the logical (xi, eta) plane).  The charge crossing each dual face during
 * the step, divided by the exact face area and dt, is J_r or J_theta; the
 * azimuthal current uses the mid-point weights over the node dual volume.
 * With Ampere's update over the same dual faces this makes
 * div E - 4 pi rho invariant (Gauss's law, Eq. 19 and the continuity
 * equation).                                                                */
static void deposit(ost *s, double qw, int i0, int j0, double x0, double y0, double x1, double y1,
                    double vphi) {
  int nr = s->nr, nt = s->nt;
  double s0x[4], s1x[4], s0y[4], s1y[4], dsx[4], dsy[4];
  shape4(x0, s0x); shape4(x1, s1x); shape4(y0, s0y); shape4(y1, s1y);
  for (int k = 0; k < 4; ++k) { dsx[k] = s1x[k] - s0x[k]; dsy[k] = s1y[k] - s0y[k]; }
  for (int b = 0; b < 4; ++b) {
    int jj = j0 - 1 + b;
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) {
      acc += dsx[a] * 0.5 * (s0y[b] + s1y[b]);
      double fx = -qw * acc;
      int ii = i0 - 1 + a;
      if (fx != 0.0 && ii >= 0 && ii < nr && jj >= 0 && jj <= nt) JR(ii, jj) += fx / (a_er(s, ii, jj) * s->dt);
    }
  }
  for (int a = 0; a < 4; ++a) {
    int ii = i0 - 1 + a;
    double acc = 0.0;
    for (int b = 0; b < 3; ++b) {
      acc += dsy[b] * 0.5 * (s0x[a] + s1x[a]);
      double fy = -qw * acc;
      int jj = j0 - 1 + b;
      if (fy != 0.0 && ii >= 0 && ii <= nr && jj >= 0 && jj < nt) JT(ii, jj) += fy / (a_et(s, ii, jj) * s->dt);
    }
  }
  double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1);
  int km = (int)floor(xm), lm = (int)floor(ym);
  double wx = xm - km, wy = ym - lm;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int ii = i0 + km + a, jj = j0 + lm + b;
      double wgt = (a ? wx : 1 - wx) * (b ? wy : 1 - wy);
      if (wgt != 0.0 && ii >= 0 && ii <= nr && jj >= 0 && jj <= nt) JP(ii, jj) += qw * vphi * wgt / vnode(s, ii, jj);
    }
}

/* The gather at one position and one deposit into J_PIC, exactly as the
 * push calls them; exported for the pins of the interpolation and of the
 * azimuthal current (tests only).                                           */
void or_gather(void *st, int32_t i, int32_t j, double xo, double yo, double e[3], double b[3]) {
  gather((const ost *)st, i, j, xo, yo, e, b);
}
void or_deposit(void *st, double qw, int32_t i0, int32_t j0, double x0, double y0, double x1,
                double y1, double vphi) {
  deposit((ost *)st, qw, i0, j0, x0, y0, x1, y1, vphi);
}

static double cell_psi(const ost *s, int i, int j) {
  return 0.25 * (PSI(i, j) + PSI(i + 1, j) + PSI(i, j + 1) + PSI(i + 1, j + 1));
}

static void push_all(ost *s) {
  int nr = s->nr, nt = s->nt;
  (void)nr;
  memset(s->surf, 0, sizeof(int32_t) * nt);
  s->n_ev = 0;
  double dt = s->dt;
  for (int sp = 0; sp < s->c.n_species; ++sp) {
    double qm = s->c.q[sp] / s->c.m[sp], krr = s->rr_k[sp] * s->c.rr_scale;
    int32_t *cell = s->cell[sp];
    double *xo = s->p[sp][0], *yo = s->p[sp][1], *ur = s->p[sp][2], *ut = s->p[sp][3], *up = s->p[sp][4],
           *w = s->p[sp][5];
    for (int64_t p = 0; p < s->n[sp]; ++p) {
      if (cell[p] < 0) continue;
      int i = cell[p] / nt, j = cell[p] % nt;
      double r = s->c.r_min * exp((i + xo[p]) * s->dlog), t = (j + yo[p]) * s->dth;
      double e[3], b[3], u[3] = {ur[p], ut[p], up[p]}, un[3], rad;
      gather(s, i, j, xo[p], yo[p], e, b);
      or_push_local(qm, krr, dt, u, e, b, un, &rad);
      s->radiated += w[p] * s->c.m[sp] * rad;
      /* Sect. 5.1: momentum transverse to B is removed in an r_star-thick
       * shell above the surface. */
      if (r < s->c.shell_r) {
        double b2 = dot(b, b);
        if (b2 > B2_MIN) {
          double ub = dot(un, b) / b2;
          for (int k = 0; k < 3; ++k) un[k] = ub * b[k];
        }
      }
      double g = sqrt(1.0 + dot(un, un));
      double dr, dth, dph, uo[3];
      or_move_local(r, t, dt, un, &dr, &dth, &dph, uo);
      double dxi = log1p(dr / r) / s->dlog, deta = dth / s->dth;
      /* new logical position relative to the start cell */
      double X1 = xo[p] + dxi, Y1 = yo[p] + deta;
      if (!isfinite(X1) || !isfinite(Y1) || !isfinite(uo[0] + uo[1] + uo[2])) {
        /* a non-finite state is removed without depositing */
        cell[p] = -1;
        s->nonfinite += 1;
        continue;
      }
      /* reflection at the axis (only reached through rounding) */
      if (j + Y1 < 0.0) Y1 = -2.0 * j - Y1;
      if (j + Y1 > nt) Y1 = 2.0 * (nt - j) - Y1;
      int dead = 0;
      if (i + X1 < 0.0) { X1 = -(double)i; dead = 1; }        /* absorbed by the star */
      else if (i + X1 > s->xi_abs) dead = 1;                    /* absorbing layer */
      int di = (int)floor(X1), dj = (int)floor(Y1);
      double xn = X1 - di, yn = Y1 - dj;
      if (xn >= 1.0) { xn -= 1.0; di += 1; }
      if (yn >= 1.0) { yn -= 1.0; dj += 1; }
      int i1 = i + di, j1 = j + dj;
      if (j1 >= nt) { j1 = nt - 1; yn = nextafter(1.0, 0.0); }
      if (!dead && blend(s, cell_psi(s, i1, j1)) >= 1.0) dead = 1; /* force-free cell: no particles */
      deposit(s, s->c.q[sp] * w[p], i, j, xo[p], yo[p], X1, Y1, un[2] / g);
      if (dead) {
        cell[p] = -1;
        s->killed += w[p];
        continue;
      }
      cell[p] = i1 * nt + j1;
      xo[p] = xn; yo[p] = yn;
      ur[p] = uo[0]; ut[p] = uo[1]; up[p] = uo[2];
      if (i1 == 0) s->surf[j1] += 1;
      /* Sect. 5.1: a lepton above the threshold Lorentz factor creates a pair
       * at its position, moving along its direction with gamma_s; the parent
       * is left as it is (reading), at most one pair per parent and step.    */
      if (s->c.gamma_th > 0 && sp < 2 && 1.0 + dot(uo, uo) > s->c.gamma_th * s->c.gamma_th) {
        if (s->n_ev >= s->cap_ev) { fprintf(stderr, "oracle: pair event capacity exceeded\n"); abort(); }
        double a = sqrt(s->c.gamma_s * s->c.gamma_s - 1.0) / sqrt(dot(uo, uo));
        int64_t e = s->n_ev++;
        s->ev_cell[e] = cell[p];
        s->ev[0][e] = xn; s->ev[1][e] = yn;
        s->ev[2][e] = a * uo[0]; s->ev[3][e] = a * uo[1]; s->ev[4][e] = a * uo[2];
        s->ev[5][e] = w[p];
      }
    }
  }
}

/* The pairs of this step's creation events, appended to species 0 (e-) and
 * 1 (e+) in event order after the injected ones.                           */
static void create_pairs(ost *s) {
  if (s->c.n_species < 2) { s->n_ev = 0; return; }
  for (int64_t e = 0; e < s->n_ev; ++e)
    for (int sp = 0; sp < 2; ++sp) {
      if (s->n[sp] >= s->cap) { fprintf(stderr, "oracle: particle capacity exceeded\n"); abort(); }
      int64_t p = s->n[sp]++;
      s->cell[sp][p] = s->ev_cell[e];
      for (int k = 0; k < 6; ++k) s->p[sp][k][p] = s->ev[k][e];
      s->created += s->ev[5][e];
    }
  s->n_ev = 0;
}

/* ----------------------------------------------------------- 4/6. Faraday
 * Eq. 18 in Stokes form over the exact primary faces; h = fraction of dt.   */
static void faraday(ost *s, double h) {
  int nr = s->nr, nt = s->nt;
  double k = h * s->dt; /* c = 1 */
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double circ = 2 * PI * rn(s, i) * (sin(tn(s, j + 1)) * EP(i, j + 1) - sin(tn(s, j)) * EP(i, j));
      BR(i, j) -= k * circ / a_br(s, i, j);
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      if (j == 0 || j == nt) { BT(i, j) = 0.0; continue; }
      double circ = -2 * PI * sin(tn(s, j)) * (rn(s, i + 1) * EP(i + 1, j) - rn(s, i) * EP(i, j));
      BT(i, j) -= k * circ / a_bt(s, i, j);
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double circ = (rn(s, i + 1) * ET(i + 1, j) - rn(s, i) * ET(i, j)) * s->dth -
                    (ER(i, j + 1) - ER(i, j)) * (rn(s, i + 1) - rn(s, i));
      BP(i, j) -= k * circ / a_bp(s, i);
    }
}

static void absorb_b(ost *s) {
  int nr = s->nr, nt = s->nt;
  for (int i = 0; i <= nr; ++i) {
    double sg = sigma_abs(s, rn(s, i));
    if (sg > 0) for (int j = 0; j < nt; ++j) BR(i, j) -= sg * (BR(i, j) - BR0(i, j));
  }
  for (int i = 0; i < nr; ++i) {
    double sg = sigma_abs(s, rh(s, i));
    if (sg <= 0) continue;
    for (int j = 0; j <= nt; ++j) BT(i, j) -= sg * (BT(i, j) - BT0(i, j));
    for (int j = 0; j < nt; ++j) BP(i, j) -= sg * (BP(i, j) - BP0(i, j));
  }
}

/* ---------------------------------------------------------------- 5. Ampere
 * Eq. 19 in Stokes form over the exact dual faces, with the hybrid current of
 * Eq. 28: J = (1 - f) J_PIC + f J_FFE, J_FFE interpolated from the nodes as
 * in the correction step.  Then the star and outer boundaries and the
 * absorber.  J_PIC is cleared for the next deposit.                         */
static void ampere(ost *s) {
  int nr = s->nr, nt = s->nt;
  double k = s->dt, fp = 4 * PI * s->dt;
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) {
      double circ = 0.0;
      if (j < nt) circ += sin(th(s, j)) * BP(i, j);
      if (j > 0) circ -= sin(th(s, j - 1)) * BP(i, j - 1);
      circ *= 2 * PI * rh(s, i);
      double f = blend(s, 0.5 * (PSI(i, j) + PSI(i + 1, j)));
      double jt = (1 - f) * JR(i, j) + f * edge_r_mean(s, 10, i, j);
      ER(i, j) += k * circ / a_er(s, i, j) - fp * jt;
    }
  for (int i = 1; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double circ = -2 * PI * sin(th(s, j)) * (rh(s, i) * BP(i, j) - rh(s, i - 1) * BP(i - 1, j));
      double f = blend(s, 0.5 * (PSI(i, j) + PSI(i, j + 1)));
      double jt = (1 - f) * JT(i, j) + f * 0.5 * (NODE(11, i, j) + NODE(11, i, j + 1));
      ET(i, j) += k * circ / a_et(s, i, j) - fp * jt;
    }
  for (int i = 1; i < nr; ++i)
    for (int j = 1; j < nt; ++j) {
      double circ = (rh(s, i) * BT(i, j) - rh(s, i - 1) * BT(i - 1, j)) * (thi(s, j) - tlo(s, j)) -
                    (BR(i, j) - BR(i, j - 1)) * (rh(s, i) - rh(s, i - 1));
      double f = blend(s, PSI(i, j));
      double jt = (1 - f) * JP(i, j) + f * NODE(12, i, j);
      EP(i, j) += k * circ / a_ep(s, i, j) - fp * jt;
    }
  field_bc(s);
  for (int i = 0; i < nr; ++i) {
    double sg = sigma_abs(s, rh(s, i));
    if (sg > 0) for (int j = 0; j <= nt; ++j) ER(i, j) *= (1 - sg);
  }
  for (int i = 0; i <= nr; ++i) {
    double sg = sigma_abs(s, rn(s, i));
    if (sg <= 0) continue;
    for (int j = 0; j < nt; ++j) ET(i, j) *= (1 - sg);
    for (int j = 0; j <= nt; ++j) EP(i, j) *= (1 - sg);
  }
  for (int q = 6; q <= 8; ++q) memset(s->f[q], 0, sizeof(double) * fsize(s, q));
}

/* ------------------------------------------------------------ 7. injection
 * Reading of "maintain the density at the inner boundary at every time step"
 * (Sect. 5.1) and of continuous injection with kappa_inj (Sect. 4): in every
 * surface cell of the PIC domain the number of pairs is topped up to the
 * target kappa n_GJ V / w.  New pairs are co-located (neutral at birth),
 * uniformly placed in the first cell layer by Philox4x32-10 keyed
 * (seed; step, cell, k), in corotation with zero poloidal momentum.
 * Appended in cell-major, then k, order.                                    */
static void inject(ost *s) {
  if (s->c.inject != OR_INJ_ON) return;
  int nt = s->nt, nsp = s->c.n_species < 2 ? s->c.n_species : 2;
  /* e- with e+ (Sect. 4), or e- with protons from the crust (Sect. 5.1) */
  int isp[2] = {0, 1};
  if (s->c.inject_species[0] != s->c.inject_species[1]) {
    isp[0] = s->c.inject_species[0];
    isp[1] = s->c.inject_species[1];
  }
  uint32_t key[2] = {(uint32_t)s->c.seed, (uint32_t)(s->c.seed >> 32)};
  for (int j = 0; j < nt; ++j) {
    int32_t need = s->target[j] - s->surf[j] / 2;
    for (int32_t k = 0; k < need; ++k) {
      uint32_t ctr[4] = {(uint32_t)s->step, (uint32_t)((uint64_t)s->step >> 32), (uint32_t)j, (uint32_t)k}, x[4];
      or_philox4x32_10(ctr, key, x);
      double ox = (double)(x[0] >> 8) * (1.0 / 16777216.0);
      double oy = (double)(x[1] >> 8) * (1.0 / 16777216.0);
      double r = s->c.r_min * exp(ox * s->dlog), t = (j + oy) * s->dth;
      double v = s->omega * r * sin(t);
      double uphi = v / sqrt(1.0 - v * v);
      for (int ks = 0; ks < nsp; ++ks) {
        int sp = isp[ks];
        if (s->n[sp] >= s->cap) { fprintf(stderr, "oracle: particle capacity exceeded\n"); abort(); }
        int64_t p = s->n[sp]++;
        s->cell[sp][p] = j; /* i = 0 */
        s->p[sp][0][p] = ox; s->p[sp][1][p] = oy;
        s->p[sp][2][p] = 0.0; s->p[sp][3][p] = 0.0; s->p[sp][4][p] = uphi;
        s->p[sp][5][p] = s->c.w_inj;
        s->injected += s->c.w_inj;
      }
    }
  }
}

/* ------------------------------------------------------------------ 8. sort
 * Stable counting sort by tile key (tile = tile_r x tile_t cells), dropping
 * removed particles.  Ties keep their prior order.                          */
static void sort_species(ost *s, int sp) {
  int64_t n = s->n[sp], ntt = ncells_theta_tiles(s);
  int64_t ntr = (s->nr + s->c.tile_r - 1) / s->c.tile_r, nk = ntr * ntt;
  int64_t *cnt = (int64_t *)calloc(nk + 1, sizeof(int64_t));
  int32_t *cell = s->cell[sp];
  for (int64_t p = 0; p < n; ++p) {
    if (cell[p] < 0) continue;
    int64_t key = (cell[p] / s->nt / s->c.tile_r) * ntt + (cell[p] % s->nt) / s->c.tile_t;
    cnt[key + 1]++;
  }
  for (int64_t k = 0; k < nk; ++k) cnt[k + 1] += cnt[k];
  int64_t live = cnt[nk];
  int32_t *nc = (int32_t *)malloc(sizeof(int32_t) * (live ? live : 1));
  double *np[6];
  for (int q = 0; q < 6; ++q) np[q] = (double *)malloc(sizeof(double) * (live ? live : 1));
  for (int64_t p = 0; p < n; ++p) {
    if (cell[p] < 0) continue;
    int64_t key = (cell[p] / s->nt / s->c.tile_r) * ntt + (cell[p] % s->nt) / s->c.tile_t;
    int64_t d = cnt[key]++;
    nc[d] = cell[p];
    for (int q = 0; q < 6; ++q) np[q][d] = s->p[sp][q][p];
  }
  memcpy(cell, nc, sizeof(int32_t) * live);
  for (int q = 0; q < 6; ++q) { memcpy(s->p[sp][q], np[q], sizeof(double) * live); free(np[q]); }
  free(nc);
  free(cnt);
  s->n[sp] = live;
}

int or_sort_now(void *st) {
  ost *s = (ost *)st;
  for (int sp = 0; sp < s->c.n_species; ++sp) sort_species(s, sp);
  return 0;
}

int or_step(void *st, int32_t nsteps, int32_t stages) {
  ost *s = (ost *)st;
  for (int32_t n = 0; n < nsteps; ++n) {
    if (stages & OR_ST_NODE) node_pass_a(s);
    if (stages & OR_ST_PUSH) push_all(s);
    if (stages & OR_ST_FARADAY1) faraday(s, 0.5);
    if (stages & OR_ST_AMPERE) ampere(s);
    if (stages & OR_ST_CORRECT) correct_e(s);
    if (stages & OR_ST_FARADAY2) { faraday(s, 0.5); absorb_b(s); }
    if (stages & OR_ST_INJECT) { inject(s); create_pairs(s); }
    s->step++;
    if ((stages & OR_ST_SORT) && s->c.sort_every > 0 && s->step % s->c.sort_every == 0)
      for (int sp = 0; sp < s->c.n_species; ++sp) sort_species(s, sp);
  }
  return 0;
}

/* ------------------------------------------------- maps and spectra (5.2) */
int or_species_maps(void *st, int sp, double *density, double *energy) {
  ost *s = (ost *)st;
  int64_t nc = (int64_t)s->nr * s->nt;
  for (int64_t c = 0; c < nc; ++c) { density[c] = 0.0; energy[c] = 0.0; }
  for (int64_t p = 0; p < s->n[sp]; ++p) {
    int32_t c = s->cell[sp][p];
    if (c < 0) continue;
    double u2 = s->p[sp][2][p] * s->p[sp][2][p] + s->p[sp][3][p] * s->p[sp][3][p] + s->p[sp][4][p] * s->p[sp][4][p];
    double gamma = sqrt(1.0 + u2);
    density[c] += s->p[sp][5][p];
    energy[c] += s->p[sp][5][p] * s->c.m[sp] * (gamma - 1.0);
  }
  for (int i = 0; i < s->nr; ++i)
    for (int j = 0; j < s->nt; ++j) {
      double v = 2.0 * PI / 3.0 * (pow(rn(s, i + 1), 3) - pow(rn(s, i), 3)) * dcp(s, j);
      density[(int64_t)i * s->nt + j] /= v;
      energy[(int64_t)i * s->nt + j] /= v;
    }
  return 0;
}

int or_spectrum(void *st, int sp, int nbins, double lg_min, double lg_max, double *out) {
  ost *s = (ost *)st;
  for (int b = 0; b < nbins; ++b) out[b] = 0.0;
  for (int64_t p = 0; p < s->n[sp]; ++p) {
    if (s->cell[sp][p] < 0) continue;
    double u2 = s->p[sp][2][p] * s->p[sp][2][p] + s->p[sp][3][p] * s->p[sp][3][p] + s->p[sp][4][p] * s->p[sp][4][p];
    double x = floor((log10(sqrt(1.0 + u2)) - lg_min) * nbins / (lg_max - lg_min));
    int b = x < 0 ? 0 : (x > nbins - 1 ? nbins - 1 : (int)x);
    out[b] += s->p[sp][5][p];
  }
  return 0;
}

/* ----------------------------------------------------------- diagnostics */
int or_node_charge(void *st, double *q) {
  ost *s = (ost *)st;
  int nt = s->nt;
  memset(q, 0, sizeof(double) * fsize(s, 9));
  for (int sp = 0; sp < s->c.n_species; ++sp)
    for (int64_t p = 0; p < s->n[sp]; ++p) {
      int32_t c = s->cell[sp][p];
      if (c < 0) continue;
      int i = c / nt, j = c % nt;
      double x = s->p[sp][0][p], y = s->p[sp][1][p], qw = s->c.q[sp] * s->p[sp][5][p];
      q[(int64_t)i * (nt + 1) + j] += qw * (1 - x) * (1 - y);
      q[(int64_t)(i + 1) * (nt + 1) + j] += qw * x * (1 - y);
      q[(int64_t)i * (nt + 1) + j + 1] += qw * (1 - x) * y;
      q[(int64_t)(i + 1) * (nt + 1) + j + 1] += qw * x * y;
    }
  return 0;
}

/* Poynting flux through the sphere r_{i+1/2} (Eq. 35):
 * L = (c/4 pi) sum over the sphere of (E_theta B_phi - E_phi B_theta) dA.    */
static double poynting(const ost *s, int i) {
  int nt = s->nt;
  double l = 0.0, r = rh(s, i);
  for (int j = 0; j < nt; ++j)
    l += 0.5 * (ET(i, j) + ET(i + 1, j)) * BP(i, j) * 2 * PI * r * r * dcp(s, j);
  for (int j = 0; j <= nt; ++j)
    l -= 0.5 * (EP(i, j) + EP(i + 1, j)) * BT(i, j) * a_er(s, i, j);
  return l / (4 * PI);
}

int or_diagnostics(void *st, or_diag *o, double *lprof) {
  ost *s = (ost *)st;
  int nr = s->nr, nt = s->nt;
  memset(o, 0, sizeof(*o));
  /* psi from the current B_r */
  double *psi = (double *)malloc(sizeof(double) * fsize(s, 9));
  for (int i = 0; i <= nr; ++i) {
    double acc = 0.0, r2 = rn(s, i) * rn(s, i);
    psi[(int64_t)i * (nt + 1)] = 0.0;
    for (int j = 0; j < nt; ++j) { acc += BR(i, j) * r2 * dcp(s, j); psi[(int64_t)i * (nt + 1) + j + 1] = acc; }
  }
  int iout = (int)floor(log(2.0 * s->c.r_lc / s->c.r_min) / s->dlog + 0.5);
  if (iout > nr) iout = nr;
  o->psi_open = psi[(int64_t)iout * (nt + 1) + nt / 2];
  free(psi);
  /* L(r) and the dissipation rate of Eq. 36 */
  double sin_ = 0, sout = 0;
  int nin = 0, nout = 0;
  for (int i = 0; i < nr; ++i) {
    double l = poynting(s, i), r = rh(s, i);
    if (lprof) lprof[i] = l;
    if (r >= s->c.r_min && r <= 2 * s->c.r_min) { sin_ += l; nin++; }
    if (r >= 2 * s->c.r_lc && r <= 3 * s->c.r_lc) { sout += l; nout++; }
  }
  o->l_in = nin ? sin_ / nin : 0;
  o->l_out = nout ? sout / nout : 0;
  o->eps = (o->l_out != 0) ? fabs(o->l_in - o->l_out) / fabs(o->l_out) : 0;
  /* Gauss residual on interior nodes away from the boundaries */
  double *q = (double *)malloc(sizeof(double) * fsize(s, 9));
  or_node_charge(s, q);
  int imax = (int)floor(s->xi_abs) - 2;
  if (imax > nr - 2) imax = nr - 2;
  double sum2 = 0;
  int64_t cnt = 0;
  for (int i = 2; i <= imax; ++i)
    for (int j = 0; j <= nt; ++j) {
      double flux = ER(i, j) * a_er(s, i, j) - ER(i - 1, j) * a_er(s, i - 1, j);
      if (j < nt) flux += ET(i, j) * a_et(s, i, j);
      if (j > 0) flux -= ET(i, j - 1) * a_et(s, i, j - 1);
      double v = vnode(s, i, j), qq = q[(int64_t)i * (nt + 1) + j];
      double res = (flux / (4 * PI) - qq) / v;
      if (fabs(res) > o->gauss_max) o->gauss_max = fabs(res);
      if (fabs(qq / v) > o->rho_max) o->rho_max = fabs(qq / v);
      sum2 += res * res;
      cnt++;
    }
  o->gauss_rms = cnt ? sqrt(sum2 / cnt) : 0;
  free(q);
  /* field energies: value^2 times the volume of its (edge x dual face) or
   * (face x dual edge) box, over 8 pi */
  double ue = 0, ub = 0;
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) ue += ER(i, j) * ER(i, j) * a_er(s, i, j) * (rn(s, i + 1) - rn(s, i));
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j) ue += ET(i, j) * ET(i, j) * a_et(s, i, j) * rn(s, i) * s->dth;
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j <= nt; ++j) ue += EP(i, j) * EP(i, j) * a_ep(s, i, j) * 2 * PI * rn(s, i) * sin(tn(s, j));
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j) ub += BR(i, j) * BR(i, j) * a_br(s, i, j) * (rhi(s, i) - rlo(s, i));
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j <= nt; ++j) ub += BT(i, j) * BT(i, j) * a_bt(s, i, j) * rh(s, i) * (thi(s, j) - tlo(s, j));
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nt; ++j) ub += BP(i, j) * BP(i, j) * a_bp(s, i) * 2 * PI * rh(s, i) * sin(th(s, j));
  o->u_e = ue / (8 * PI);
  o->u_b = ub / (8 * PI);
  for (int sp = 0; sp < s->c.n_species; ++sp) {
    double ke = 0, cn = 0;
    for (int64_t p = 0; p < s->n[sp]; ++p) {
      if (s->cell[sp][p] < 0) continue;
      double u0 = s->p[sp][2][p], u1 = s->p[sp][3][p], u2 = s->p[sp][4][p];
      ke += s->p[sp][5][p] * s->c.m[sp] * (sqrt(1 + u0 * u0 + u1 * u1 + u2 * u2) - 1);
      cn += 1;
    }
    o->kinetic[sp] = ke;
    o->count[sp] = cn;
  }
  o->injected = s->injected;
  o->killed = s->killed;
  o->radiated = s->radiated;
  o->nonfinite = s->nonfinite;
  o->created = s->created;
  o->clamps = s->clamps;
  {
    double bad = 0;
    for (int k = 0; k < 6; ++k)
      for (int64_t q = 0; q < fsize(s, k); ++q) bad += !isfinite(s->f[k][q]);
    o->nonfinite_fields = bad;
  }
  return 0;
}
