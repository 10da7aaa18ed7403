/*
 * hff_oracle.h -- plain, slow FP64 CPU oracle for one time step of the hybrid
 * force-free / particle-in-cell scheme of Soudais, Cerutti & Contopoulos (2024)
 * for the axisymmetric aligned rotator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; the two agree only because both follow the same written
 * definitions of the scheme.
 *
 * Units: Gaussian with c = 1 (and r_star = r_min, B_star = b_star as given).
 * Grid: log-spaced in r, uniform in theta on [0, pi] (Sect. 4).
 * Field layout (row-major, theta index fastest):
 *   E_r  (i+1/2, j)    nr     x (nt+1)
 *   E_th (i,   j+1/2)  (nr+1) x nt
 *   E_ph (i,   j)      (nr+1) x (nt+1)
 *   B_r  (i,   j+1/2)  (nr+1) x nt
 *   B_th (i+1/2, j)    nr     x (nt+1)
 *   B_ph (i+1/2, j+1/2) nr    x nt
 * J_r, J_th, J_ph share the E locations.  Node scalars (psi, ...) are
 * (nr+1) x (nt+1).
 */
#ifndef HFF_ORACLE_H
#define HFF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Initial field geometry. */
enum { OR_DIPOLE = 0, OR_MONOPOLE = 1, OR_SYNTH = 2, OR_UNIFORM = 3, OR_MICHEL = 4 };

/* Injection modes: OR_INJ_OFF, or top-up to kappa * n_GJ in the first cell
 * layer (Sect. 4 for the monopole, Sect. 5.1 for the dipole). */
enum { OR_INJ_OFF = 0, OR_INJ_ON = 1 };

/* Stage bits.  One full step runs the stages in the order NODE, PUSH,
 * FARADAY1, AMPERE, CORRECT, FARADAY2, INJECT, SORT. */
enum {
  OR_ST_NODE = 1,      /* psi and J_perp at nodes                   */
  OR_ST_CORRECT = 2,   /* Delta E at nodes, E += f * <Delta E>      */
  OR_ST_PUSH = 4,      /* particle push, move, deposit              */
  OR_ST_FARADAY1 = 8,  /* B^n -> B^{n+1/2}                          */
  OR_ST_AMPERE = 16,   /* E^n -> E^{n+1} with blended J, BCs        */
  OR_ST_FARADAY2 = 32, /* B^{n+1/2} -> B^{n+1}, absorber on B       */
  OR_ST_INJECT = 64,   /* surface pair injection                    */
  OR_ST_SORT = 128,    /* stable tile sort + compaction (cadence)   */
  OR_ST_ALL = 255
};

typedef struct or_config {
  int32_t nr, nt;            /* cells in r and theta                         */
  double r_min, r_max;       /* r_min = stellar radius                       */
  double r_lc;               /* light-cylinder radius, Omega = 1 / r_lc      */
  double b_star;             /* surface field scale                          */
  int32_t geom;              /* OR_DIPOLE ...                                */
  double courant;            /* fraction of the 2D CFL limit                 */
  double r_abs;              /* absorbing layer start                        */
  double absorb_strength;    /* damping per step at r_max                    */
  int32_t n_breaks;          /* blend table size (0 = f == 0 everywhere)     */
  double psi_break[4];       /* in units of psi_unit (see or_psi_unit)       */
  double f_break[4];         /* f value at each break                        */
  int32_t n_species;         /* 1 .. 4                                       */
  double q[4], m[4];         /* charge (units of e) and mass per species     */
  int32_t inject;            /* OR_INJ_*                                     */
  double kappa_inj;          /* multiplicity of the injected plasma          */
  double w_inj;              /* weight of an injected macro-particle         */
  double gamma_rad;          /* radiation-reaction Lorentz factor (0 = off)  */
  double b_ref;              /* field at which gamma_rad is quoted           */
  double rr_scale;           /* ramp multiplier of the radiation reaction    */
  double shell_r;            /* u_perp removed for r < shell_r               */
  double synth_psi_open;     /* OR_SYNTH open flux, units of psi_unit        */
  uint64_t seed;             /* injection RNG key                            */
  int64_t capacity;          /* particles per species                        */
  int32_t tile_r, tile_t;    /* sort tile shape in cells                     */
  int32_t sort_every;        /* sort cadence in steps (0 = never)            */
  double gamma_th;           /* pair creation threshold (0 = off), Sect. 5.1 */
  double gamma_s;            /* Lorentz factor of the created pairs          */
  int32_t inject_species[2]; /* species injected together; equal = (0, 1)   */
  int32_t ff_delta_only;     /* 0: the corrected node E returns to the edges,
                                1: only the corrections Delta E (Sect. 3),
                                2: only the corrections, except on the radial
                                edges at the star, where the corrected node
                                E of row 1 returns                          */
  double ff_filter;          /* sigma of the fourth-difference filter of E_r
                                along r and E_th along theta where f > 0
                                (0 = off; 1 removes the odd-even mode)      */
} or_config;

typedef struct or_diag {
  double psi_open;           /* psi at (r nearest 2 R_LC, theta = pi/2)      */
  double eps;                /* |L_in - L_out| / L_out  (Eq. 36)             */
  double l_in, l_out;
  double gauss_max, gauss_rms, rho_max; /* density units                     */
  double u_e, u_b;           /* field energies                               */
  double kinetic[4];         /* sum w m (gamma - 1) per species              */
  double count[4];
  double injected, killed, radiated, nonfinite;
  double created;            /* weight of the pairs created (both species)   */
  double clamps;             /* running count of E^2 > B^2 renormalisations  */
  double nonfinite_fields;   /* non-finite E or B values on the mesh now     */
} or_diag;

/* Per-cell number density sum(w)/V and kinetic energy density
 * sum(w m (gamma-1))/V of species sp (nr x nt, theta fastest; Sect. 5.2). */
int or_species_maps(void *st, int sp, double *density, double *energy);
/* Sum of weights of species sp in nbins bins uniform in log10(gamma) on
 * [lg_min, lg_max), out-of-range particles in the end bins (Sect. 5.2). */
int or_spectrum(void *st, int sp, int nbins, double lg_min, double lg_max, double *out);

void *or_create(const or_config *cfg);
double or_config_dt(const or_config *cfg);
void or_destroy(void *st);
double or_dt(void *st);
double or_psi_unit(void *st);
int64_t or_step_index(void *st);
void or_set_step_index(void *st, int64_t step); /* one step split into stage groups */

/* which: 0..5 = E_r E_th E_ph B_r B_th B_ph; 6..8 = J_r J_th J_ph (PIC);
 *        9 = psi (nodes); 10..12 = J_perp at nodes; 13..15 = Delta E at nodes;
 *        16..18 = initial B_r B_th B_ph. */
int64_t or_field_size(void *st, int which);
int or_get_field(void *st, int which, double *out);
int or_set_field(void *st, int which, const double *in);

int64_t or_count(void *st, int species);
int or_set_particles(void *st, int species, int64_t n, const int32_t *cell,
                     const double *xo, const double *yo, const double *ur,
                     const double *ut, const double *up, const double *w);
int or_get_particles(void *st, int species, int32_t *cell, double *xo,
                     double *yo, double *ur, double *ut, double *up, double *w);
int32_t or_surface_count(void *st, int j);
/* Overwrites one surface count (particles in cell (0, j) after the last
 * push).  For tests that hand the oracle a state pushed elsewhere and check
 * the injection that follows from it. */
void or_set_surface_count(void *st, int j, int32_t v);
int32_t or_inject_target(void *st, int j);

void or_set_rr_scale(void *st, double v);
int or_step(void *st, int32_t nsteps, int32_t stages);
/* Stable tile sort of every species now, without advancing the step. */
int or_sort_now(void *st);

/* Diagnostics (Sect. 4): L(r) at every half-node row r_{i+1/2} into l_prof
 * (nr values, may be NULL). */
int or_diagnostics(void *st, or_diag *out, double *l_prof);
/* Node charges from CIC deposit of the live particles, (nr+1) x (nt+1). */
int or_node_charge(void *st, double *q_out);

/* Pure functions used by the pins. */
void or_push_local(double qm, double krr, double dt, const double u[3],
                   const double e[3], const double b[3], double out[3],
                   double *radiated_dgamma);
void or_move_local(double r, double th, double dt, const double u[3],
                   double *dr, double *dth, double *dphi, double u_out[3]);
double or_blend(void *st, double psi);
/* The linear gather of E and B at offset (xo, yo) of cell (i, j), and one
 * charge-conserving deposit of charge qw moving from (x0, y0) to (x1, y1)
 * (logical coordinates relative to node (i0, j0)) with azimuthal velocity
 * vphi, added to J_r, J_th, J_ph, as the push performs them. */
void or_gather(void *st, int32_t i, int32_t j, double xo, double yo, double e[3], double b[3]);
void or_deposit(void *st, double qw, int32_t i0, int32_t j0, double x0, double y0, double x1,
                double y1, double vphi);

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]);

#ifdef __cplusplus
}
#endif
#endif
