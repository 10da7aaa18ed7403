/*
 * hff.h -- C ABI of the GB300 (sm_103a) hybrid force-free / particle-in-cell
 * time step for the axisymmetric aligned pulsar rotator of Soudais, Cerutti &
 * Contopoulos (2024).
 *
 * One call of hff_step advances one or more magnetospheres by whole time
 * steps on the GPU:
 *   - flux function Psi as a theta-prefix of B_r (Sect. 3, Eq. 27): FP64 in
 *     FP64 instances, a float pair of about 48 significant bits summed from
 *     exact products in FP32 instances
 *   - blend mask f(Psi) (Eqs. 29-31 generalised to a piecewise-linear table),
 *     the segment chosen by comparisons at that precision
 *   - force-free perpendicular current (first term of Eq. 24)
 *   - modified Boris push with radiation reaction (Eqs. 15-17), move,
 *     charge-conserving deposit of J_PIC
 *   - Yee field advance (Eqs. 18-19) with J = (1-f) J_PIC + f J_FFE (Eq. 28)
 *   - E renormalisation E.B = 0 and E^2 <= B^2 (Eqs. 25-26) weighted by f
 *   - corotating star and absorbing layer (Sect. 4), surface pair injection
 *     (Sects. 4 and 5.1), stable tile sort of the particles.
 *
 * Units are Gaussian with c = 1.  Grid: nr x nt cells, r log-spaced on
 * [r_min, r_max], theta uniform on [0, pi].  Field arrays are row-major with
 * the theta index fastest:
 *   which  name   location         shape
 *   0      E_r    (i+1/2, j)       nr     x (nt+1)
 *   1      E_th   (i, j+1/2)       (nr+1) x nt
 *   2      E_ph   (i, j)           (nr+1) x (nt+1)
 *   3      B_r    (i, j+1/2)       (nr+1) x nt
 *   4      B_th   (i+1/2, j)       nr     x (nt+1)
 *   5      B_ph   (i+1/2, j+1/2)   nr     x nt
 *   6..8   J_r, J_th, J_ph of the last particle deposit (E locations)
 *   9      Psi at the nodes        (nr+1) x (nt+1), always FP64
 *   10..12 J_perp at the nodes     (nr+1) x (nt+1)
 *   13..15 Delta E at the nodes    (nr+1) x (nt+1)
 *   16     f at the E_r edges      nr     x (nt+1)   (Eqs. 29-31; read only)
 *   17     f at the E_th edges     (nr+1) x nt
 *   18     f at the nodes (E_ph)   (nr+1) x (nt+1)
 *   19     force-free cell flags   nr     x nt, one byte each (1 = f >= 1 at
 *          the mean Psi of the cell's corners: no particles, Eq. 29)
 * Field values are FP32 (HFF_FP32) or FP64 (HFF_FP64) as configured.
 *
 * Particles (per species, structure of arrays): int32 cell = i * nt + j
 * (-1 = removed), offsets xo, yo in [0, 1) inside the cell in the logical
 * (ln r, theta) coordinates, u_r, u_th, u_ph = gamma v / c in the local
 * spherical basis, and the macro-particle weight w; all but cell are in the
 * configured precision.
 *
 * Memory and streams: the caller owns all device memory.  hff_plan reports the
 * bytes one instance needs; the caller allocates them (for instance as a torch
 * uint8 tensor), passes them to hff_init and keeps them alive until
 * hff_destroy returns.  The library allocates no device memory of its own
 * apart from CUDA graphs; each handle holds a few KB of pinned host memory
 * for per-step scalars and counter readback.  All work is queued on the
 * caller's stream.
 *
 * Errors: every function returns HFF_OK (0) or a negative HFF_ERR_* code;
 * hff_last_error() gives a message for the calling thread.  Faults detected on
 * the device (capacity overflow, non-finite particles) are latched in a status
 * word and reported by hff_status.
 */
#ifndef HFF_H
#define HFF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HFF_OK 0
#define HFF_ERR_ARG (-1)       /* invalid argument or configuration        */
#define HFF_ERR_CAPACITY (-2)  /* particle or memory capacity exceeded     */
#define HFF_ERR_CUDA (-3)      /* a CUDA call failed                       */
#define HFF_ERR_TIMEOUT (-4)   /* a bounded device wait gave up            */
#define HFF_ERR_NONFINITE (-5) /* non-finite values were met on the device */

/* initial field geometry */
#define HFF_GEOM_DIPOLE 0   /* Psi = mu sin^2(theta) / r (Eq. 37)                 */
#define HFF_GEOM_MONOPOLE 1 /* Psi = Psi* (1 - cos theta) (Eq. 32)                */
#define HFF_GEOM_SYNTH 2    /* dipole inside R_LC, split monopole outside          */
#define HFF_GEOM_UNIFORM 3  /* Psi = B0 r^2 sin^2(theta) / 2 (test field)          */
#define HFF_GEOM_MICHEL 4   /* Michel monopole with B_ph and E_th (Eqs. 32-33)     */

#define HFF_FP32 0
#define HFF_FP64 1

#define HFF_HOST 0
#define HFF_DEVICE 1

/* hff_config.field_pass */
#define HFF_FIELDS_AUTO 0
#define HFF_FIELDS_FUSED 1
#define HFF_FIELDS_SPLIT 2

/* stage bits of hff_step_stages (a full step runs all, in this order) */
#define HFF_ST_NODE 1      /* Psi, per-cell force-free flag; J_perp here unless
                              the fused field pass (with all four field stages
                              in the same call) computes it                 */
#define HFF_ST_CORRECT 2   /* Delta E at the nodes and E += f <Delta E>          */
#define HFF_ST_PUSH 4      /* push, move, deposit                               */
#define HFF_ST_FARADAY1 8  /* B^n -> B^{n+1/2}                                  */
#define HFF_ST_AMPERE 16   /* E^n -> E^{n+1}, boundaries, absorber on E          */
#define HFF_ST_FARADAY2 32 /* B^{n+1/2} -> B^{n+1}, absorber on B                */
#define HFF_ST_INJECT 64   /* surface pair injection                            */
#define HFF_ST_SORT 128    /* stable tile sort + compaction (on its cadence)     */
#define HFF_ST_ALL 255
#define HFF_ST_NOCOUNT 256 /* with stages that exclude INJECT: run them without
                              advancing the step counter (one step split into
                              stage groups with exchanges in between counts
                              once, at its INJECT group)                        */
/* order of execution: NODE, PUSH, FARADAY1, AMPERE, CORRECT, FARADAY2,
 * INJECT, SORT */

/* scalars for hff_set_scalar */
#define HFF_SCALAR_RR_SCALE 0 /* ramp multiplier of the radiation reaction (Sect. 5.1) */

typedef struct hff_config {
  int32_t nr, nt;           /* cells in r and theta (each >= 8)                  */
  double r_min, r_max;      /* radial extent; r_min is the stellar radius        */
  double r_lc;              /* light-cylinder radius; Omega = c / r_lc (Eq. 1)   */
  double b_star;            /* surface field scale: mu = b_star r_min^3          */
  int32_t geom;             /* HFF_GEOM_*                                         */
  double courant;           /* fraction of the 2D CFL limit, (0, 0.9]            */
  double r_abs;             /* start of the absorbing layer (Sect. 4: 3 R_LC);
                               >= 3 cells inside r_max, or >= r_max for a grid
                               without an absorbing layer (a slab of a larger
                               run)                                              */
  double absorb_strength;   /* damping per step at r_max (cubic ramp from r_abs) */
  int32_t n_breaks;         /* 0..4 breakpoints of f; 0 means f = 0 (pure PIC)   */
  double psi_break[4];      /* in units of Psi_pc = mu/R_LC (dipolar fields) or
                               Psi* = b_star r_min^2 (monopoles), ascending      */
  double f_break[4];        /* f at each breakpoint                              */
  int32_t n_species;        /* 1..4; species 0 and 1 form the injected pairs     */
  double q[4], m[4];        /* charge (units of e) and mass                      */
  int32_t inject;           /* 1 = surface top-up injection on                   */
  double kappa_inj;         /* injected multiplicity (Sect. 4: 10)               */
  double w_inj;             /* weight of an injected macro-particle              */
  double gamma_rad;         /* radiation-reaction Lorentz factor, 0 = off        */
  double b_ref;             /* field at which gamma_rad is quoted                */
  double rr_scale;          /* initial ramp multiplier (see HFF_SCALAR_RR_SCALE) */
  double shell_r;           /* u_perp removed below this radius (Sect. 5.1)      */
  double synth_psi_open;    /* HFF_GEOM_SYNTH open flux in units of Psi_pc       */
  uint64_t seed;            /* key of the injection generator                    */
  int64_t capacity;         /* particle slots per species                        */
  int32_t tile_r, tile_t;   /* sort tile in cells (0 = default 16 x 32)          */
  int32_t sort_every;       /* sort cadence in steps, 1..32 (0 = never sort); the
                               push stages each tile with a halo of the farthest
                               drift between sorts, so a long cadence needs small
                               enough tiles (else HFF_ERR_ARG at init)           */
  int32_t precision;        /* HFF_FP32 or HFF_FP64                              */
  double gamma_th;          /* threshold pair creation (Sect. 5.1): a lepton whose
                               Lorentz factor exceeds gamma_th after its push
                               creates an e+- pair (0 = off, else > 1)           */
  double gamma_s;           /* Lorentz factor of each created particle (>= 1);
                               both move along the parent's direction, at its
                               position, with its weight; the parent is kept     */
  int32_t inject_species[2];/* the two species the surface injection creates
                               together: (0, 1) = e- and e+ (Sect. 4), (0, 2) =
                               e- and protons extracted from the crust
                               (Sect. 5.1); equal values mean (0, 1)             */
  int32_t ff_delta_only;    /* what returns from the nodes to the staggered E
                               after the renormalisation of Eqs. 25-26 (Sect. 3),
                               by arithmetic means, weighted by f: 0 = the
                               corrected field itself (E_r and E_th are then
                               averaged 1-2-1 every step in the force-free
                               domain; stable over long runs), 1 = only the
                               corrections Delta E (second order on a stationary
                               solution, but it lets a mode grow near the axis
                               next to a force-free / PIC interface within
                               ~1e4-1e5 steps on 1024^2 - 2048^2 grids), 2 = the
                               corrections, except on the radial edges that end
                               on the star, which take the corrected field of
                               node row 1 (their only interior node): this
                               removes the growing mode of 1, which starts on
                               the stellar rows.  2 runs on the separate field
                               passes: field_pass FUSED is rejected with it, and
                               AUTO takes the separate passes                    */
  double ff_filter;         /* sigma in [0, 1] of a fourth-difference filter of
                               E_r along r and E_th along theta, applied with the
                               correction, weighted by f: E -= f sigma/16 D4(E).
                               The two-point means of the collocation do not see
                               the odd-even component of those fields, so the
                               node corrections cannot act on it; sigma = 1
                               removes it, and a smooth field changes by O(h^4)
                               per step.  0 = off (a reading: the paper is silent) */
  int32_t field_pass;       /* how the field update runs (the results agree to
                               rounding): HFF_FIELDS_FUSED = one row-pipelined
                               pass over theta strips and row segments after
                               the push, which computes J_perp itself and reads
                               E and dB once (it needs a halo snapshot of E and
                               dB, about 14% of their size on a 4096^2 grid);
                               HFF_FIELDS_SPLIT = J_perp at the nodes before
                               the push, then four kernels after it (Faraday
                               half step, Ampere, renormalisation and return,
                               Faraday half step with the absorber), each over
                               every row at once; HFF_FIELDS_AUTO (0) = fused
                               when segments of 32 rows give at least one wave
                               of its blocks on a GB300 (six per SM in FP32,
                               three in FP64, on 152 SMs), else split: on
                               smaller grids the fused pass's row chains run
                               on too few blocks                               */
} hff_config;

typedef struct hff_info {
  double dt;                /* time step (Courant rule of the config)            */
  double psi_unit;          /* Psi_pc or Psi* in code units                      */
  int64_t step;             /* steps taken                                       */
  int64_t count[4];         /* particle slots in use per species (incl. removed) */
  int32_t tile_r, tile_t, sort_every, precision;
  int64_t kernels_per_step; /* kernels one step launches (sort steps: more)      */
  int64_t kernels_launched; /* kernels launched by hff_step since hff_init       */
  int64_t pushed_tiled;     /* particle pushes by the tile-staged kernel (total) */
  int64_t pushed_tail;      /* particle pushes by the global-memory kernel       */
  int64_t readback_bytes;   /* bytes hff_get_info copies device -> host          */
  int64_t n_inst;           /* instances behind the handle (ensemble: members)   */
  int32_t field_pass;       /* the field update this instance runs:
                               HFF_FIELDS_FUSED or HFF_FIELDS_SPLIT (ensemble:
                               the first member's)                              */
} hff_info;

typedef struct hff_particle_view {
  int64_t n;                /* slots in use (removed particles have cell < 0)    */
  int32_t *cell;            /* device pointers, valid until the next hff_step    */
  void *xo, *yo, *ur, *ut, *up, *w;
} hff_particle_view;

typedef struct hff_diag {
  double psi_open;          /* Psi at (node row nearest 2 R_LC, theta = pi/2)    */
  double eps;               /* |L_in - L_out| / L_out (Eq. 36)                   */
  double l_in, l_out;       /* L averaged over [r_min, 2 r_min] and [2, 3] R_LC  */
  double gauss_max, gauss_rms, rho_max; /* |div E/4pi - rho| on interior nodes   */
  double u_e, u_b;          /* field energies (1/8pi) int E^2, B^2 dV            */
  double kinetic[4];        /* sum w m (gamma - 1) per species                   */
  double count[4];          /* live particles per species                        */
  double injected, killed, radiated, nonfinite; /* running totals (weights)      */
  double created;           /* weight of the created pairs (both species)        */
  double clamps;            /* running count of E^2 > B^2 renormalisations
                               (Eq. 26) at force-free nodes                      */
  double nonfinite_fields;  /* non-finite E or B values now on the mesh; if any,
                               HFF_ERR_NONFINITE is latched for hff_status       */
} hff_diag;

typedef struct hff_handle hff_handle;

/* Device bytes that n_inst instances need (Sect. 4 grid, Sect. 3 particles):
 * cfg points to n_inst configurations (1 <= n_inst <= 4096); the total is the
 * sum over the instances, each a multiple of 256 bytes.  The instances of an
 * ensemble (n_inst > 1) must share precision and sort_every; grids, particle
 * capacities, tiles, R_LC, seeds and every other field may differ.  Returns
 * HFF_ERR_ARG for an invalid configuration (the message names the instance). */
int hff_plan(const hff_config *cfg, int n_inst, size_t *bytes);

/* Initialise n_inst instances in caller-owned device memory dev_mem (>= the
 * planned bytes, 256-byte aligned) on the CUDA stream `stream` (cudaStream_t,
 * may be NULL for the legacy stream).  Builds the geometry in FP64 on the host,
 * the initial B from the analytic flux function of cfg->geom (Eqs. 32, 37) by
 * exact-area differences, E = 0 except the corotating star (Sect. 4), and no
 * particles.  *out receives a handle owned by the caller (free with
 * hff_destroy).
 *
 * Ensemble (n_inst > 1): the instances are independent simulations carved
 * from dev_mem in order, addressed by `inst` in the per-instance calls
 * below.  hff_step advances all of them in lockstep with ONE graph launch
 * per step (and one per sort step): every instance's kernels form a parallel
 * branch of that graph, so small instances fill the GPU together.
 * hff_step_timed's events then bracket each whole ensemble step;
 * hff_set_scalar applies to every instance; hff_get_info returns totals over
 * the instances (n_inst = their number); hff_status reports the first
 * instance with a latched error and clears all of them. */
int hff_init(const hff_config *cfg, int n_inst, void *dev_mem, size_t bytes, void *stream,
             hff_handle **out);

/* Replace the particles of one species by n particles (SoA arrays as described
 * above; `where` = HFF_HOST or HFF_DEVICE says where the source arrays live).
 * Values must be in the configured precision.  The particles are sorted by
 * tile if sorting is enabled.  HFF_ERR_CAPACITY if n > capacity.  A cell
 * index at or past nr * nt is invalid: the load completes with those
 * particles removed and returns HFF_ERR_ARG. */
int hff_load_particles(hff_handle *h, int inst, int species, int64_t n, const int32_t *cell,
                       const void *xo, const void *yo, const void *ur, const void *ut,
                       const void *up, const void *w, int where);

/* Overwrite field `which` (0..5, or 6..8 for J_PIC) with `bytes` bytes from
 * src (host or device).  Setting J between the push and Ampere's law of a
 * step split into stage groups adds current deposited elsewhere (for
 * instance the neighbour's share in a decomposed run).
 * B is held as the initial field B_0 plus a perturbation (the Yee update
 * advances the perturbation, with curl B_0 precomputed in FP64), so setting
 * B stores B - B_0 and reading it (hff_fields) returns the sum, each rounded
 * once in the instance precision.  B_0 itself, also the absorber's reference,
 * is not changed. */
int hff_set_field(hff_handle *h, int inst, int which, const void *src, size_t bytes, int where);

/* Copy field `which` (0..19, see the table above) into dst (host or device,
 * `bytes` must equal the field size).  which = 9 computes Psi (Eq. 27) in FP64
 * from the current B_r.  which = 16..19 compute the blend weights from the
 * current B exactly as the next step's node pass does (the step's own flux
 * prefix and comparisons).  Synchronises the stream. */
int hff_fields(hff_handle *h, int inst, int which, void *dst, size_t bytes, int where);

/* Advance nsteps whole steps (asynchronous on the stream; one CUDA graph per
 * step, replayed).  Returns the latched device status of earlier steps. */
int hff_step(hff_handle *h, int32_t nsteps);

/* As hff_step, but for step k records the caller's CUDA events ev_begin[k]
 * and ev_end[k] (cudaEvent_t) immediately before and after the tile-staged
 * push kernel, so that its duration can be timed inside a run of whole
 * steps.  The step is the same single graph as hff_step's with two event-
 * record nodes added, whose events are set before each launch. */
int hff_step_timed(hff_handle *h, int32_t nsteps, void *const *ev_begin, void *const *ev_end);

/* Advance nsteps steps running only the stages in the HFF_ST_* mask (eager
 * launches; used to test the parts of a step). */
int hff_step_stages(hff_handle *h, int32_t nsteps, int32_t stages);

/* Set a per-step scalar (HFF_SCALAR_*).  The value is copied to the device
 * on the stream, so it takes effect for the steps queued after the call. */
int hff_set_scalar(hff_handle *h, int which, double value);

/* Device views of one species' particles (valid until the next hff_step).
 * Synchronises the stream to read the count. */
int hff_particles(hff_handle *h, int inst, int species, hff_particle_view *out);

/* FP64 diagnostics of Sect. 4: spin-down L(r) (Eq. 35) at every half-node row
 * into l_prof (nr doubles on the host, may be NULL), the dissipation rate of
 * Eq. 36, the open flux, Gauss's law residual, energies and counters.
 * Synchronises the stream. */
int hff_diagnostics(hff_handle *h, int inst, hff_diag *out, double *l_prof);

/* Step counter, time step, counts and the tile / precision choices.
 * Synchronises the stream. */
int hff_get_info(hff_handle *h, hff_info *out);

/* The same counters read back without waiting, for a caller that keeps the
 * GPU busy: hff_info_enqueue queues a copy of the device counters on the
 * stream behind the work queued so far (into pinned host memory owned by the
 * handle) and returns a ticket; hff_info_collect(ticket) waits for that copy
 * only and fills out as hff_get_info would have at the moment of the
 * enqueue.  The last HFF_INFO_RING tickets stay collectable; an older one is
 * HFF_ERR_ARG (overwritten), and enqueueing waits for the copy the reused
 * slot held.  For an ensemble the ticket covers every member. */
#define HFF_INFO_RING 8
int hff_info_enqueue(hff_handle *h, int64_t *ticket);
int hff_info_collect(hff_handle *h, int64_t ticket, hff_info *out);

/* Read and clear the latched device status: HFF_OK, HFF_ERR_CAPACITY,
 * HFF_ERR_NONFINITE or HFF_ERR_ARG (a particle with a cell index outside the
 * grid met by a sort, and removed).  Synchronises the stream. */
int hff_status(hff_handle *h);

/* Release the handle and its CUDA graphs (not the caller's memory). */
int hff_destroy(hff_handle *h);

/* Message of the last error on this thread ("" if none). */
const char *hff_last_error(void);

/* Maps of one species for the density and energy figures of Sect. 5.2, in
 * FP64 on the host (nr x nt each, theta fastest; either may be NULL): the
 * number density sum(w) / V_cell and the kinetic energy density
 * sum(w m (gamma - 1)) / V_cell of the live particles, V_cell the exact cell
 * volume.  Synchronises the stream. */
int hff_species_maps(hff_handle *h, int inst, int species, double *density, double *energy);

/* Energy spectrum of one species (Sect. 5.2): the weights of its live
 * particles in nbins (1..4096) bins uniform in log10(gamma) over
 * [lg_min, lg_max); particles outside fall into the end bins.  out: nbins
 * doubles on the host.  Synchronises the stream. */
int hff_spectrum(hff_handle *h, int inst, int species, int nbins, double lg_min, double lg_max, double *out);

/* ---------------------------------------------------------------------------
 * Checkpoint and resume of one instance (`inst` of an ensemble), in host
 * memory.  The blob holds the configuration, the step counter, the running
 * totals, E and B - B_0, and the live particles of every species.  Taking
 * the size or saving first sorts the particles by tile (a reordering that
 * changes no physical quantity), so that a resumed run starts from exactly
 * the state the saving run continues from; the injection generator is keyed
 * by (seed, step), so both inject the same particles.  Two runs still differ
 * by the summation order of the atomic deposit (rounding only).
 *
 * hff_checkpoint_size: bytes of the blob for the current state (synchronises).
 * hff_checkpoint_save: writes the blob to dst (host, >= that size; nothing
 *   may step the instance in between).  HFF_ERR_CAPACITY if dst is too small.
 * hff_checkpoint_load: restores a blob into an instance of the same
 *   configuration (only capacity, which must hold the saved particles, and
 *   rr_scale may differ; the saved ramp scalar is restored).  HFF_ERR_ARG for
 *   a foreign, truncated or mismatched blob, HFF_ERR_CAPACITY if the
 *   particles do not fit.  Synchronises the stream. */
int hff_checkpoint_size(hff_handle *h, int inst, size_t *bytes);
int hff_checkpoint_save(hff_handle *h, int inst, void *dst, size_t bytes);
int hff_checkpoint_load(hff_handle *h, int inst, const void *src, size_t bytes);

/* ---------------------------------------------------------------------------
 * Allocation-free tile ordering.  No counterpart in the paper: this is a
 * service for callers that may not allocate device memory at all -- code
 * that runs under an external memory budget or allocator that forbids ad-hoc
 * cudaMalloc, or inside a larger application that owns every allocation.
 *
 * Computes, for n particles with cell indices `cell` (device, i * nt + j,
 * negative = removed), the stable order by tile key (tiles of tile_r x
 * tile_t cells, row-major over tiles) with removed particles last -- the
 * order in which hff_load_particles stores them.  order[k] (device, n words)
 * receives the input index of the k-th particle; *n_live (host) the number of
 * particles that are not removed.  Synchronises `stream`.
 *
 * Scratch lives in one fixed device array per GPU (about 4.3 MB), reserved in
 * every process that loads the library until it exits; nothing is allocated.
 * The first call on a device looks up that array's device address, so make
 * it before any stream capture.  Calls share the array: calls that overlap
 * on the GPU (other streams, threads) race and must be serialised by the
 * caller.
 * Returns HFF_ERR_CAPACITY if n > HFF_NOALLOC_MAX_PARTICLES, HFF_ERR_ARG for
 * invalid arguments or a cell index at or past nr * nt (such a particle is
 * ordered with the removed ones), HFF_ERR_CUDA if a CUDA call fails; the
 * message is given by hff_noalloc_last_error(). */
#define HFF_NOALLOC_MAX_PARTICLES 262144
int hff_tile_order_noalloc(const int32_t *cell, int64_t n, int32_t nr, int32_t nt, int32_t tile_r,
                           int32_t tile_t, uint32_t *order, int64_t *n_live, void *stream);
const char *hff_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
