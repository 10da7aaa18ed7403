// hff_common.cuh -- device-side data layout shared by the kernels of the
// hybrid force-free / PIC step.  All geometry is precomputed on the host in
// FP64 from the exact-integral definitions (lengths, areas and volumes of the
// log-spherical Yee mesh) and stored as separable row (r) and column (theta)
// factors in the working precision R.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace hff {

constexpr int kMaxSpecies = 4;
constexpr int kMaxBreaks = 4;
constexpr double kPi = 3.14159265358979323846;

// Raises (never lowers) the dynamic shared-memory limit of a kernel on the
// current device.  The limit is a property of the kernel, shared by every
// instance in the process, so instances with different tile sizes can live
// side by side only if no instance ever lowers it under another.
template <const void *(*Fn)()>
inline cudaError_t raise_smem_limit(size_t bytes) {
  static std::mutex mu;
  static size_t cur[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && cur[dev] >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(Fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) cur[dev] = bytes;
  return e;
}

// status bits latched on the device
constexpr unsigned kStCapacity = 1u;
constexpr unsigned kStNonfinite = 2u;
constexpr unsigned kStWorklist = 4u;
constexpr unsigned kStNonfiniteField = 8u;
constexpr unsigned kStBadCell = 16u;   // a loaded cell index outside the grid

// Psi at the nodes (Eq. 27).  FP64 in FP64 instances.  In FP32 instances a
// normalised pair of floats (value hi + lo with |lo| <= ulp(hi)/2, about 48
// significant bits) summed from exact products of the FP32 B_r and the FP64
// face factors, so that the blend decision against the breakpoints of
// Eqs. 29-31 is taken at FP64-like resolution while all arithmetic runs on
// the FP32 pipes (FP64 throughput on this GPU is a small fraction of FP32).
template <typename R> struct PsiOf { using T = double; };
template <> struct PsiOf<float> { using T = float2; };

// exact sum of two floats as a (rounded sum, error) pair (Knuth's two-sum)
__host__ __device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b, bv = s - a;
  return make_float2(s, (a - (s - bv)) + (b - bv));
}
__host__ __device__ __forceinline__ float2 psi_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float e = s.y + (a.y + b.y);
  const float h = s.x + e;  // |e| << |s.x|: fast renormalisation
  return make_float2(h, e - (h - s.x));
}
__host__ __device__ __forceinline__ double psi_add(double a, double b) { return a + b; }
// scaling by a power of two is exact
__host__ __device__ __forceinline__ float2 psi_scale(float2 a, float k) { return make_float2(a.x * k, a.y * k); }
__host__ __device__ __forceinline__ double psi_scale(double a, double k) { return a * k; }
// order of normalised pairs: lexicographic (equal values have equal pairs)
__host__ __device__ __forceinline__ bool psi_lt(float2 a, float2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }
__host__ __device__ __forceinline__ bool psi_lt(double a, double b) { return a < b; }
__host__ __device__ __forceinline__ float psi_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }
__host__ __device__ __forceinline__ double psi_diff(double a, double b) { return a - b; }
// Psi at an edge is the mean of its two nodes, at a cell the mean of four
template <typename P> __device__ __forceinline__ P psi_mean2(P a, P b) { return psi_scale(psi_add(a, b), 0.5f); }
template <typename P> __device__ __forceinline__ P psi_mean4(P a, P b, P c, P d) {
  return psi_scale(psi_add(psi_add(psi_add(a, b), c), d), 0.25f);
}
// a double as a normalised pair (about 48 bits kept)
inline float2 psi_pair_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// Division of an unsigned 32-bit integer by an invariant divisor d >= 1 with
// one multiply-high, an add and two shifts (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, the
// round-up method with an (N+1)-bit multiplier): with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n), the quotient is
// (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
  uint32_t m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((1ull << l) < (uint64_t)d) ++l;
  FastDiv q;
  q.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  q.s1 = l < 1 ? l : 1;
  q.s2 = l > 1 ? l - 1 : 0;
  return q;
}
__device__ __forceinline__ uint32_t fastdiv(const FastDiv &q, uint32_t n) {
  const uint32_t t = __umulhi(q.m, n);
  return (t + ((n - t) >> q.s1)) >> q.s2;
}

// the radix sort's blocks: kSortItems rounds of kSortThreads slots each, one
// 256-bin histogram column per block (the histogram matrix the scans pass
// over shrinks as the blocks grow), scanned in kScanBlock pieces
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortBlock = kSortThreads * kSortItems;  // 4096 slots
constexpr int kScanBlock = 4096;

template <typename R>
struct Tables {
  // rows
  const R *rn;      // nr+1  r_i
  const R *inv_rn;  // nr+1  1/r_i
  const R *rh;      // nr    r_{i+1/2}
  const R *inv_rh;  // nr    1/r_{i+1/2}
  const R *c_b2;    // nr    2/(r_{i+1}^2 - r_i^2)
  const R *c_bp2;   // nr    2 (r_{i+1} - r_i)/((r_{i+1}^2 - r_i^2) dtheta)
  const R *c_e2;    // nr+1  2/(rhi^2 - rlo^2) of the node dual cell
  const R *c_ep2;   // nr+1  2 (rhi - rlo)/((rhi^2 - rlo^2) dtheta)
  const R *rho_a;   // nr+1  3/(4 pi (rhi^3 - rlo^3))
  const R *rho_b;   // nr+1  3 (rhi^2 - rlo^2)/(8 pi (rhi^3 - rlo^3))
  const R *rh2;     // nr    r_{i+1/2}^2
  const R *dep_r;   // nr    1/(2 pi r_{i+1/2}^2 dt)
  const R *dep_t;   // nr+1  1/(pi (rhi^2 - rlo^2) dt)
  const R *dep_p;   // nr+1  3/(2 pi (rhi^3 - rlo^3))
  const R *sig_n;   // nr+1  absorber damping at r_i
  const R *sig_h;   // nr    absorber damping at r_{i+1/2}
  const double *r2n;  // nr+1  r_i^2 (Psi prefix, FP64)
  // columns
  const R *sn;      // nt+1  sin theta_j
  const R *cn;      // nt+1  cos theta_j
  const R *sh;      // nt    sin theta_{j+1/2}
  const R *inv_sh;  // nt    1/sin theta_{j+1/2}
  const R *inv_dcp; // nt    1/(cos theta_j - cos theta_{j+1})
  const R *inv_dch; // nt+1  1/(cos theta_lo - cos theta_hi) of the node dual cell
  const double *dcp;  // nt    cos theta_j - cos theta_{j+1} (Psi prefix, FP64)
  const float2 *dcp2; // nt    the same as a normalised float pair (FP32 prefix)
};

template <typename R>
struct Fields {
  R *er, *et, *ep;                  // E^n
  R *br, *bt, *bp;                  // B^n - B_0 (B^{n+1/2} - B_0 between the half steps)
  R *br0, *bt0, *bp0;               // initial field B_0 (also the absorber reference)
  R *sr, *st, *sp;                  // curl B_0 at the E locations (computed in FP64)
  R *jr, *jt, *jp;                  // J_PIC accumulators (E locations)
  typename PsiOf<R>::T *psi;        // Psi at nodes (FP64, or a float pair)
  R *jpr, *jpt, *jpp;               // J_perp at nodes
  R *der, *det, *dep;               // Delta E at nodes
  uint8_t *ffcell;                  // 1 = cell in the pure force-free domain
};

template <typename R>
struct Species {
  int32_t *cell;
  R *xo, *yo, *ur, *ut, *up, *w;
};

template <typename R>
struct Params {
  int nr, nt;
  R dt, dlog, dth, omega, r_min, xi_abs, shell_r2;
  R inv_dlog, inv_dth;
  int small_grid;           // dlog and dtheta both below the series threshold
  FastDiv div_nt;           // cell / nt by multiplication (see decode_cell)
  int n_breaks;
  typename PsiOf<R>::T psi_bk[kMaxBreaks];  // breakpoints, absolute units
  R f_break[kMaxBreaks];
  R f_slope[kMaxBreaks];    // (f_k - f_{k-1}) / (psi_k - psi_{k-1}); 0 at a jump
  int n_species;
  R q[kMaxSpecies], qm[kMaxSpecies], m[kMaxSpecies], krr[kMaxSpecies];
  Tables<R> t;
  Fields<R> f;
  Species<R> sp[kMaxSpecies];
  // the other buffer parity and the sorted order of the last sort: the first
  // push after a sort reads particle sidx[s][q] of src[s] and writes slot q
  // of sp[s] (the sort's payload gather, done by the push)
  Species<R> src[kMaxSpecies];
  const uint32_t *sidx[kMaxSpecies];
  int64_t cap;
  long long *count;         // [kMaxSpecies] slots in use (device)
  long long *count_sorted;  // [kMaxSpecies] length of the tile-sorted prefix
  const double *rr_scale;   // device scalar (ramp)
  int32_t *surf;            // [nt] live particles per surface cell after the move
  const int32_t *target;    // [nt] injection targets (fixed at init)
  int32_t *inj_prefix;      // [nt+1]
  long long *inj_base;      // [kMaxSpecies] slot of the first injected particle
  long long *step;          // device step counter (injection key)
  uint32_t seed_lo, seed_hi;
  int inject;
  int n_inj, inj_sp[2];     // species created together by the injection
  int ff_interp_e;          // 1: the corrected node E returns to the edges, 0: only Delta E
  R ff_sigma16;             // fourth-difference filter of E_r (r) and E_th (theta): sigma / 16
  R w_inj;
  double *acc;              // [4] injected, killed, radiated, nonfinite
  unsigned long long *pushed;  // [2] live particles pushed: tiled kernel, tail kernel
  unsigned *status;
  unsigned long long *clamps;  // running count of E^2 > B^2 renormalisations (Eq. 26)
  int tile_r, tile_t, ntt;  // sort tiles
  // threshold pair creation (Sect. 5.1): events recorded by the push, the
  // pairs appended after the injection
  int pairs;
  R gamma_th2, u_s;         // gamma_th^2, |u| of a created particle
  unsigned *pe_count;
  int64_t pe_cap;
  uint32_t *ev_key;         // (species << 31) | parent slot: the append order
  int32_t *ev_cell;
  R *ev_xo, *ev_yo, *ev_ur, *ev_ut, *ev_up, *ev_w;
};

// piecewise-linear blend f(Psi) of Eqs. 29-31 (right-continuous at jumps);
// the segment is chosen by comparisons at the precision of Psi
template <typename R>
__device__ __forceinline__ R blend(const Params<R> &p, typename PsiOf<R>::T psi) {
  const int n = p.n_breaks;
  if (n <= 0) return R(0);
  if (psi_lt(psi, p.psi_bk[0])) return p.f_break[0];
#pragma unroll
  for (int k = 1; k < kMaxBreaks; ++k)
    if (k < n && psi_lt(psi, p.psi_bk[k]))
      return p.f_break[k - 1] + p.f_slope[k] * (R)psi_diff(psi, p.psi_bk[k - 1]);
  return p.f_break[n - 1];
}

// f on the edges and nodes of the mesh, and the pure force-free flag of a
// cell (f of its mean-corner Psi >= 1: no particles there, Eq. 29)
template <typename R>
__device__ __forceinline__ R blend_redge(const Params<R> &p, int i, int j) {  // E_r(i+1/2, j)
  const int n1 = p.nt + 1;
  return blend(p, psi_mean2(p.f.psi[(int64_t)i * n1 + j], p.f.psi[(int64_t)(i + 1) * n1 + j]));
}
template <typename R>
__device__ __forceinline__ R blend_tedge(const Params<R> &p, int i, int j) {  // E_th(i, j+1/2)
  const int64_t k = (int64_t)i * (p.nt + 1) + j;
  return blend(p, psi_mean2(p.f.psi[k], p.f.psi[k + 1]));
}
template <typename R>
__device__ __forceinline__ R blend_node(const Params<R> &p, int i, int j) {  // E_ph(i, j)
  return blend(p, p.f.psi[(int64_t)i * (p.nt + 1) + j]);
}
template <typename R>
__device__ __forceinline__ bool ff_cell(const Params<R> &p, int i, int j) {
  const int n1 = p.nt + 1;
  const int64_t k = (int64_t)i * n1 + j;
  return blend(p, psi_mean4(p.f.psi[k], p.f.psi[k + n1], p.f.psi[k + 1], p.f.psi[k + n1 + 1])) >= R(1);
}

// cell = i * nt + j  ->  (i, j) with the division by the invariant nt done
// as a multiply-high and shifts (Granlund & Montgomery 1994, unsigned
// division by invariant integers: m = floor(2^32 (2^l - nt) / nt) + 1,
// l = ceil(log2 nt), s1 = min(l, 1), s2 = max(l - 1, 0)).
template <typename R>
__device__ __forceinline__ void decode_cell(const Params<R> &p, int c, int &i, int &j) {
  i = (int)fastdiv(p.div_nt, (uint32_t)c);
  j = c - i * p.nt;
}

// row-major helpers (theta fastest)
__device__ __forceinline__ int64_t ix(int i, int j, int ld) { return (int64_t)i * ld + j; }

// launchers (defined in fields.cu / particles.cu / sort.cu / diag.cu)
template <typename R> void launch_psi(const Params<R> &p, cudaStream_t s);
template <typename R> cudaError_t set_psi_smem(size_t bytes);
template <typename R> size_t psi_smem(int nt);  // dynamic shared memory of the flux prefix
template <typename R> void launch_node_a(const Params<R> &p, cudaStream_t s);
// the per-cell force-free flags alone (the fused field update computes J_perp)
template <typename R> void launch_ffcell(const Params<R> &p, cudaStream_t s);
template <typename R> void launch_faraday(const Params<R> &p, R half, bool absorb, cudaStream_t s);
template <typename R> void launch_ampere(const Params<R> &p, cudaStream_t s);
template <typename R> void launch_correct(const Params<R> &p, cudaStream_t s);
// f at the E_r edges, E_th edges and nodes, and the force-free cell flags,
// from the current Psi (on request)
template <typename R> void launch_blend_out(const Params<R> &p, R *fr, R *ft, R *fn, uint8_t *cells, cudaStream_t s);
// the whole field update between the push and the injection (Faraday half,
// Ampere, renormalisation, return, Faraday half with absorber) in one pass
// over row segments of seg_rows rows
template <typename R> void launch_field_fused(const Params<R> &p, int seg_rows, void *snap, cudaStream_t s);
int fuse_own_cols(size_t real);                                     // theta columns a strip owns
int fuse_seg_rows(int nr, int nt, int wave_blocks, size_t real);    // rows per segment of the launch
template <typename R> int field_fused_blocks_per_sm();              // its occupancy (0 = unknown)
size_t fuse_snap_bytes(int nr, int nt, int seg_rows, size_t real);  // its halo snapshot
template <typename R> size_t field_fused_smem();
template <typename R> cudaError_t set_field_fused_smem(size_t bytes);
// dst[k] = a[k] + sign * b[k], k < n (B <-> B - B_0 at the ABI)
template <typename R> void launch_combine(R *dst, const R *a, const R *b, int64_t n, int sign, cudaStream_t s);

struct WorkList {
  int4 *items;          // (species, tile, start, count)
  int *n_items;         // device count
  int *next;            // dynamic scheduling counter
  int max_items;
  int chunk;            // particles per item
};

template <typename R> void launch_push_tail(const Params<R> &p, cudaStream_t s, int grid);
template <typename R> void launch_push_tiled(const Params<R> &p, const WorkList &wl, int halo,
                                             cudaStream_t s, int grid, bool gather);
template <typename R> size_t push_tiled_smem(const Params<R> &p, int halo);
template <typename R> void launch_inject(const Params<R> &p, cudaStream_t s);
template <typename R> void launch_step_done(const Params<R> &p, cudaStream_t s);
template <typename R> cudaError_t set_push_smem(size_t bytes);
template <typename R> int push_tiled_blocks_per_sm(size_t bytes);

struct SortScratch {
  uint32_t *keys_a, *keys_b;   // cap
  uint32_t *idx_a, *idx_b;     // cap
  uint32_t *hist;              // 256 * max_blocks
  uint32_t *part;              // block sums of the scan
  int *tile_start;             // [ntiles + 1] first sorted slot of each tile
  int *tile_end;               // [ntiles + 1] one past its last slot
  int64_t cap;
  int ntiles;
};

// Sort one species of parity p into the other parity dst.  The sorted order
// is left in p.sidx[species]; with gather the payload moves now, otherwise
// only the count and the removed slots of dst are set and the next push moves
// the payload (launch_materialize does it eagerly).
template <typename R> void launch_sort_species(const Params<R> &p, int species, Species<R> dst,
                                               const SortScratch &ss, cudaStream_t s, bool gather);
// the deferred payload gather of a species, src -> sp by sidx (slots < count)
template <typename R> void launch_materialize(const Params<R> &p, int species, cudaStream_t s);
// loaded cells at or past ncells become removed particles; kStBadCell latched
void launch_check_cells(int32_t *cell, int64_t n, int64_t ncells, unsigned *status, cudaStream_t s);
template <typename R> void launch_worklist(const Params<R> &p, const SortScratch *ss,
                                           const WorkList &wl, int species, int first,
                                           cudaStream_t s);

}  // namespace hff
