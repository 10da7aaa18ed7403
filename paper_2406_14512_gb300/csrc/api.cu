// api.cu -- the C ABI of include/hff.h: memory plan in caller-owned device
// memory, FP64 host geometry and initial fields, the step as CUDA graphs
// (one per particle-buffer parity, plus the sort), and the read-side calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hff.h"
#include "diag.cuh"
#include "hff_common.cuh"

using namespace hff;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &m) {
  g_err = m;
  return code;
}

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) return fail(HFF_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Particles per work item of the tiled push.  A grid whose tiles already
// give the GPU enough items (tiles x species >= 4096) keeps 8192, so that
// every item amortises the staging of its tile; a small instance takes the
// largest power of two from 512 to 8192 at or below capacity / 4096, so that
// it still offers a few thousand items (blocks) to the GPU.  Members of an
// ensemble keep 8192 (the members fill the GPU together, and short items
// only re-stage their tiles).  The work list is sized for the shortest.
constexpr int kChunkMin = 512, kChunkMax = 8192;
int chunk_of(const hff_config &c) {
  const int tr = c.tile_r > 0 ? c.tile_r : 16, tt = c.tile_t > 0 ? c.tile_t : 32;
  const int64_t tiles = (int64_t)((c.nr + tr - 1) / tr) * ((c.nt + tt - 1) / tt);
  if (tiles * c.n_species >= 4096) return kChunkMax;
  int k = kChunkMin;
  while (k < kChunkMax && (int64_t)(2 * k) * 4096 <= c.capacity) k *= 2;
  return k;
}

// ------------------------------------------------------------------ geometry
// FP64 grid of Sect. 4: r log-spaced, theta uniform, geometric half nodes,
// dual cells clipped at r_min, r_max and the axis; exact-integral measures.
struct Geom {
  int nr, nt;
  double r_min, r_max, dlog, dth;
  double rn(int i) const { return r_min * std::exp(i * dlog); }
  double rh(int i) const { return r_min * std::exp((i + 0.5) * dlog); }
  double tn(int j) const { return j * dth; }
  double th(int j) const { return (j + 0.5) * dth; }
  double rlo(int i) const { return i == 0 ? r_min : rh(i - 1); }
  double rhi(int i) const { return i == nr ? r_max : rh(i); }
  double tlo(int j) const { return j == 0 ? 0.0 : th(j - 1); }
  double thi(int j) const { return j == nt ? kPi : th(j); }
  double dcp(int j) const { return std::cos(tn(j)) - std::cos(tn(j + 1)); }
  double dch(int j) const { return std::cos(tlo(j)) - std::cos(thi(j)); }
  double a_br(int i, int j) const { return 2 * kPi * rn(i) * rn(i) * dcp(j); }
  double a_bt(int i, int j) const { return kPi * std::sin(tn(j)) * (rn(i + 1) * rn(i + 1) - rn(i) * rn(i)); }
};

double courant_dt(const hff_config &c) {
  const double dlog = std::log(c.r_max / c.r_min) / c.nr, dth = kPi / c.nt;
  double best = 1e300;
  for (int i = 0; i < c.nr; ++i) {
    const double r0 = c.r_min * std::exp(i * dlog), r1 = c.r_min * std::exp((i + 1) * dlog);
    const double dr = r1 - r0, rt = r0 * dth;
    const double l = 1.0 / std::sqrt(1.0 / (dr * dr) + 1.0 / (rt * rt));
    if (l < best) best = l;
  }
  return c.courant * best;
}

double psi_unit_of(const hff_config &c) {
  if (c.geom == HFF_GEOM_MONOPOLE || c.geom == HFF_GEOM_MICHEL) return c.b_star * c.r_min * c.r_min;
  return c.b_star * c.r_min * c.r_min * c.r_min / c.r_lc;
}

// blend of Eqs. 29-31 in FP64 on the host (injection eligibility at init)
double blend_host(const hff_config &c, double unit, double psi) {
  const int n = c.n_breaks;
  if (n <= 0) return 0.0;
  if (psi < c.psi_break[0] * unit) return c.f_break[0];
  for (int k = 1; k < n; ++k) {
    const double x0 = c.psi_break[k - 1] * unit, x1 = c.psi_break[k] * unit;
    if (psi < x1) return c.f_break[k - 1] + (c.f_break[k] - c.f_break[k - 1]) * (psi - x0) / (x1 - x0);
  }
  return c.f_break[n - 1];
}

// analytic flux functions of the initial fields (Eqs. 32 and 37)
double psi_analytic(const hff_config &c, double unit, double r, double t) {
  const double mu = c.b_star * c.r_min * c.r_min * c.r_min, pst = c.b_star * c.r_min * c.r_min;
  const double sn = std::sin(t), cs = std::cos(t);
  switch (c.geom) {
    case HFF_GEOM_DIPOLE: return mu * sn * sn / r;
    case HFF_GEOM_MONOPOLE:
    case HFF_GEOM_MICHEL: return pst * (1.0 - cs);
    case HFF_GEOM_UNIFORM: return 0.5 * c.b_star * r * r * sn * sn;
    case HFF_GEOM_SYNTH: {
      const double w = 0.5 * (1.0 - std::tanh((r - c.r_lc) / (0.2 * c.r_lc)));
      return w * mu * sn * sn / r + (1.0 - w) * c.synth_psi_open * unit * (1.0 - std::fabs(cs));
    }
  }
  return 0.0;
}

int validate(const hff_config *c) {
  if (!c) return fail(HFF_ERR_ARG, "null config");
  if (c->nr < 8 || c->nt < 8) return fail(HFF_ERR_ARG, "nr and nt must be >= 8");
  if ((int64_t)(c->nr + 1) * (c->nt + 1) > (int64_t)1 << 31) return fail(HFF_ERR_ARG, "grid too large");
  if (!(c->r_min > 0 && c->r_max > c->r_min && c->r_lc > 0)) return fail(HFF_ERR_ARG, "bad radii");
  if (!(c->courant > 0 && c->courant <= 0.9)) return fail(HFF_ERR_ARG, "courant must be in (0, 0.9]");
  if (c->geom < 0 || c->geom > 4) return fail(HFF_ERR_ARG, "bad geom");
  if (c->n_breaks < 0 || c->n_breaks > 4) return fail(HFF_ERR_ARG, "n_breaks must be 0..4");
  for (int k = 1; k < c->n_breaks; ++k)
    if (c->psi_break[k] < c->psi_break[k - 1]) return fail(HFF_ERR_ARG, "psi_break must ascend");
  if (c->n_species < 1 || c->n_species > 4) return fail(HFF_ERR_ARG, "n_species must be 1..4");
  for (int s = 0; s < c->n_species; ++s)
    if (!(c->m[s] > 0)) return fail(HFF_ERR_ARG, "masses must be positive");
  if (c->capacity < 0 || c->capacity > 2000000000LL) return fail(HFF_ERR_ARG, "capacity out of range");
  if (c->sort_every < 0 || c->sort_every > 32) return fail(HFF_ERR_ARG, "sort_every must be 0..32");
  if (c->precision != HFF_FP32 && c->precision != HFF_FP64) return fail(HFF_ERR_ARG, "bad precision");
  const double dlog = std::log(c->r_max / c->r_min) / c->nr;
  const double xi_abs = std::log(c->r_abs / c->r_min) / dlog;
  if (!(c->r_abs > c->r_min) || (xi_abs > c->nr - 3 && c->r_abs < c->r_max))
    return fail(HFF_ERR_ARG, "r_abs must lie >= 3 cells inside r_max, or at or beyond r_max (no absorber)");
  if (c->tile_r < 0 || c->tile_t < 0 || c->tile_r > 64 || c->tile_t > 128)
    return fail(HFF_ERR_ARG, "tile out of range");
  if (!(c->gamma_th == 0 || c->gamma_th > 1) || (c->gamma_th > 0 && !(c->gamma_s >= 1.0)))
    return fail(HFF_ERR_ARG, "pair creation needs gamma_th = 0 (off) or > 1, and gamma_s >= 1");
  if (c->gamma_th > 0 && c->n_species < 2) return fail(HFF_ERR_ARG, "pair creation needs species 0 and 1");
  if (!(c->ff_filter >= 0.0 && c->ff_filter <= 1.0)) return fail(HFF_ERR_ARG, "ff_filter must be in [0, 1]");
  if (c->ff_delta_only < 0 || c->ff_delta_only > 2) return fail(HFF_ERR_ARG, "ff_delta_only must be 0, 1 or 2");
  if (c->ff_delta_only == 2 && c->field_pass == HFF_FIELDS_FUSED)
    return fail(HFF_ERR_ARG, "ff_delta_only = 2 runs on the separate field passes (field_pass AUTO or SPLIT)");
  if (c->field_pass != HFF_FIELDS_AUTO && c->field_pass != HFF_FIELDS_FUSED && c->field_pass != HFF_FIELDS_SPLIT)
    return fail(HFF_ERR_ARG, "field_pass must be HFF_FIELDS_AUTO, HFF_FIELDS_FUSED or HFF_FIELDS_SPLIT");
  if (c->inject_species[0] != c->inject_species[1])
    for (int k = 0; k < 2; ++k)
      if (c->inject_species[k] < 0 || c->inject_species[k] >= c->n_species)
        return fail(HFF_ERR_ARG, "inject_species must name existing species");
  return HFF_OK;
}

// The field update of a configuration: HFF_FIELDS_AUTO takes the fused pass
// when segments of 32 rows give at least one wave of its blocks (six per SM
// in FP32, three in FP64, on the 152 SMs of a GB300: a property of the grid,
// so that hff_plan needs no GPU); on smaller grids its row chains run on too
// few blocks and the separate passes, each over every row at once, are
// faster (1024^2: 1.92 against 2.00 ms per step; a 32-instance ensemble of
// grids up to 1024 x 512: 2.01 against 2.31 ms).
static bool fused_fields(const hff_config &c) {
  if (c.field_pass != HFF_FIELDS_AUTO) return c.field_pass == HFF_FIELDS_FUSED;
  if (c.ff_delta_only == 2) return false;  // the stellar-row return exists in the separate passes only
  const bool fp64 = c.precision == HFF_FP64;
  const int own = fuse_own_cols(fp64 ? sizeof(double) : sizeof(float));
  const int64_t strips = (c.nt + 1 + own - 1) / own, segs = (c.nr + 1 + 31) / 32;
  return strips * segs >= 152 * (fp64 ? 3 : 6);
}

// ----------------------------------------------------------- memory layout
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    return o;
  }
};

struct Offsets {
  size_t f[22];          // er et ep dbr dbt dbp br0 bt0 bp0 jr jt jp psi jpr jpt jpp der det dep sr st sp
  size_t ffcell;
  size_t tab_r[16];      // rn inv_rn rh inv_rh c_b2 c_bp2 c_e2 c_ep2 rho_a rho_b rh2 dep_r dep_t dep_p sig_n sig_h
  size_t tab_c[6];       // sn sh inv_sh inv_dcp inv_dch cn
  size_t r2n, dcp;       // FP64 prefix factors
  size_t dcp2;           // dcp as normalised float pairs (FP32 prefix)
  size_t dg[9];          // FP64 diag geometry: rn rh rlo rhi sn sh dch tlo thi
  size_t part[2][kMaxSpecies][7];
  size_t small;          // counters block
  size_t surf, target, inj_prefix;
  size_t keys_a, keys_b, idx_a, idx_b, hist, spart, tstart, tend;
  size_t sidx[kMaxSpecies];  // sorted order of the last sort, per species
  size_t items;
  size_t qnode, rows, psi64;
  size_t fsnap;          // halo snapshot of the fused field update
  int seg_rows;          // rows per segment of the fused field update
  size_t ev[8];          // pair-creation events: key cell xo yo ur ut up w
  size_t spec;           // spectrum bins (on request)
  int64_t ev_cap;
  int ntiles, ntt, max_items, nb, nparts;
  size_t total;
};

struct Small {  // device counters, one 256-byte block
  long long count[kMaxSpecies];
  long long count_sorted[kMaxSpecies];
  long long inj_base[kMaxSpecies];
  long long step;
  double acc[5];              // injected, killed, radiated, nonfinite, created
  unsigned pe_count;          // pair-creation events of the current step
  double rr;
  double kin[kMaxSpecies];
  double cnt[kMaxSpecies];
  unsigned long long pushed[2];
  unsigned long long clamps;
  unsigned status;
  int n_items;
  int next;
};

int tile_r_of(const hff_config &c) { return c.tile_r > 0 ? c.tile_r : 16; }
int tile_t_of(const hff_config &c) { return c.tile_t > 0 ? c.tile_t : 32; }

void layout(const hff_config &c, Offsets &o) {
  Layout L;
  const size_t R = c.precision == HFF_FP64 ? 8 : 4;
  const size_t nr = c.nr, nt = c.nt, nn = (nr + 1) * (nt + 1);
  const size_t sz[22] = {nr * (nt + 1), (nr + 1) * nt, nn, (nr + 1) * nt, nr * (nt + 1), nr * nt,
                         (nr + 1) * nt, nr * (nt + 1), nr * nt, nr * (nt + 1), (nr + 1) * nt, nn,
                         nn, nn, nn, nn, nn, nn, nn, nr * (nt + 1), (nr + 1) * nt, nn};
  // Psi (slot 12) is FP64 or a float pair: 8 bytes per node either way
  for (int k = 0; k < 22; ++k) o.f[k] = L.take(sz[k] * (k == 12 ? 8 : R));
  o.ffcell = L.take(nr * nt);
  const size_t rl[16] = {nr + 1, nr + 1, nr, nr, nr, nr, nr + 1, nr + 1, nr + 1, nr + 1, nr, nr, nr + 1, nr + 1, nr + 1, nr};
  for (int k = 0; k < 16; ++k) o.tab_r[k] = L.take(rl[k] * R);
  const size_t cl[6] = {nt + 1, nt, nt, nt, nt + 1, nt + 1};
  for (int k = 0; k < 6; ++k) o.tab_c[k] = L.take(cl[k] * R);
  o.r2n = L.take((nr + 1) * 8);
  o.dcp = L.take(nt * 8);
  o.dcp2 = L.take(nt * 8);
  const size_t dl[9] = {nr + 1, nr, nr + 1, nr + 1, nt + 1, nt, nt + 1, nt + 1, nt + 1};
  for (int k = 0; k < 9; ++k) o.dg[k] = L.take(dl[k] * 8);
  const size_t cap = (size_t)c.capacity;
  const int parities = c.sort_every > 0 ? 2 : 1;
  std::memset(o.part, 0, sizeof(o.part));
  std::memset(o.sidx, 0, sizeof(o.sidx));
  for (int p = 0; p < parities; ++p)
    for (int s = 0; s < c.n_species; ++s) {
      o.part[p][s][0] = L.take(cap * 4);
      for (int k = 1; k < 7; ++k) o.part[p][s][k] = L.take(cap * R);
    }
  o.small = L.take(sizeof(Small));
  o.surf = L.take(nt * 4);
  o.target = L.take(nt * 4);
  o.inj_prefix = L.take((nt + 1) * 4);
  const int tr = tile_r_of(c), tt = tile_t_of(c);
  o.ntt = (int)((nt + tt - 1) / tt);
  o.ntiles = (int)((nr + tr - 1) / tr) * o.ntt;
  o.nb = (int)((cap + kSortBlock - 1) / kSortBlock);
  o.nparts = (int)(((size_t)o.nb * 256 + kScanBlock - 1) / kScanBlock);
  o.max_items = c.n_species * (o.ntiles + (int)((cap + kChunkMin - 1) / kChunkMin)) + 1;
  if (c.sort_every > 0) {
    for (int s = 0; s < c.n_species; ++s) o.sidx[s] = L.take(cap * 4);
    o.keys_a = L.take(cap * 4); o.keys_b = L.take(cap * 4);
    o.idx_a = L.take(cap * 4); o.idx_b = L.take(cap * 4);
    o.hist = L.take((size_t)o.nb * 256 * 4 + 4);
    o.spart = L.take((size_t)o.nparts * 4 + 4);
    o.tstart = L.take(((size_t)o.ntiles + 1) * 4);
    o.tend = L.take(((size_t)o.ntiles + 1) * 4);
    o.items = L.take((size_t)o.max_items * sizeof(int4));
  }
  // pair-creation events of one step (bounded; overflow is latched)
  o.ev_cap = c.gamma_th > 0 ? cap / 4 + 1024 : 0;
  for (int k = 0; k < 8; ++k) o.ev[k] = o.ev_cap ? L.take((size_t)o.ev_cap * (k < 2 ? 4 : R)) : 0;
  o.spec = L.take(4096 * 8);
  o.qnode = L.take(nn * 8);
  o.rows = L.take((nr + 1) * 8 * 8);
  o.psi64 = L.take(nn * 8);
  // the fused field update's snapshot is sized for its shortest segments:
  // one wave of up to eight blocks on each of the 152 SMs of a GB300 (a
  // property of the grid, not of the device, so that hff_plan needs no GPU);
  // hff_init lengthens them to the measured occupancy
  o.seg_rows = fuse_seg_rows(c.nr, c.nt, 152 * 8, R);
  o.fsnap = fused_fields(c) ? L.take(fuse_snap_bytes(c.nr, c.nt, o.seg_rows, R)) : 0;
  o.total = (L.off + 255) & ~size_t(255);
}

}  // namespace

// ------------------------------------------------------------------ handle
constexpr int kInfoRing = HFF_INFO_RING;

struct hff_handle {
  hff_config c;
  cudaStream_t st = nullptr, cap_st = nullptr;
  char *base = nullptr;
  Offsets o;
  Geom g;
  double dt = 0, psi_unit = 0, xi_abs = 0;
  int halo = 0, push_grid = 0, tail_grid = 0;
  bool fused = false;  // the field update runs as the fused pass (fused_fields)
  int seg_rows = 0;    // rows per segment of the fused field update (>= o.seg_rows)
  Params<float> pf[2];
  Params<double> pd[2];
  WorkList wl{};
  SortScratch ss{};
  DiagGeom dg{};
  Small *small = nullptr;
  int parity = 0;
  int64_t step = 0;
  // a sort leaves the payload gather to the next push (pending): the step
  // graphs are cached per [buffer parity][pending]
  bool pending = false;
  cudaGraphExec_t g_step[2][2] = {}, g_sort[2] = {nullptr, nullptr};
  // the timed step: the same graph as g_step plus two external event-record
  // nodes around the tiled push, whose events are set per launch
  cudaGraphExec_t g_timed[2][2] = {};
  cudaGraph_t gg_timed[2][2] = {};
  cudaGraphNode_t n_evb[2][2] = {}, n_eve[2][2] = {};
  cudaEvent_t ev_ph[2] = {nullptr, nullptr};
  int64_t k_step[2][2] = {}, k_sort[2] = {0, 0}, k_timed[2][2] = {};
  int64_t launched = 0;
  // pinned host staging: per-step scalars (a ring, so queued copies never
  // see a later value) and the counter readback
  double *pin_scalar = nullptr;
  unsigned pin_next = 0;
  // one event per quarter of the scalar ring, recorded when the writes move
  // on to the next quarter: a quarter is reused only after its copies ran
  cudaEvent_t ev_scalar[4] = {};
  Small *pin_small = nullptr;
  // asynchronous counter read-back (hff_info_enqueue / hff_info_collect): a
  // ring of pinned copies, each with its event and the host-side counters of
  // the moment it was queued; allocated on first use
  Small *pin_ring = nullptr;
  cudaEvent_t ev_info[kInfoRing] = {};
  int64_t info_step[kInfoRing] = {}, info_launched[kInfoRing] = {};
  int64_t info_next = 0;
  // ensemble (n_inst > 1): the members are ordinary instances carved from
  // the caller's buffer; one graph holds every member's step as a parallel
  // branch (fork streams joined by events at capture time)
  std::vector<hff_handle *> members;
  std::vector<cudaStream_t> fork;
  std::vector<cudaEvent_t> join;
  cudaEvent_t ev_fork = nullptr;
};

constexpr unsigned kScalarRing = 1024;

namespace {

template <typename R> Params<R> *params(hff_handle *h);
template <> Params<float> *params<float>(hff_handle *h) { return h->pf; }
template <> Params<double> *params<double>(hff_handle *h) { return h->pd; }

// a breakpoint of Eqs. 29-31 in the representation of Psi
template <typename R> typename PsiOf<R>::T psi_value(double x);
template <> double psi_value<double>(double x) { return x; }
template <> float2 psi_value<float>(double x) { return psi_pair_of(x); }

template <typename R>
void fill_params(hff_handle *h) {
  const hff_config &c = h->c;
  const Offsets &o = h->o;
  char *b = h->base;
  for (int par = 0; par < 2; ++par) {
    Params<R> &p = params<R>(h)[par];
    std::memset(&p, 0, sizeof(p));
    p.nr = c.nr; p.nt = c.nt;
    p.dt = (R)h->dt; p.dlog = (R)h->g.dlog; p.dth = (R)h->g.dth; p.omega = (R)(1.0 / c.r_lc);
    p.r_min = (R)c.r_min; p.xi_abs = (R)h->xi_abs; p.shell_r2 = (R)(c.shell_r * c.shell_r);
    p.inv_dlog = (R)(1.0 / h->g.dlog); p.inv_dth = (R)(1.0 / h->g.dth);
    p.small_grid = (h->g.dlog < 0.03 && h->g.dth < 0.03) ? 1 : 0;
    p.div_nt = make_fastdiv((uint32_t)c.nt);  // cell index -> row
    p.n_breaks = c.n_breaks;
    for (int k = 0; k < kMaxBreaks; ++k) {
      const double x = c.psi_break[k] * h->psi_unit;
      p.psi_bk[k] = psi_value<R>(x);
      p.f_break[k] = (R)c.f_break[k];
      const double x0 = k > 0 ? c.psi_break[k - 1] * h->psi_unit : x;
      p.f_slope[k] = (k > 0 && x > x0) ? (R)((c.f_break[k] - c.f_break[k - 1]) / (x - x0)) : R(0);
    }
    p.n_species = c.n_species;
    for (int s = 0; s < c.n_species; ++s) {
      p.q[s] = (R)c.q[s]; p.m[s] = (R)c.m[s]; p.qm[s] = (R)(c.q[s] / c.m[s]);
      // radiation-reaction strength (Eq. 16 enters du/dt as g / (m c)):
      // (2/3) r_0^2 = |q_0| / (gamma_rad^2 b_ref) for species 0, scaled by the
      // classical radius r_s = q_s^2 / m_s of the others
      double k = 0.0;
      if (c.gamma_rad > 0) {
        const double r0c = c.q[0] * c.q[0] / c.m[0], rsc = c.q[s] * c.q[s] / c.m[s];
        const double two3 = std::fabs(c.q[0]) / (c.gamma_rad * c.gamma_rad * c.b_ref);
        k = two3 * (rsc / r0c) * (rsc / r0c) / c.m[s];
      }
      p.krr[s] = (R)k;
    }
    Tables<R> &t = p.t;
    const R **tr[16] = {&t.rn, &t.inv_rn, &t.rh, &t.inv_rh, &t.c_b2, &t.c_bp2, &t.c_e2, &t.c_ep2,
                        &t.rho_a, &t.rho_b, &t.rh2, &t.dep_r, &t.dep_t, &t.dep_p, &t.sig_n, &t.sig_h};
    for (int k = 0; k < 16; ++k) *tr[k] = reinterpret_cast<const R *>(b + o.tab_r[k]);
    const R **tc[6] = {&t.sn, &t.sh, &t.inv_sh, &t.inv_dcp, &t.inv_dch, &t.cn};
    for (int k = 0; k < 6; ++k) *tc[k] = reinterpret_cast<const R *>(b + o.tab_c[k]);
    t.r2n = reinterpret_cast<const double *>(b + o.r2n);
    t.dcp = reinterpret_cast<const double *>(b + o.dcp);
    t.dcp2 = reinterpret_cast<const float2 *>(b + o.dcp2);
    Fields<R> &f = p.f;
    R **fp[22] = {&f.er, &f.et, &f.ep, &f.br, &f.bt, &f.bp, &f.br0, &f.bt0, &f.bp0, &f.jr, &f.jt, &f.jp,
                  nullptr, &f.jpr, &f.jpt, &f.jpp, &f.der, &f.det, &f.dep, &f.sr, &f.st, &f.sp};
    for (int k = 0; k < 22; ++k)
      if (fp[k]) *fp[k] = reinterpret_cast<R *>(b + o.f[k]);
    f.psi = reinterpret_cast<typename PsiOf<R>::T *>(b + o.f[12]);
    f.ffcell = reinterpret_cast<uint8_t *>(b + o.ffcell);
    const int pp = (c.sort_every > 0) ? par : 0, po = (c.sort_every > 0) ? par ^ 1 : 0;
    for (int s = 0; s < c.n_species; ++s) {
      p.sp[s].cell = reinterpret_cast<int32_t *>(b + o.part[pp][s][0]);
      R **q[6] = {&p.sp[s].xo, &p.sp[s].yo, &p.sp[s].ur, &p.sp[s].ut, &p.sp[s].up, &p.sp[s].w};
      for (int k = 0; k < 6; ++k) *q[k] = reinterpret_cast<R *>(b + o.part[pp][s][k + 1]);
      p.src[s].cell = reinterpret_cast<int32_t *>(b + o.part[po][s][0]);
      R **r[6] = {&p.src[s].xo, &p.src[s].yo, &p.src[s].ur, &p.src[s].ut, &p.src[s].up, &p.src[s].w};
      for (int k = 0; k < 6; ++k) *r[k] = reinterpret_cast<R *>(b + o.part[po][s][k + 1]);
      p.sidx[s] = c.sort_every > 0 ? reinterpret_cast<const uint32_t *>(b + o.sidx[s]) : nullptr;
    }
    p.cap = c.capacity;
    p.count = h->small->count;
    p.count_sorted = h->small->count_sorted;
    p.rr_scale = &h->small->rr;
    p.surf = reinterpret_cast<int32_t *>(b + o.surf);
    p.target = reinterpret_cast<const int32_t *>(b + o.target);
    p.inj_prefix = reinterpret_cast<int32_t *>(b + o.inj_prefix);
    p.inj_base = h->small->inj_base;
    p.step = &h->small->step;
    p.seed_lo = (uint32_t)c.seed;
    p.seed_hi = (uint32_t)(c.seed >> 32);
    p.inject = c.inject;
    p.n_inj = c.n_species < 2 ? c.n_species : 2;
    const bool dflt = c.inject_species[0] == c.inject_species[1];
    p.inj_sp[0] = dflt ? 0 : c.inject_species[0];
    p.inj_sp[1] = dflt ? 1 : c.inject_species[1];
    // 1: the corrected node E returns (ff_delta_only 0); 0: Delta E (1);
    // 2: Delta E, the radial edges at the star taking E''(1) (2)
    p.ff_interp_e = c.ff_delta_only == 0 ? 1 : (c.ff_delta_only == 2 ? 2 : 0);
    p.ff_sigma16 = (R)(c.ff_filter / 16.0);
    p.w_inj = (R)c.w_inj;
    p.acc = h->small->acc;
    p.pushed = h->small->pushed;
    p.status = &h->small->status;
    p.clamps = &h->small->clamps;
    p.tile_r = tile_r_of(c); p.tile_t = tile_t_of(c); p.ntt = o.ntt;
    p.pairs = c.gamma_th > 0 ? 1 : 0;
    p.gamma_th2 = (R)(c.gamma_th * c.gamma_th);
    p.u_s = (R)std::sqrt(c.gamma_s > 1 ? c.gamma_s * c.gamma_s - 1.0 : 0.0);
    p.pe_count = &h->small->pe_count;
    p.pe_cap = o.ev_cap;
    if (o.ev_cap) {
      p.ev_key = reinterpret_cast<uint32_t *>(b + o.ev[0]);
      p.ev_cell = reinterpret_cast<int32_t *>(b + o.ev[1]);
      R **e[6] = {&p.ev_xo, &p.ev_yo, &p.ev_ur, &p.ev_ut, &p.ev_up, &p.ev_w};
      for (int k = 0; k < 6; ++k) *e[k] = reinterpret_cast<R *>(b + o.ev[k + 2]);
    }
  }
}

template <typename R>
int upload(hff_handle *h, size_t off, const std::vector<double> &v) {
  std::vector<R> tmp(v.begin(), v.end());
  CK(cudaMemcpyAsync(h->base + off, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}
int upload_d(hff_handle *h, size_t off, const std::vector<double> &v) {
  CK(cudaMemcpyAsync(h->base + off, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

double sigma_abs(const hff_config &c, double r) {
  if (r <= c.r_abs) return 0.0;
  const double x = (r - c.r_abs) / (c.r_max - c.r_abs);
  return c.absorb_strength * x * x * x;
}

template <typename R>
int init_state(hff_handle *h) {
  const hff_config &c = h->c;
  const Geom &g = h->g;
  const int nr = c.nr, nt = c.nt;
  const double dt = h->dt;
  int rc;
  // row tables
  std::vector<double> T[16];
  for (auto &v : T) v.clear();
  for (int i = 0; i <= nr; ++i) {
    const double lo = g.rlo(i), hi = g.rhi(i);
    T[0].push_back(g.rn(i));
    T[1].push_back(1.0 / g.rn(i));
    T[6].push_back(2.0 / (hi * hi - lo * lo));
    T[7].push_back(2.0 * (hi - lo) / ((hi * hi - lo * lo) * g.dth));
    T[8].push_back(3.0 / (4 * kPi * (hi * hi * hi - lo * lo * lo)));
    T[9].push_back(3.0 * (hi * hi - lo * lo) / (8 * kPi * (hi * hi * hi - lo * lo * lo)));
    T[12].push_back(1.0 / (kPi * (hi * hi - lo * lo) * dt));
    T[13].push_back(3.0 / (2 * kPi * (hi * hi * hi - lo * lo * lo)));
    T[14].push_back(sigma_abs(c, g.rn(i)));
  }
  for (int i = 0; i < nr; ++i) {
    const double a = g.rn(i), b = g.rn(i + 1);
    T[2].push_back(g.rh(i));
    T[3].push_back(1.0 / g.rh(i));
    T[4].push_back(2.0 / (b * b - a * a));
    T[5].push_back(2.0 * (b - a) / ((b * b - a * a) * g.dth));
    T[10].push_back(g.rh(i) * g.rh(i));
    T[11].push_back(1.0 / (2 * kPi * g.rh(i) * g.rh(i) * dt));
    T[15].push_back(sigma_abs(c, g.rh(i)));
  }
  for (int k = 0; k < 16; ++k)
    if ((rc = upload<R>(h, h->o.tab_r[k], T[k])) != HFF_OK) return rc;
  std::vector<double> C[6];
  for (int j = 0; j <= nt; ++j) {
    C[0].push_back(std::sin(g.tn(j)));
    C[4].push_back(1.0 / g.dch(j));
    C[5].push_back(std::cos(g.tn(j)));
  }
  for (int j = 0; j < nt; ++j) {
    C[1].push_back(std::sin(g.th(j)));
    C[2].push_back(1.0 / std::sin(g.th(j)));
    C[3].push_back(1.0 / g.dcp(j));
  }
  for (int k = 0; k < 6; ++k)
    if ((rc = upload<R>(h, h->o.tab_c[k], C[k])) != HFF_OK) return rc;
  std::vector<double> r2n, dcp;
  for (int i = 0; i <= nr; ++i) r2n.push_back(g.rn(i) * g.rn(i));
  for (int j = 0; j < nt; ++j) dcp.push_back(g.dcp(j));
  if ((rc = upload_d(h, h->o.r2n, r2n)) != HFF_OK) return rc;
  if ((rc = upload_d(h, h->o.dcp, dcp)) != HFF_OK) return rc;
  {  // the same factors as normalised float pairs, for the FP32 prefix
    std::vector<float2> d2(nt);
    for (int j = 0; j < nt; ++j) d2[j] = psi_pair_of(dcp[j]);
    CK(cudaMemcpyAsync(h->base + h->o.dcp2, d2.data(), d2.size() * sizeof(float2), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  {  // FP64 diagnostic geometry
    std::vector<double> D[9];
    for (int i = 0; i <= nr; ++i) { D[0].push_back(g.rn(i)); D[2].push_back(g.rlo(i)); D[3].push_back(g.rhi(i)); }
    for (int i = 0; i < nr; ++i) D[1].push_back(g.rh(i));
    for (int j = 0; j <= nt; ++j) {
      D[4].push_back(std::sin(g.tn(j))); D[6].push_back(g.dch(j));
      D[7].push_back(g.tlo(j)); D[8].push_back(g.thi(j));
    }
    for (int j = 0; j < nt; ++j) D[5].push_back(std::sin(g.th(j)));
    for (int k = 0; k < 9; ++k)
      if ((rc = upload_d(h, h->o.dg[k], D[k])) != HFF_OK) return rc;
    const double **dp[9] = {&h->dg.rn, &h->dg.rh, &h->dg.rlo, &h->dg.rhi, &h->dg.sn, &h->dg.sh, &h->dg.dch,
                            &h->dg.tlo, &h->dg.thi};
    for (int k = 0; k < 9; ++k) *dp[k] = reinterpret_cast<const double *>(h->base + h->o.dg[k]);
    h->dg.dcp = reinterpret_cast<const double *>(h->base + h->o.dcp);
    h->dg.dth = g.dth;
    int imax = (int)std::floor(h->xi_abs) - 2;
    if (imax > nr - 2) imax = nr - 2;
    h->dg.imax = imax;
  }
  // initial B from the analytic flux function by exact-area differences
  // (B = grad Psi x phi / (r sin theta)), so that div B = 0 exactly
  const double unit = h->psi_unit;
  std::vector<double> br((size_t)(nr + 1) * nt), bt((size_t)nr * (nt + 1), 0.0), bp((size_t)nr * nt, 0.0);
  std::vector<double> er((size_t)nr * (nt + 1), 0.0), et((size_t)(nr + 1) * nt, 0.0), ep((size_t)(nr + 1) * (nt + 1), 0.0);
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j)
      br[(size_t)i * nt + j] = (psi_analytic(c, unit, g.rn(i), g.tn(j + 1)) - psi_analytic(c, unit, g.rn(i), g.tn(j))) *
                               2 * kPi / g.a_br(i, j);
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nt; ++j)
      bt[(size_t)i * (nt + 1) + j] =
          -(psi_analytic(c, unit, g.rn(i + 1), g.tn(j)) - psi_analytic(c, unit, g.rn(i), g.tn(j))) * 2 * kPi / g.a_bt(i, j);
  if (c.geom == HFF_GEOM_MICHEL) {  // Eq. 33 and E_theta = B_phi
    const double pst = c.b_star * c.r_min * c.r_min;
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nt; ++j) bp[(size_t)i * nt + j] = -(pst / c.r_lc) * std::sin(g.th(j)) / g.rh(i);
    for (int i = 0; i <= nr; ++i)
      for (int j = 0; j < nt; ++j) et[(size_t)i * nt + j] = -(pst / c.r_lc) * std::sin(g.th(j)) / g.rn(i);
  }
  // corotating star and conducting outer wall (Sect. 4)
  const double omega = 1.0 / c.r_lc;
  for (int j = 0; j < nt; ++j) {
    et[j] = -omega * g.rn(0) * std::sin(g.th(j)) * br[j];
    et[(size_t)nr * nt + j] = 0.0;
  }
  // B is held as B_0 + dB: B_0 in the reference slots, dB = 0 (the buffer
  // was cleared), and curl B_0 at the E locations in FP64 from the FP64 B_0,
  // the same dual-face circulations as the Ampere kernel (Eq. 19)
  const std::vector<double> *F[6] = {&er, &et, &ep, &br, &bt, &bp};
  for (int k = 0; k < 3; ++k)
    if ((rc = upload<R>(h, h->o.f[k], *F[k])) != HFF_OK) return rc;
  for (int k = 3; k < 6; ++k)
    if ((rc = upload<R>(h, h->o.f[k + 3], *F[k])) != HFF_OK) return rc;
  {
    std::vector<double> sr((size_t)nr * (nt + 1), 0.0), st((size_t)(nr + 1) * nt, 0.0),
        sp((size_t)(nr + 1) * (nt + 1), 0.0);
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j <= nt; ++j) {
        double v = 0.0;
        if (j < nt) v += std::sin(g.th(j)) * bp[(size_t)i * nt + j];
        if (j > 0) v -= std::sin(g.th(j - 1)) * bp[(size_t)i * nt + j - 1];
        sr[(size_t)i * (nt + 1) + j] = v / (g.rh(i) * g.dch(j));
      }
    for (int i = 1; i < nr; ++i) {
      const double lo = g.rlo(i), hi = g.rhi(i);
      const double ce2 = 2.0 / (hi * hi - lo * lo), cep2 = 2.0 * (hi - lo) / ((hi * hi - lo * lo) * g.dth);
      for (int j = 0; j < nt; ++j)
        st[(size_t)i * nt + j] = -ce2 * (g.rh(i) * bp[(size_t)i * nt + j] - g.rh(i - 1) * bp[(size_t)(i - 1) * nt + j]);
      for (int j = 1; j < nt; ++j)
        sp[(size_t)i * (nt + 1) + j] =
            ce2 * (g.rh(i) * bt[(size_t)i * (nt + 1) + j] - g.rh(i - 1) * bt[(size_t)(i - 1) * (nt + 1) + j]) -
            cep2 * (br[(size_t)i * nt + j] - br[(size_t)i * nt + j - 1]);
    }
    if ((rc = upload<R>(h, h->o.f[19], sr)) != HFF_OK) return rc;
    if ((rc = upload<R>(h, h->o.f[20], st)) != HFF_OK) return rc;
    if ((rc = upload<R>(h, h->o.f[21], sp)) != HFF_OK) return rc;
  }
  // injection targets: eligibility f < 1 at the frozen stellar surface
  // (Sect. 3) and kappa n_GJ V / w with n_GJ = Omega |B_r| / (2 pi e c)
  std::vector<int32_t> tgt(nt, 0);
  {
    double pacc = 0.0;
    const double r0 = g.rn(0), r1 = g.rn(1);
    for (int j = 0; j < nt; ++j) {
      const double p0 = pacc;
      pacc += br[j] * r0 * r0 * g.dcp(j);
      const double fs = blend_host(c, unit, 0.5 * (p0 + pacc));
      if (c.inject && fs < 1.0 && c.w_inj > 0) {
        const double ngj = omega * std::fabs(br[j]) / (2 * kPi * std::fabs(c.q[0]));
        const double v = 2.0 * kPi / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0) * g.dcp(j);
        tgt[j] = (int32_t)std::floor(c.kappa_inj * ngj * v / c.w_inj + 0.5);
      }
    }
  }
  CK(cudaMemcpyAsync(h->base + h->o.target, tgt.data(), nt * 4, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

// --------------------------------------------------------- step enqueueing
// parts: 1 = up to the tiled push, 2 = the tiled push, 4 = the rest
template <typename R>
int enqueue_step(hff_handle *h, int par, int stages, cudaStream_t s, int parts = 7, bool gather = false) {
  Params<R> &p = params<R>(h)[par];
  constexpr int kFieldStages = HFF_ST_FARADAY1 | HFF_ST_AMPERE | HFF_ST_CORRECT | HFF_ST_FARADAY2;
  // the fused field update computes J_perp itself from E^n, B^n
  const bool fused = h->fused && (stages & kFieldStages) == kFieldStages;
  if ((parts & 1) && (stages & HFF_ST_NODE)) {
    launch_psi<R>(p, s);
    if (fused) launch_ffcell<R>(p, s);
    else launch_node_a<R>(p, s);
  }
  if ((parts & 1) && (stages & HFF_ST_PUSH) && h->c.sort_every > 0)
    CK(cudaMemsetAsync(&h->small->next, 0, sizeof(int), s));
  if ((parts & 1) && (stages & HFF_ST_PUSH) && h->c.gamma_th > 0)  // events of this step only
    CK(cudaMemsetAsync(&h->small->pe_count, 0, sizeof(unsigned), s));
  if ((parts & 2) && (stages & HFF_ST_PUSH) && h->c.sort_every > 0)
    launch_push_tiled<R>(p, h->wl, h->halo, s, h->push_grid, gather);
  if (!(parts & 4)) {
    CK(cudaGetLastError());
    return HFF_OK;
  }
  if (stages & HFF_ST_PUSH) launch_push_tail<R>(p, s, h->tail_grid);
  if (fused) {
    // the whole field update in one pass; J_PIC cleared for the next deposit
    launch_field_fused<R>(p, h->seg_rows, h->base + h->o.fsnap, s);
    const int64_t nr = h->c.nr, nt = h->c.nt;
    CK(cudaMemsetAsync(p.f.jr, 0, (size_t)(nr * (nt + 1)) * sizeof(R), s));
    CK(cudaMemsetAsync(p.f.jt, 0, (size_t)((nr + 1) * nt) * sizeof(R), s));
    CK(cudaMemsetAsync(p.f.jp, 0, (size_t)((nr + 1) * (nt + 1)) * sizeof(R), s));
  } else {
    if (stages & HFF_ST_FARADAY1) launch_faraday<R>(p, R(0.5), false, s);
    if (stages & HFF_ST_AMPERE) launch_ampere<R>(p, s);
    if (stages & HFF_ST_CORRECT) launch_correct<R>(p, s);
    if (stages & HFF_ST_FARADAY2) launch_faraday<R>(p, R(0.5), true, s);
  }
  if (stages & HFF_ST_INJECT) launch_inject<R>(p, s);
  else if (!(stages & HFF_ST_NOCOUNT)) launch_step_done<R>(p, s);
  CK(cudaGetLastError());
  return HFF_OK;
}

template <typename R>
int enqueue_sort(hff_handle *h, int par, cudaStream_t s, bool gather) {
  if (h->c.capacity <= 0) return HFF_OK;  // nothing to sort
  Params<R> &p = params<R>(h)[par];
  Params<R> &q = params<R>(h)[par ^ 1];
  for (int sp = 0; sp < h->c.n_species; ++sp) {
    launch_sort_species<R>(p, sp, q.sp[sp], h->ss, s, gather);
    launch_worklist<R>(p, &h->ss, h->wl, sp, sp == 0 ? 1 : 0, s);
  }
  CK(cudaGetLastError());
  return HFF_OK;
}

int count_kernels(cudaGraph_t g, int64_t *n) {
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  int64_t k = 0;
  for (auto &x : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(x, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *n = k;
  return HFF_OK;
}

template <typename F>
int capture(hff_handle *h, F &&fn, cudaGraphExec_t *out, int64_t *nk) {
  CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
  const int rc = fn(h->cap_st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
  if (rc != HFF_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(HFF_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  int r2 = count_kernels(g, nk);
  if (r2 != HFF_OK) { cudaGraphDestroy(g); return r2; }
  const cudaError_t e2 = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return fail(HFF_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e2));
  return HFF_OK;
}

// the deferred payload gather, done now (before anything reads particles)
template <typename R>
int materialize(hff_handle *h) {
  if (!h->pending) return HFF_OK;
  Params<R> &p = params<R>(h)[h->parity];
  for (int sp = 0; sp < h->c.n_species; ++sp) launch_materialize<R>(p, sp, h->st);
  CK(cudaGetLastError());
  h->pending = false;
  return HFF_OK;
}
int materialize_any(hff_handle *h) {
  return h->c.precision == HFF_FP64 ? materialize<double>(h) : materialize<float>(h);
}

// a sort with its payload gather, now (loads and stage-by-stage stepping)
template <typename R>
int run_sort_now(hff_handle *h, cudaStream_t s) {
  int rc = materialize<R>(h);
  if (rc != HFF_OK) return rc;
  rc = enqueue_sort<R>(h, h->parity, s, true);
  if (rc != HFF_OK) return rc;
  h->parity ^= 1;
  return HFF_OK;
}

// the sort at the end of a graph-replayed step: its payload moves with the
// next push
template <typename R>
int graph_sort(hff_handle *h, int par) {
  if (!h->g_sort[par]) {
    const int rc = capture(h, [&](cudaStream_t s) { return enqueue_sort<R>(h, par, s, false); }, &h->g_sort[par],
                           &h->k_sort[par]);
    if (rc != HFF_OK) return rc;
  }
  CK(cudaGraphLaunch(h->g_sort[par], h->st));
  h->launched += h->k_sort[par];
  h->parity ^= 1;
  h->pending = true;
  return HFF_OK;
}

template <typename R>
int do_step(hff_handle *h, int32_t n) {
  for (int32_t k = 0; k < n; ++k) {
    const int par = h->parity, gz = h->pending ? 1 : 0;
    if (!h->g_step[par][gz]) {
      int rc = capture(h, [&](cudaStream_t s) { return enqueue_step<R>(h, par, HFF_ST_ALL, s, 7, gz != 0); },
                       &h->g_step[par][gz], &h->k_step[par][gz]);
      if (rc != HFF_OK) return rc;
    }
    CK(cudaGraphLaunch(h->g_step[par][gz], h->st));
    h->launched += h->k_step[par][gz];
    h->pending = false;
    h->step++;
    if (h->c.sort_every > 0 && h->step % h->c.sort_every == 0) {
      const int rc = graph_sort<R>(h, par);
      if (rc != HFF_OK) return rc;
    }
  }
  return HFF_OK;
}

// The timed step graph: the kernels of g_step with an external event-record
// node before and after the tiled push (placeholder events at capture; the
// caller's events are set into the instantiated graph before each launch).
template <typename R>
int capture_timed(hff_handle *h, int par, int gz) {
  for (int e = 0; e < 2; ++e)
    if (!h->ev_ph[e]) CK(cudaEventCreateWithFlags(&h->ev_ph[e], cudaEventDisableTiming));
  CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step<R>(h, par, HFF_ST_ALL, h->cap_st, 1, gz != 0);
  if (rc == HFF_OK && cudaEventRecordWithFlags(h->ev_ph[0], h->cap_st, cudaEventRecordExternal) != cudaSuccess)
    rc = fail(HFF_ERR_CUDA, "event record node");
  if (rc == HFF_OK) rc = enqueue_step<R>(h, par, HFF_ST_ALL, h->cap_st, 2, gz != 0);
  if (rc == HFF_OK && cudaEventRecordWithFlags(h->ev_ph[1], h->cap_st, cudaEventRecordExternal) != cudaSuccess)
    rc = fail(HFF_ERR_CUDA, "event record node");
  if (rc == HFF_OK) rc = enqueue_step<R>(h, par, HFF_ST_ALL, h->cap_st, 4, gz != 0);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
  if (rc != HFF_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(HFF_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (auto &x : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(x, &t));
    if (t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev = nullptr;
    CK(cudaGraphEventRecordNodeGetEvent(x, &ev));
    if (ev == h->ev_ph[0]) h->n_evb[par][gz] = x;
    if (ev == h->ev_ph[1]) h->n_eve[par][gz] = x;
  }
  int64_t nk = 0;
  rc = count_kernels(g, &nk);
  if (rc != HFF_OK || !h->n_evb[par][gz] || !h->n_eve[par][gz]) {
    cudaGraphDestroy(g);
    return rc != HFF_OK ? rc : fail(HFF_ERR_CUDA, "event nodes not found in the timed graph");
  }
  const cudaError_t e2 = cudaGraphInstantiate(&h->g_timed[par][gz], g, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(HFF_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e2));
  }
  h->gg_timed[par][gz] = g;  // kept: its node handles address the instantiated graph
  h->k_timed[par][gz] = nk;
  return HFF_OK;
}

template <typename R>
int do_step_timed(hff_handle *h, int32_t n, void *const *evb, void *const *eve) {
  for (int32_t k = 0; k < n; ++k) {
    const int par = h->parity, gz = h->pending ? 1 : 0;
    if (!h->g_timed[par][gz]) {
      const int rc = capture_timed<R>(h, par, gz);
      if (rc != HFF_OK) return rc;
    }
    cudaEvent_t b = (evb && evb[k]) ? (cudaEvent_t)evb[k] : h->ev_ph[0];
    cudaEvent_t e = (eve && eve[k]) ? (cudaEvent_t)eve[k] : h->ev_ph[1];
    CK(cudaGraphExecEventRecordNodeSetEvent(h->g_timed[par][gz], h->n_evb[par][gz], b));
    CK(cudaGraphExecEventRecordNodeSetEvent(h->g_timed[par][gz], h->n_eve[par][gz], e));
    CK(cudaGraphLaunch(h->g_timed[par][gz], h->st));
    h->launched += h->k_timed[par][gz];
    h->pending = false;
    h->step++;
    if (h->c.sort_every > 0 && h->step % h->c.sort_every == 0) {
      const int rc = graph_sort<R>(h, par);
      if (rc != HFF_OK) return rc;
    }
  }
  return HFF_OK;
}

template <typename R>
int do_stages(hff_handle *h, int32_t n, int32_t stages) {
  int rc = materialize<R>(h);
  if (rc != HFF_OK) return rc;
  for (int32_t k = 0; k < n; ++k) {
    rc = enqueue_step<R>(h, h->parity, stages, h->st);
    if (rc != HFF_OK) return rc;
    if ((stages & HFF_ST_NOCOUNT) && !(stages & HFF_ST_INJECT)) continue;
    h->step++;
    if ((stages & HFF_ST_SORT) && h->c.sort_every > 0 && h->step % h->c.sort_every == 0) {
      rc = run_sort_now<R>(h, h->st);
      if (rc != HFF_OK) return rc;
    }
  }
  return HFF_OK;
}

// ------------------------------------------------------------ ensembles
int max_inst() { return 4096; }

int validate_all(const hff_config *cfg, int n_inst) {
  if (!cfg) return fail(HFF_ERR_ARG, "null config");
  if (n_inst < 1 || n_inst > max_inst()) return fail(HFF_ERR_ARG, "n_inst must be in [1, 4096]");
  for (int k = 0; k < n_inst; ++k) {
    const int rc = validate(&cfg[k]);
    if (rc != HFF_OK) return n_inst > 1 ? fail(rc, "instance " + std::to_string(k) + ": " + g_err) : rc;
    if (cfg[k].precision != cfg[0].precision || cfg[k].sort_every != cfg[0].sort_every)
      return fail(HFF_ERR_ARG, "the instances of an ensemble share precision and sort_every");
  }
  return HFF_OK;
}

size_t planned_bytes(const hff_config &c) {
  Offsets o;
  layout(c, o);
  return o.total;
}

bool is_ensemble(const hff_handle *h) { return !h->members.empty(); }

// the instance `inst` of a handle (a plain instance is its own instance 0)
hff_handle *member(hff_handle *h, int inst) {
  if (!h) return nullptr;
  if (!is_ensemble(h)) return inst == 0 ? h : nullptr;
  return inst >= 0 && inst < (int)h->members.size() ? h->members[inst] : nullptr;
}

// Members loaded a different number of times sit on different buffer
// parities; a sort of already-sorted particles only moves them to the other
// buffer, so it brings every member to member 0's parity without changing a
// result.  Members whose deferred gather was done early by a read are
// brought back in line by doing it for all.
template <typename R>
int ens_align(hff_handle *e) {
  const hff_handle *m0 = e->members[0];
  bool mixed = false;
  for (hff_handle *m : e->members) {
    if (m->step != m0->step) return fail(HFF_ERR_ARG, "the instances of an ensemble are at different steps");
    mixed = mixed || m->pending != m0->pending;
  }
  for (hff_handle *m : e->members) {
    int rc = mixed ? materialize<R>(m) : HFF_OK;
    if (rc == HFF_OK && m->parity != e->members[0]->parity) rc = run_sort_now<R>(m, m->st);
    if (rc != HFF_OK) return rc;
  }
  return HFF_OK;
}

template <typename R>
int ens_capture(hff_handle *e, bool sort, int par, bool gather, cudaGraphExec_t *out, int64_t *nk) {
  return capture(e, [&](cudaStream_t s) {
    CK(cudaEventRecord(e->ev_fork, s));
    for (size_t k = 0; k < e->members.size(); ++k) {
      hff_handle *m = e->members[k];
      CK(cudaStreamWaitEvent(e->fork[k], e->ev_fork, 0));
      const int rc = sort ? enqueue_sort<R>(m, par, e->fork[k], false)
                          : enqueue_step<R>(m, par, HFF_ST_ALL, e->fork[k], 7, gather);
      if (rc != HFF_OK) return rc;
      CK(cudaEventRecord(e->join[k], e->fork[k]));
      CK(cudaStreamWaitEvent(s, e->join[k], 0));
    }
    return HFF_OK;
  }, out, nk);
}

// One graph launch per ensemble step (plus one per sort step); evb / eve, if
// given, bracket each whole step.
template <typename R>
int ens_step(hff_handle *e, int32_t n, void *const *evb, void *const *eve) {
  int rc = ens_align<R>(e);
  if (rc != HFF_OK) return rc;
  const int every = e->c.sort_every;
  for (int32_t k = 0; k < n; ++k) {
    const int par = e->members[0]->parity, gz = e->members[0]->pending ? 1 : 0;
    if (!e->g_step[par][gz]) {
      rc = ens_capture<R>(e, false, par, gz != 0, &e->g_step[par][gz], &e->k_step[par][gz]);
      if (rc != HFF_OK) return rc;
    }
    if (evb && evb[k]) CK(cudaEventRecord((cudaEvent_t)evb[k], e->st));
    CK(cudaGraphLaunch(e->g_step[par][gz], e->st));
    e->launched += e->k_step[par][gz];
    for (hff_handle *m : e->members) { m->step++; m->pending = false; }
    e->step = e->members[0]->step;
    if (every > 0 && e->step % every == 0) {
      if (!e->g_sort[par]) {
        rc = ens_capture<R>(e, true, par, false, &e->g_sort[par], &e->k_sort[par]);
        if (rc != HFF_OK) return rc;
      }
      CK(cudaGraphLaunch(e->g_sort[par], e->st));
      e->launched += e->k_sort[par];
      for (hff_handle *m : e->members) { m->parity ^= 1; m->pending = true; }
      e->parity ^= 1;
    }
    if (eve && eve[k]) CK(cudaEventRecord((cudaEvent_t)eve[k], e->st));
  }
  return HFF_OK;
}

void destroy_handle(hff_handle *h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  for (int p = 0; p < 2; ++p) {
    if (h->g_sort[p]) cudaGraphExecDestroy(h->g_sort[p]);
    for (int g = 0; g < 2; ++g) {
      if (h->g_step[p][g]) cudaGraphExecDestroy(h->g_step[p][g]);
      if (h->g_timed[p][g]) cudaGraphExecDestroy(h->g_timed[p][g]);
      if (h->gg_timed[p][g]) cudaGraphDestroy(h->gg_timed[p][g]);
    }
  }
  for (int e = 0; e < 2; ++e)
    if (h->ev_ph[e]) cudaEventDestroy(h->ev_ph[e]);
  for (hff_handle *m : h->members) destroy_handle(m);
  for (cudaStream_t f : h->fork) cudaStreamDestroy(f);
  for (cudaEvent_t ev : h->join) cudaEventDestroy(ev);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->pin_scalar) cudaFreeHost(h->pin_scalar);
  if (h->pin_small) cudaFreeHost(h->pin_small);
  if (h->pin_ring) cudaFreeHost(h->pin_ring);
  for (int k = 0; k < 4; ++k)
    if (h->ev_scalar[k]) cudaEventDestroy(h->ev_scalar[k]);
  for (int k = 0; k < kInfoRing; ++k)
    if (h->ev_info[k]) cudaEventDestroy(h->ev_info[k]);
  delete h;
}

}  // namespace

// ==================================================================== ABI
extern "C" {

int hff_plan(const hff_config *cfg, int n_inst, size_t *bytes) {
  int rc = validate_all(cfg, n_inst);
  if (rc != HFF_OK) return rc;
  if (!bytes) return fail(HFF_ERR_ARG, "null bytes");
  size_t total = 0;
  for (int k = 0; k < n_inst; ++k) total += planned_bytes(cfg[k]);  // each a multiple of 256
  *bytes = total;
  return HFF_OK;
}

static int init_one(const hff_config *cfg, void *dev_mem, size_t bytes, void *stream, hff_handle **out);

int hff_init(const hff_config *cfg, int n_inst, void *dev_mem, size_t bytes, void *stream, hff_handle **out) {
  int rc = validate_all(cfg, n_inst);
  if (rc != HFF_OK) return rc;
  if (!dev_mem || !out) return fail(HFF_ERR_ARG, "null pointer");
  if (((uintptr_t)dev_mem & 255) != 0) return fail(HFF_ERR_ARG, "dev_mem must be 256-byte aligned");
  if (n_inst == 1) return init_one(cfg, dev_mem, bytes, stream, out);
  size_t need = 0;
  for (int k = 0; k < n_inst; ++k) need += planned_bytes(cfg[k]);
  if (bytes < need) return fail(HFF_ERR_CAPACITY, "dev_mem smaller than hff_plan bytes");
  hff_handle *e = new hff_handle();
  e->c = cfg[0];
  e->st = (cudaStream_t)stream;
  auto bail = [&](int code) {
    const std::string msg = g_err;
    destroy_handle(e);
    g_err = msg;
    return code;
  };
  if (cudaStreamCreateWithFlags(&e->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(HFF_ERR_CUDA, "stream or event create failed"));
  double cap_sum = 0;
  for (int k = 0; k < n_inst; ++k) cap_sum += (double)cfg[k].capacity;
  size_t off = 0;
  for (int k = 0; k < n_inst; ++k) {
    hff_handle *m = nullptr;
    const size_t b = planned_bytes(cfg[k]);
    rc = init_one(&cfg[k], (char *)dev_mem + off, b, stream, &m);
    if (rc != HFF_OK) return bail(fail(rc, "instance " + std::to_string(k) + ": " + g_err));
    m->wl.chunk = kChunkMax;  // see chunk_of
    e->members.push_back(m);
    off += b;
    cudaStream_t f = nullptr;
    cudaEvent_t j = nullptr;
    if (cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking) != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "stream create failed"));
    e->fork.push_back(f);
    if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "event create failed"));
    e->join.push_back(j);
    // the members' persistent pushes run side by side: each gets a grid in
    // proportion to its share of the particles, at least one block per SM
    if (cap_sum > 0 && m->push_grid > 0) {
      int dev = 0, nsm = 1;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      const int g = (int)std::ceil(m->push_grid * (double)cfg[k].capacity / cap_sum);
      m->push_grid = std::min(m->push_grid, std::max(nsm, g));
      m->tail_grid = std::min(m->tail_grid, std::max(nsm, (int)std::ceil(m->tail_grid * (double)cfg[k].capacity / cap_sum)));
    }
  }
  *out = e;
  return HFF_OK;
}

static int init_one(const hff_config *cfg, void *dev_mem, size_t bytes, void *stream, hff_handle **out) {
  int rc;
  hff_handle *h = new hff_handle();
  h->c = *cfg;
  h->c.tile_r = tile_r_of(*cfg);
  h->c.tile_t = tile_t_of(*cfg);
  layout(h->c, h->o);
  if (bytes < h->o.total) {
    delete h;
    return fail(HFF_ERR_CAPACITY, "dev_mem smaller than hff_plan bytes");
  }
  h->st = (cudaStream_t)stream;
  h->base = (char *)dev_mem;
  h->g = Geom{cfg->nr, cfg->nt, cfg->r_min, cfg->r_max, std::log(cfg->r_max / cfg->r_min) / cfg->nr,
              kPi / cfg->nt};
  h->dt = courant_dt(*cfg);
  h->psi_unit = psi_unit_of(*cfg);
  h->xi_abs = std::log(cfg->r_abs / cfg->r_min) / h->g.dlog;
  h->small = reinterpret_cast<Small *>(h->base + h->o.small);
  auto bail = [&](int code) {
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->pin_scalar) cudaFreeHost(h->pin_scalar);
    if (h->pin_small) cudaFreeHost(h->pin_small);
    delete h;
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(HFF_ERR_CUDA, "stream create failed"));
  if (cudaMallocHost(&h->pin_scalar, sizeof(double) * kScalarRing) != cudaSuccess ||
      cudaMallocHost(&h->pin_small, sizeof(Small)) != cudaSuccess)
    return bail(fail(HFF_ERR_CUDA, "pinned host staging failed"));
  if (cudaMemsetAsync(h->base, 0, h->o.total, h->st) != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "memset failed"));
  const int parities = cfg->sort_every > 0 ? 2 : 1;
  for (int p = 0; p < parities; ++p)
    for (int s = 0; s < cfg->n_species; ++s)
      if (cfg->capacity > 0 &&
          cudaMemsetAsync(h->base + h->o.part[p][s][0], 0xFF, (size_t)cfg->capacity * 4, h->st) != cudaSuccess)
        return bail(fail(HFF_ERR_CUDA, "memset failed"));
  {
    const double one = cfg->rr_scale;
    if (cudaMemcpyAsync(&h->small->rr, &one, sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
      return bail(fail(HFF_ERR_CUDA, "init copy failed"));
  }
  // halo of the tiled push: farthest drift between sorts (Courant-bounded)
  {
    const double dxi = -std::log(1.0 - h->dt / cfg->r_min) / h->g.dlog;
    const double deta = std::asin(std::fmin(1.0, h->dt / cfg->r_min)) / h->g.dth;
    const double d = std::fmax(dxi, deta);
    h->halo = (int)std::ceil((cfg->sort_every > 0 ? cfg->sort_every : 1) * d + 1e-9);
  }
  h->wl.items = reinterpret_cast<int4 *>(h->base + h->o.items);
  h->wl.n_items = &h->small->n_items;
  h->wl.next = &h->small->next;
  h->wl.max_items = h->o.max_items;
  h->wl.chunk = chunk_of(*cfg);
  h->ss.keys_a = reinterpret_cast<uint32_t *>(h->base + h->o.keys_a);
  h->ss.keys_b = reinterpret_cast<uint32_t *>(h->base + h->o.keys_b);
  h->ss.idx_a = reinterpret_cast<uint32_t *>(h->base + h->o.idx_a);
  h->ss.idx_b = reinterpret_cast<uint32_t *>(h->base + h->o.idx_b);
  h->ss.hist = reinterpret_cast<uint32_t *>(h->base + h->o.hist);
  h->ss.part = reinterpret_cast<uint32_t *>(h->base + h->o.spart);
  h->ss.tile_start = reinterpret_cast<int *>(h->base + h->o.tstart);
  h->ss.tile_end = reinterpret_cast<int *>(h->base + h->o.tend);
  h->ss.cap = cfg->capacity;
  h->ss.ntiles = h->o.ntiles;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  h->tail_grid = nsm * 4;
  {
    const size_t psm = cfg->precision == HFF_FP64 ? psi_smem<double>(cfg->nt) : psi_smem<float>(cfg->nt);
    const cudaError_t e = cfg->precision == HFF_FP64 ? set_psi_smem<double>(psm) : set_psi_smem<float>(psm);
    if (e != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "cannot set the flux-prefix shared memory size"));
    const cudaError_t e2 = cfg->precision == HFF_FP64 ? set_field_fused_smem<double>(field_fused_smem<double>())
                                                      : set_field_fused_smem<float>(field_fused_smem<float>());
    if (e2 != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "cannot set the fused field update's shared memory size"));
    h->fused = fused_fields(*cfg);
    // one wave of the fused field update at its occupancy on this device
    const int occ = cfg->precision == HFF_FP64 ? field_fused_blocks_per_sm<double>() : field_fused_blocks_per_sm<float>();
    h->seg_rows = std::max(h->o.seg_rows, fuse_seg_rows(cfg->nr, cfg->nt, std::max(1, occ) * nsm,
                                                         cfg->precision == HFF_FP64 ? sizeof(double) : sizeof(float)));
  }
  if (cfg->precision == HFF_FP32) {
    fill_params<float>(h);
    rc = init_state<float>(h);
    if (rc == HFF_OK && cfg->sort_every > 0) {
      const size_t smem = push_tiled_smem<float>(h->pf[0], h->halo);
      if (smem > 200 * 1024) return bail(fail(HFF_ERR_ARG, "tile + halo too large for shared memory"));
      if (set_push_smem<float>(smem) != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "cannot set shared memory size"));
      h->push_grid = nsm * std::max(1, std::min(8, push_tiled_blocks_per_sm<float>(smem)));
    }
  } else {
    fill_params<double>(h);
    rc = init_state<double>(h);
    if (rc == HFF_OK && cfg->sort_every > 0) {
      const size_t smem = push_tiled_smem<double>(h->pd[0], h->halo);
      if (smem > 200 * 1024) return bail(fail(HFF_ERR_ARG, "tile + halo too large for shared memory"));
      if (set_push_smem<double>(smem) != cudaSuccess) return bail(fail(HFF_ERR_CUDA, "cannot set shared memory size"));
      h->push_grid = nsm * std::max(1, std::min(8, push_tiled_blocks_per_sm<double>(smem)));
    }
  }
  if (rc != HFF_OK) return bail(rc);
  *out = h;
  return HFF_OK;
}

int hff_load_particles(hff_handle *h, int inst, int species, int64_t n, const int32_t *cell, const void *xo,
                       const void *yo, const void *ur, const void *ut, const void *up, const void *w, int where) {
  h = member(h, inst);
  if (!h) return fail(HFF_ERR_ARG, "bad handle or instance");
  if (species < 0 || species >= h->c.n_species) return fail(HFF_ERR_ARG, "bad species");
  if (n < 0) return fail(HFF_ERR_ARG, "negative count");
  {
    const int rc = materialize_any(h);  // the other species keep their particles
    if (rc != HFF_OK) return rc;
  }
  if (n > h->c.capacity) return fail(HFF_ERR_CAPACITY, "more particles than capacity");
  const size_t R = h->c.precision == HFF_FP64 ? 8 : 4;
  const int pp = (h->c.sort_every > 0) ? h->parity : 0;
  const cudaMemcpyKind kind = where == HFF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const void *src[7] = {cell, xo, yo, ur, ut, up, w};
  for (int k = 0; k < 7; ++k) {
    if (n > 0 && !src[k]) return fail(HFF_ERR_ARG, "null particle array");
    if (n > 0) CK(cudaMemcpyAsync(h->base + h->o.part[pp][species][k], src[k], n * (k == 0 ? 4 : R), kind, h->st));
  }
  if (h->c.capacity > n)
    CK(cudaMemsetAsync(h->base + h->o.part[pp][species][0] + n * 4, 0xFF, (h->c.capacity - n) * 4, h->st));
  // a cell index at or past nr * nt is invalid input: that particle is
  // removed (cell = -1) and the load reports HFF_ERR_ARG after completing
  launch_check_cells(reinterpret_cast<int32_t *>(h->base + h->o.part[pp][species][0]), n,
                     (int64_t)h->c.nr * h->c.nt, &h->small->status, h->st);
  const long long nn = n, zero = 0;
  CK(cudaMemcpyAsync(&h->small->count[species], &nn, sizeof(nn), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(&h->small->count_sorted[species], &zero, sizeof(zero), cudaMemcpyHostToDevice, h->st));
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, &h->small->status, sizeof(st), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (st & kStBadCell) {  // clear this bit only; other latched errors stay for hff_status
    const unsigned rest = st & ~kStBadCell;
    CK(cudaMemcpyAsync(&h->small->status, &rest, sizeof(rest), cudaMemcpyHostToDevice, h->st));
  }
  if (h->c.sort_every > 0) {
    const int rc = h->c.precision == HFF_FP64 ? run_sort_now<double>(h, h->st) : run_sort_now<float>(h, h->st);
    if (rc != HFF_OK) return rc;
  }
  CK(cudaStreamSynchronize(h->st));
  if (st & kStBadCell)
    return fail(HFF_ERR_ARG, "a particle cell index is at or past nr * nt; such particles were removed");
  return HFF_OK;
}

// dst = a + sign * (field at offset b_off), in the instance precision
static void combine_field(hff_handle *h, void *dst, const void *a, size_t b_off, int64_t n, int sign) {
  if (h->c.precision == HFF_FP64)
    launch_combine<double>((double *)dst, (const double *)a, (const double *)(h->base + b_off), n, sign, h->st);
  else
    launch_combine<float>((float *)dst, (const float *)a, (const float *)(h->base + b_off), n, sign, h->st);
}

static int64_t field_elems(const hff_handle *h, int which) {
  const int64_t nr = h->c.nr, nt = h->c.nt;
  switch (which) {
    case 0: case 6: case 16: return nr * (nt + 1);
    case 1: case 7: case 17: return (nr + 1) * nt;
    case 3: return (nr + 1) * nt;
    case 4: return nr * (nt + 1);
    case 5: case 19: return nr * nt;
    default: return (nr + 1) * (nt + 1);
  }
}

// bytes of one element of output `which` of hff_fields
static size_t field_elem_bytes(const hff_handle *h, int which) {
  if (which == 9) return 8;
  if (which == 19) return 1;
  return h->c.precision == HFF_FP64 ? 8 : 4;
}

int hff_set_field(hff_handle *h, int inst, int which, const void *src, size_t bytes, int where) {
  h = member(h, inst);
  if (!h || which < 0 || which > 8 || !src) return fail(HFF_ERR_ARG, "bad arguments");
  const size_t R = h->c.precision == HFF_FP64 ? 8 : 4;
  if (bytes != (size_t)field_elems(h, which) * R) return fail(HFF_ERR_ARG, "byte count does not match the field");
  if (which < 3 || which >= 6) {  // E, or J_PIC (offset table slots 9..11)
    const int slot = which < 3 ? which : which + 3;
    CK(cudaMemcpyAsync(h->base + h->o.f[slot], src, bytes, where == HFF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st));
  } else {  // B is held as B_0 + dB: store dB = B - B_0
    const void *b = src;
    if (where == HFF_HOST) {  // stage through the FP64 node scratch (>= any field)
      CK(cudaMemcpyAsync(h->base + h->o.psi64, src, bytes, cudaMemcpyHostToDevice, h->st));
      b = h->base + h->o.psi64;
    }
    combine_field(h, h->base + h->o.f[which], b, h->o.f[which + 3], field_elems(h, which), -1);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

int hff_fields(hff_handle *h, int inst, int which, void *dst, size_t bytes, int where) {
  h = member(h, inst);
  if (!h || which < 0 || which > 19 || !dst) return fail(HFF_ERR_ARG, "bad arguments");
  const size_t want = (size_t)field_elems(h, which) * field_elem_bytes(h, which);
  if (bytes != want) return fail(HFF_ERR_ARG, "byte count does not match the field");
  const cudaMemcpyKind kind = where == HFF_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (which >= 16) {
    // the blend weights from the current B, as the next step's node pass
    // computes them: the step's own flux prefix, then f on request, staged in
    // the FP64 node scratch (room for f at the three locations and the flags)
    const int rc = materialize_any(h);
    if (rc != HFF_OK) return rc;
    // one output at a time, staged in the FP64 node scratch (>= any of them)
    char *sc = h->base + h->o.psi64;
    void *o[4] = {nullptr, nullptr, nullptr, nullptr};
    o[which - 16] = sc;
    if (h->c.precision == HFF_FP64) {
      launch_psi<double>(h->pd[h->parity], h->st);
      launch_blend_out<double>(h->pd[h->parity], (double *)o[0], (double *)o[1], (double *)o[2], (uint8_t *)o[3],
                               h->st);
    } else {
      launch_psi<float>(h->pf[h->parity], h->st);
      launch_blend_out<float>(h->pf[h->parity], (float *)o[0], (float *)o[1], (float *)o[2], (uint8_t *)o[3],
                              h->st);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst, sc, bytes, kind, h->st));
  } else if (which == 9) {
    double *psi = reinterpret_cast<double *>(h->base + h->o.psi64);
    if (h->c.precision == HFF_FP64) launch_psi64<double>(h->pd[0], psi, h->st);
    else launch_psi64<float>(h->pf[0], psi, h->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst, psi, bytes, kind, h->st));
  } else {
    // offset table order: 0..5 fields, 6..8 initial B, 9..11 J, 12 psi,
    // 13..15 J_perp, 16..18 Delta E
    const int slot = which <= 5 ? which : which + 3;
    if (which >= 3 && which <= 5) {  // B = B_0 + dB
      void *out = where == HFF_HOST ? (void *)(h->base + h->o.psi64) : dst;
      combine_field(h, out, h->base + h->o.f[which + 3], h->o.f[which], field_elems(h, which), +1);
      CK(cudaGetLastError());
      if (where == HFF_HOST) CK(cudaMemcpyAsync(dst, out, bytes, kind, h->st));
    } else {
      CK(cudaMemcpyAsync(dst, h->base + h->o.f[slot], bytes, kind, h->st));
    }
  }
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

int hff_step(hff_handle *h, int32_t nsteps) {
  if (!h || nsteps < 0) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h))
    return h->c.precision == HFF_FP64 ? ens_step<double>(h, nsteps, nullptr, nullptr)
                                      : ens_step<float>(h, nsteps, nullptr, nullptr);
  return h->c.precision == HFF_FP64 ? do_step<double>(h, nsteps) : do_step<float>(h, nsteps);
}

int hff_step_timed(hff_handle *h, int32_t nsteps, void *const *ev_begin, void *const *ev_end) {
  if (!h || nsteps < 0) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h))
    return h->c.precision == HFF_FP64 ? ens_step<double>(h, nsteps, ev_begin, ev_end)
                                      : ens_step<float>(h, nsteps, ev_begin, ev_end);
  return h->c.precision == HFF_FP64 ? do_step_timed<double>(h, nsteps, ev_begin, ev_end)
                                    : do_step_timed<float>(h, nsteps, ev_begin, ev_end);
}

int hff_step_stages(hff_handle *h, int32_t nsteps, int32_t stages) {
  if (!h || nsteps < 0) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h)) {
    for (hff_handle *m : h->members) {
      const int rc = hff_step_stages(m, nsteps, stages);
      if (rc != HFF_OK) return rc;
    }
    h->step = h->members[0]->step;
    return HFF_OK;
  }
  return h->c.precision == HFF_FP64 ? do_stages<double>(h, nsteps, stages) : do_stages<float>(h, nsteps, stages);
}

int hff_set_scalar(hff_handle *h, int which, double value) {
  if (!h || which != HFF_SCALAR_RR_SCALE) return fail(HFF_ERR_ARG, "bad scalar");
  if (is_ensemble(h)) {
    for (hff_handle *m : h->members) {
      const int rc = hff_set_scalar(m, which, value);
      if (rc != HFF_OK) return rc;
    }
    h->c.rr_scale = value;
    return HFF_OK;
  }
  h->c.rr_scale = value;
  constexpr unsigned kQuarter = kScalarRing / 4;
  const unsigned idx = h->pin_next++ % kScalarRing;
  if (idx % kQuarter == 0) {
    const unsigned q = idx / kQuarter;
    if (!h->ev_scalar[0])
      for (int k = 0; k < 4; ++k)
        if (cudaEventCreateWithFlags(&h->ev_scalar[k], cudaEventDisableTiming) != cudaSuccess)
          return fail(HFF_ERR_CUDA, "event create failed");
    CK(cudaEventRecord(h->ev_scalar[(q + 3) % 4], h->st));  // the quarter just filled
    CK(cudaEventSynchronize(h->ev_scalar[q]));               // the quarter about to be reused
  }
  double *slot = h->pin_scalar + idx;
  *slot = value;
  CK(cudaMemcpyAsync(&h->small->rr, slot, sizeof(double), cudaMemcpyHostToDevice, h->st));
  return HFF_OK;
}

int hff_particles(hff_handle *h, int inst, int species, hff_particle_view *out) {
  h = member(h, inst);
  if (!h || species < 0 || species >= h->c.n_species || !out) return fail(HFF_ERR_ARG, "bad arguments");
  {
    const int rc = materialize_any(h);
    if (rc != HFF_OK) return rc;
  }
  long long n = 0;
  CK(cudaMemcpyAsync(&n, &h->small->count[species], sizeof(n), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int pp = (h->c.sort_every > 0) ? h->parity : 0;
  out->n = n;
  out->cell = reinterpret_cast<int32_t *>(h->base + h->o.part[pp][species][0]);
  void **q[6] = {&out->xo, &out->yo, &out->ur, &out->ut, &out->up, &out->w};
  for (int k = 0; k < 6; ++k) *q[k] = h->base + h->o.part[pp][species][k + 1];
  return HFF_OK;
}

int hff_diagnostics(hff_handle *h, int inst, hff_diag *out, double *l_prof) {
  h = member(h, inst);
  if (!h || !out) return fail(HFF_ERR_ARG, "bad arguments");
  {
    const int rc = materialize_any(h);
    if (rc != HFF_OK) return rc;
  }
  const int nr = h->c.nr, nt = h->c.nt;
  double *q = reinterpret_cast<double *>(h->base + h->o.qnode);
  double *rows = reinterpret_cast<double *>(h->base + h->o.rows);
  double *psi = reinterpret_cast<double *>(h->base + h->o.psi64);
  if (h->c.precision == HFF_FP64) {
    launch_diag<double>(h->pd[h->c.sort_every > 0 ? h->parity : 0], h->dg, q, h->small->kin, h->small->cnt, rows, h->st);
    launch_psi64<double>(h->pd[0], psi, h->st);
  } else {
    launch_diag<float>(h->pf[h->c.sort_every > 0 ? h->parity : 0], h->dg, q, h->small->kin, h->small->cnt, rows, h->st);
    launch_psi64<float>(h->pf[0], psi, h->st);
  }
  CK(cudaGetLastError());
  std::vector<double> hr((size_t)(nr + 1) * 8);
  Small sm;
  CK(cudaMemcpyAsync(hr.data(), rows, hr.size() * 8, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&sm, h->small, sizeof(Small), cudaMemcpyDeviceToHost, h->st));
  int iout = (int)std::floor(std::log(2.0 * h->c.r_lc / h->c.r_min) / h->g.dlog + 0.5);
  if (iout > nr) iout = nr;
  double po = 0;
  CK(cudaMemcpyAsync(&po, psi + (size_t)iout * (nt + 1) + nt / 2, 8, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  std::memset(out, 0, sizeof(*out));
  out->psi_open = po;
  double sin_ = 0, sout = 0, ue = 0, ub = 0, g2 = 0, gc = 0, gmax = 0, rmax = 0, bad = 0;
  int nin = 0, nout = 0;
  for (int i = 0; i <= nr; ++i) {
    const double *o = &hr[(size_t)i * 8];
    if (i < nr) {
      if (l_prof) l_prof[i] = o[0];
      const double r = h->g.rh(i);
      if (r >= h->c.r_min && r <= 2 * h->c.r_min) { sin_ += o[0]; nin++; }
      if (r >= 2 * h->c.r_lc && r <= 3 * h->c.r_lc) { sout += o[0]; nout++; }
    }
    ue += o[1]; ub += o[2]; gmax = std::fmax(gmax, o[3]); g2 += o[4]; gc += o[5]; rmax = std::fmax(rmax, o[6]);
    bad += o[7];
  }
  out->l_in = nin ? sin_ / nin : 0;
  out->l_out = nout ? sout / nout : 0;
  out->eps = out->l_out != 0 ? std::fabs(out->l_in - out->l_out) / std::fabs(out->l_out) : 0;
  out->gauss_max = gmax;
  out->gauss_rms = gc > 0 ? std::sqrt(g2 / gc) : 0;
  out->rho_max = rmax;
  out->u_e = ue / (8 * kPi);
  out->u_b = ub / (8 * kPi);
  for (int s = 0; s < kMaxSpecies; ++s) { out->kinetic[s] = sm.kin[s]; out->count[s] = sm.cnt[s]; }
  out->injected = sm.acc[0];
  out->killed = sm.acc[1];
  out->radiated = sm.acc[2];
  out->nonfinite = sm.acc[3];
  out->created = sm.acc[4];
  out->clamps = (double)sm.clamps;
  out->nonfinite_fields = bad;
  if (bad > 0) {  // latched like the device-side errors, reported by hff_status
    const unsigned bit = sm.status | kStNonfiniteField;
    CK(cudaMemcpyAsync(&h->small->status, &bit, sizeof(bit), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  return HFF_OK;
}

// the counters of one instance from a copy of its device counters and the
// host-side step and launch counts of the same moment
static void fill_info(const hff_handle *h, const Small &sm, int64_t step, int64_t launched, hff_info *out) {
  std::memset(out, 0, sizeof(*out));
  out->dt = h->dt;
  out->psi_unit = h->psi_unit;
  out->step = step;
  for (int s = 0; s < kMaxSpecies; ++s) out->count[s] = sm.count[s];
  out->tile_r = h->c.tile_r;
  out->tile_t = h->c.tile_t;
  out->sort_every = h->c.sort_every;
  out->precision = h->c.precision;
  out->kernels_per_step = h->k_step[0][0] ? h->k_step[0][0] : h->k_step[1][0];
  out->kernels_launched = launched;
  out->pushed_tiled = (int64_t)sm.pushed[0];
  out->pushed_tail = (int64_t)sm.pushed[1];
  out->readback_bytes = (int64_t)sizeof(Small);
  out->n_inst = 1;
  out->field_pass = h->fused ? HFF_FIELDS_FUSED : HFF_FIELDS_SPLIT;
}

// an ensemble's counters: the members' totals (counts, pushes, bytes read)
static void ensemble_info(const hff_handle *h, const hff_info *mi, hff_info *out) {
  hff_info sum;
  std::memset(&sum, 0, sizeof(sum));
  for (size_t k = 0; k < h->members.size(); ++k) {
    for (int s = 0; s < kMaxSpecies; ++s) sum.count[s] += mi[k].count[s];
    sum.pushed_tiled += mi[k].pushed_tiled;
    sum.pushed_tail += mi[k].pushed_tail;
    sum.readback_bytes += mi[k].readback_bytes;
    sum.n_inst += 1;
  }
  const hff_handle *m0 = h->members[0];
  sum.dt = m0->dt;
  sum.psi_unit = m0->psi_unit;
  sum.step = mi[0].step;
  sum.tile_r = m0->c.tile_r;
  sum.tile_t = m0->c.tile_t;
  sum.sort_every = h->c.sort_every;
  sum.precision = h->c.precision;
  sum.kernels_per_step = h->k_step[0][0] ? h->k_step[0][0] : h->k_step[1][0];
  sum.kernels_launched = h->launched;
  sum.field_pass = m0->fused ? HFF_FIELDS_FUSED : HFF_FIELDS_SPLIT;
  *out = sum;
}

int hff_get_info(hff_handle *h, hff_info *out) {
  if (!h || !out) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h)) {  // totals over the members
    std::vector<hff_info> mi(h->members.size());
    for (size_t k = 0; k < h->members.size(); ++k) {
      const int rc = hff_get_info(h->members[k], &mi[k]);
      if (rc != HFF_OK) return rc;
    }
    ensemble_info(h, mi.data(), out);
    return HFF_OK;
  }
  CK(cudaMemcpyAsync(h->pin_small, h->small, sizeof(Small), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  fill_info(h, *h->pin_small, h->step, h->launched, out);
  return HFF_OK;
}

int hff_info_enqueue(hff_handle *h, int64_t *ticket) {
  if (!h || !ticket) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h)) {  // every member's copy, under one ticket
    int64_t t = -1;
    for (hff_handle *m : h->members) {
      const int rc = hff_info_enqueue(m, &t);
      if (rc != HFF_OK) return rc;
    }
    *ticket = t;
    return HFF_OK;
  }
  if (!h->pin_ring) {
    if (cudaMallocHost(&h->pin_ring, sizeof(Small) * kInfoRing) != cudaSuccess) {
      h->pin_ring = nullptr;
      return fail(HFF_ERR_CUDA, "pinned host staging failed");
    }
    for (int k = 0; k < kInfoRing; ++k)
      if (cudaEventCreateWithFlags(&h->ev_info[k], cudaEventDisableTiming) != cudaSuccess)
        return fail(HFF_ERR_CUDA, "event create failed");
  }
  const int64_t t = h->info_next;
  const int slot = (int)(t % kInfoRing);
  CK(cudaEventSynchronize(h->ev_info[slot]));  // the copy this slot held last (if any) is done
  CK(cudaMemcpyAsync(h->pin_ring + slot, h->small, sizeof(Small), cudaMemcpyDeviceToHost, h->st));
  CK(cudaEventRecord(h->ev_info[slot], h->st));
  h->info_step[slot] = h->step;
  h->info_launched[slot] = h->launched;
  h->info_next = t + 1;
  *ticket = t;
  return HFF_OK;
}

int hff_info_collect(hff_handle *h, int64_t ticket, hff_info *out) {
  if (!h || !out) return fail(HFF_ERR_ARG, "bad arguments");
  if (is_ensemble(h)) {
    std::vector<hff_info> mi(h->members.size());
    for (size_t k = 0; k < h->members.size(); ++k) {
      const int rc = hff_info_collect(h->members[k], ticket, &mi[k]);
      if (rc != HFF_OK) return rc;
    }
    ensemble_info(h, mi.data(), out);
    return HFF_OK;
  }
  if (!h->pin_ring || ticket < 0 || ticket >= h->info_next || ticket < h->info_next - kInfoRing)
    return fail(HFF_ERR_ARG, "unknown or overwritten info ticket");
  const int slot = (int)(ticket % kInfoRing);
  CK(cudaEventSynchronize(h->ev_info[slot]));
  fill_info(h, h->pin_ring[slot], h->info_step[slot], h->info_launched[slot], out);
  return HFF_OK;
}

int hff_status(hff_handle *h) {
  if (!h) return fail(HFF_ERR_ARG, "null handle");
  if (is_ensemble(h)) {  // reads and clears every member; reports the first error
    int first = HFF_OK;
    std::string msg;
    for (size_t k = 0; k < h->members.size(); ++k) {
      const int rc = hff_status(h->members[k]);
      if (rc != HFF_OK && first == HFF_OK) { first = rc; msg = "instance " + std::to_string(k) + ": " + g_err; }
    }
    if (first != HFF_OK) g_err = msg;
    return first;
  }
  unsigned st = 0, zero = 0;
  CK(cudaMemcpyAsync(&st, &h->small->status, sizeof(st), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&h->small->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (st & kStCapacity) return fail(HFF_ERR_CAPACITY, "particle capacity exceeded on the device");
  if (st & kStWorklist) return fail(HFF_ERR_CAPACITY, "work list overflow");
  if (st & kStNonfinite) return fail(HFF_ERR_NONFINITE, "non-finite particle state removed");
  if (st & kStNonfiniteField) return fail(HFF_ERR_NONFINITE, "non-finite field values (seen by hff_diagnostics)");
  if (st & kStBadCell) return fail(HFF_ERR_ARG, "a particle cell index outside the grid was removed");
  return HFF_OK;
}

int hff_destroy(hff_handle *h) {
  if (!h) return fail(HFF_ERR_ARG, "null handle");
  destroy_handle(h);
  return HFF_OK;
}

// ------------------------------------------------------------ maps, spectra
int hff_species_maps(hff_handle *h, int inst, int species, double *density, double *energy) {
  h = member(h, inst);
  if (!h || species < 0 || species >= h->c.n_species) return fail(HFF_ERR_ARG, "bad arguments");
  int rc = materialize_any(h);
  if (rc != HFF_OK) return rc;
  double *d = reinterpret_cast<double *>(h->base + h->o.qnode);   // both scratch areas hold nr x nt
  double *e = reinterpret_cast<double *>(h->base + h->o.psi64);
  const int par = h->c.sort_every > 0 ? h->parity : 0;
  const double m = h->c.m[species];  // the FP64 mass of the configuration
  if (h->c.precision == HFF_FP64) launch_maps<double>(h->pd[par], h->dg, species, m, d, e, h->st);
  else launch_maps<float>(h->pf[par], h->dg, species, m, d, e, h->st);
  CK(cudaGetLastError());
  const size_t n = (size_t)h->c.nr * h->c.nt * sizeof(double);
  if (density) CK(cudaMemcpyAsync(density, d, n, cudaMemcpyDeviceToHost, h->st));
  if (energy) CK(cudaMemcpyAsync(energy, e, n, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

int hff_spectrum(hff_handle *h, int inst, int species, int nbins, double lg_min, double lg_max, double *out) {
  h = member(h, inst);
  if (!h || species < 0 || species >= h->c.n_species || !out) return fail(HFF_ERR_ARG, "bad arguments");
  if (nbins < 1 || nbins > 4096 || !(lg_max > lg_min)) return fail(HFF_ERR_ARG, "need 1 <= nbins <= 4096, lg_max > lg_min");
  int rc = materialize_any(h);
  if (rc != HFF_OK) return rc;
  double *d = reinterpret_cast<double *>(h->base + h->o.spec);
  const int par = h->c.sort_every > 0 ? h->parity : 0;
  if (h->c.precision == HFF_FP64) launch_spectrum<double>(h->pd[par], species, nbins, lg_min, lg_max, d, h->st);
  else launch_spectrum<float>(h->pf[par], species, nbins, lg_min, lg_max, d, h->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, d, (size_t)nbins * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

// ------------------------------------------------------------ checkpoints
// Blob: header, then E_r E_th E_ph dB_r dB_th dB_ph (instance precision), then
// per species its live particles: cell (int32), xo yo ur ut up w.
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  hff_config cfg;
  int64_t step;
  int64_t count[kMaxSpecies];
  double acc[5];
  double rr;
  uint64_t pushed[2];
  uint64_t payload_bytes;
};
static const char kCkptMagic[8] = {'H', 'F', 'F', 'C', 'K', 'P', 'T', '1'};

// configurations that describe the same run (capacity and the ramp scalar
// may differ); field by field, so that struct padding never matters
static bool same_run(const hff_config &a, const hff_config &b) {
  bool eq = a.nr == b.nr && a.nt == b.nt && a.r_min == b.r_min && a.r_max == b.r_max && a.r_lc == b.r_lc &&
            a.b_star == b.b_star && a.geom == b.geom && a.courant == b.courant && a.r_abs == b.r_abs &&
            a.absorb_strength == b.absorb_strength && a.n_breaks == b.n_breaks && a.n_species == b.n_species &&
            a.inject == b.inject && a.kappa_inj == b.kappa_inj && a.w_inj == b.w_inj && a.gamma_rad == b.gamma_rad &&
            a.b_ref == b.b_ref && a.shell_r == b.shell_r && a.synth_psi_open == b.synth_psi_open &&
            a.seed == b.seed && a.tile_r == b.tile_r && a.tile_t == b.tile_t && a.sort_every == b.sort_every &&
            a.precision == b.precision && a.gamma_th == b.gamma_th && a.gamma_s == b.gamma_s &&
            a.inject_species[0] == b.inject_species[0] && a.inject_species[1] == b.inject_species[1] &&
            a.ff_delta_only == b.ff_delta_only && a.ff_filter == b.ff_filter;
  for (int k = 0; k < 4; ++k)
    eq = eq && a.psi_break[k] == b.psi_break[k] && a.f_break[k] == b.f_break[k] && a.q[k] == b.q[k] && a.m[k] == b.m[k];
  return eq;
}

static size_t ckpt_payload(const hff_handle *h, const int64_t *count) {
  const size_t R = h->c.precision == HFF_FP64 ? 8 : 4;
  size_t b = 0;
  for (int k = 0; k < 6; ++k) b += (size_t)field_elems(h, k) * R;
  for (int s = 0; s < h->c.n_species; ++s) b += (size_t)count[s] * (4 + 6 * R);
  return b;
}

// Bring the instance to a sorted, gathered state (a sort of the particles
// changes their order only) and read its counters.
static int ckpt_settle(hff_handle *h, Small *sm) {
  int rc = materialize_any(h);
  if (rc == HFF_OK && h->c.sort_every > 0 && h->c.capacity > 0)
    rc = h->c.precision == HFF_FP64 ? run_sort_now<double>(h, h->st) : run_sort_now<float>(h, h->st);
  if (rc != HFF_OK) return rc;
  CK(cudaMemcpyAsync(sm, h->small, sizeof(Small), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

int hff_checkpoint_size(hff_handle *h, int inst, size_t *bytes) {
  h = member(h, inst);
  if (!h || !bytes) return fail(HFF_ERR_ARG, "bad arguments");
  Small sm;
  const int rc = ckpt_settle(h, &sm);
  if (rc != HFF_OK) return rc;
  int64_t cnt[kMaxSpecies];
  for (int s = 0; s < kMaxSpecies; ++s) cnt[s] = sm.count[s];
  *bytes = sizeof(CkptHeader) + ckpt_payload(h, cnt);
  return HFF_OK;
}

int hff_checkpoint_save(hff_handle *h, int inst, void *dst, size_t bytes) {
  h = member(h, inst);
  if (!h || !dst) return fail(HFF_ERR_ARG, "bad arguments");
  Small sm;
  int rc = ckpt_settle(h, &sm);
  if (rc != HFF_OK) return rc;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.header_bytes = sizeof(CkptHeader);
  hd.cfg = h->c;
  hd.step = h->step;
  for (int s = 0; s < kMaxSpecies; ++s) hd.count[s] = sm.count[s];
  for (int k = 0; k < 5; ++k) hd.acc[k] = sm.acc[k];
  hd.rr = sm.rr;
  hd.pushed[0] = sm.pushed[0];
  hd.pushed[1] = sm.pushed[1];
  hd.payload_bytes = ckpt_payload(h, hd.count);
  if (bytes < sizeof(hd) + hd.payload_bytes) return fail(HFF_ERR_CAPACITY, "checkpoint buffer too small");
  char *o = (char *)dst;
  std::memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  const size_t R = h->c.precision == HFF_FP64 ? 8 : 4;
  for (int k = 0; k < 6; ++k) {
    const size_t n = (size_t)field_elems(h, k) * R;
    CK(cudaMemcpyAsync(o, h->base + h->o.f[k], n, cudaMemcpyDeviceToHost, h->st));
    o += n;
  }
  const int pp = (h->c.sort_every > 0) ? h->parity : 0;
  for (int s = 0; s < h->c.n_species; ++s)
    for (int k = 0; k < 7; ++k) {
      const size_t n = (size_t)hd.count[s] * (k == 0 ? 4 : R);
      if (n) CK(cudaMemcpyAsync(o, h->base + h->o.part[pp][s][k], n, cudaMemcpyDeviceToHost, h->st));
      o += n;
    }
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

int hff_checkpoint_load(hff_handle *h, int inst, const void *src, size_t bytes) {
  h = member(h, inst);
  if (!h || !src) return fail(HFF_ERR_ARG, "bad arguments");
  if (bytes < sizeof(CkptHeader)) return fail(HFF_ERR_ARG, "not a checkpoint (too short)");
  CkptHeader hd;
  std::memcpy(&hd, src, sizeof(hd));
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != 1 || hd.header_bytes != sizeof(CkptHeader))
    return fail(HFF_ERR_ARG, "not a checkpoint of this library version");
  if (!same_run(hd.cfg, h->c))
    return fail(HFF_ERR_ARG, "checkpoint of a different configuration (only capacity and rr_scale may differ)");
  for (int s = 0; s < h->c.n_species; ++s)
    if (hd.count[s] < 0 || hd.count[s] > h->c.capacity) return fail(HFF_ERR_CAPACITY, "checkpoint exceeds capacity");
  if (hd.payload_bytes != ckpt_payload(h, hd.count) || bytes < sizeof(hd) + hd.payload_bytes)
    return fail(HFF_ERR_ARG, "checkpoint truncated");
  int rc = materialize_any(h);
  if (rc != HFF_OK) return rc;
  const char *in = (const char *)src + sizeof(hd);
  const size_t R = h->c.precision == HFF_FP64 ? 8 : 4;
  for (int k = 0; k < 6; ++k) {
    const size_t n = (size_t)field_elems(h, k) * R;
    CK(cudaMemcpyAsync(h->base + h->o.f[k], in, n, cudaMemcpyHostToDevice, h->st));
    in += n;
  }
  const int pp = (h->c.sort_every > 0) ? h->parity : 0;
  for (int s = 0; s < h->c.n_species; ++s) {
    for (int k = 0; k < 7; ++k) {
      const size_t n = (size_t)hd.count[s] * (k == 0 ? 4 : R);
      if (n) CK(cudaMemcpyAsync(h->base + h->o.part[pp][s][k], in, n, cudaMemcpyHostToDevice, h->st));
      in += n;
    }
    if (h->c.capacity > hd.count[s])
      CK(cudaMemsetAsync(h->base + h->o.part[pp][s][0] + hd.count[s] * 4, 0xFF,
                         (size_t)(h->c.capacity - hd.count[s]) * 4, h->st));
  }
  // counters: the saved state was sorted, so the sorted prefix is everything
  Small sm;
  CK(cudaMemcpyAsync(&sm, h->small, sizeof(Small), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  for (int s = 0; s < kMaxSpecies; ++s) sm.count[s] = sm.count_sorted[s] = s < h->c.n_species ? hd.count[s] : 0;
  sm.step = hd.step;
  for (int k = 0; k < 5; ++k) sm.acc[k] = hd.acc[k];
  sm.rr = hd.rr;
  sm.pushed[0] = hd.pushed[0];
  sm.pushed[1] = hd.pushed[1];
  sm.status = 0;
  sm.pe_count = 0;
  sm.clamps = 0;
  CK(cudaMemcpyAsync(h->small, &sm, sizeof(Small), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  h->step = hd.step;
  h->c.rr_scale = hd.rr;
  // rebuild the tile bounds and the work list (the sort keeps the order)
  if (h->c.sort_every > 0 && h->c.capacity > 0) {
    rc = h->c.precision == HFF_FP64 ? run_sort_now<double>(h, h->st) : run_sort_now<float>(h, h->st);
    if (rc != HFF_OK) return rc;
  }
  CK(cudaStreamSynchronize(h->st));
  return HFF_OK;
}

const char *hff_last_error(void) { return g_err.c_str(); }

}  // extern "C"
