// fields.cu -- grid kernels of the hybrid step: flux function (Eq. 27),
// force-free perpendicular current (Eq. 24, first term), Yee advance in
// Stokes form (Eqs. 18-19) with the blended current (Eq. 28), the E
// renormalisation (Eqs. 25-26), the corotating star and the absorber.
//
// Mapping: theta is the fastest index of every array, so a warp walks 32
// consecutive theta points of one r row (coalesced); blockIdx.y is the row.
// All these kernels are HBM-bound stencils: each reads its inputs once per
// step through L1/L2 (neighbour reuse hits cache) and writes its outputs once.
//
// B is held as the static initial field B_0 plus the perturbation dB, and
// the Yee update advances dB only, with curl B_0 added as a source computed
// once in FP64.  In FP32 the rounding of B then scales with |dB| instead of
// |B|: near the star of a fine grid the rounding of a stored |B| ~ 1, divided
// by a cell of 1e-3 r*, would otherwise enter E every step through the curl.
#include <algorithm>
#include <type_traits>

#include "hff_common.cuh"

namespace hff {

constexpr int kRowThreads = 128;

// ------------------------------------------------------------ Psi (Eq. 27)
// Psi(i, 0) = 0, Psi(i, j+1) = Psi(i, j) + B_r(i, j+1/2) r_i^2 dcp_j, an
// inclusive prefix along theta.  One block per r row: the row is staged
// through shared memory (coalesced in and out), each thread sums a
// contiguous chunk serially, one block-wide scan of the chunk totals gives
// the offsets, and the prefix is rounded to the working precision.  The
// staged row is padded by one word every 32 (element j at j + j/32), so that
// the threads of a warp, each walking its own contiguous chunk, hit distinct
// banks.
//
// Accumulation: FP64 for FP64 instances.  For FP32 instances every term is
// formed exactly as a float pair (B_r = B_0 + dB by two-sum, times the FP64
// face factor held as a float pair, the product by fma) and summed in a
// compensated pair (the rounding error of every addition carried in a second
// float); the prefix leaves the kernel as a normalised pair, about 48
// significant bits, at FP32 instead of FP64 throughput.
constexpr int kPsiThreads = 256;
__host__ __device__ __forceinline__ int psi_pad(int j) { return j + (j >> 5); }

struct Acc64 {
  using Term = double;
  double v;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(const Acc64 &o) { v += o.v; }
  __device__ __forceinline__ Acc64 neg() const { return {-v}; }
  __device__ __forceinline__ Acc64 shfl_up(int o) const { return {__shfl_up_sync(0xffffffffu, v, o)}; }
  __device__ __forceinline__ double times(double r2) const { return r2 * v; }
  static __device__ __forceinline__ double term(const Params<double> &p, double b0, double db, int j) {
    return (b0 + db) * p.t.dcp[j];
  }
  static __device__ __forceinline__ double zero() { return 0.0; }
};
struct Acc32x2 {
  using Term = float2;
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    const float2 s = two_sum(hi, x);
    hi = s.x;
    lo += s.y;
  }
  __device__ __forceinline__ void add(float2 t) {
    add(t.x);
    lo += t.y;
  }
  __device__ __forceinline__ void add(const Acc32x2 &o) {
    add(o.hi);
    lo += o.lo;
  }
  __device__ __forceinline__ Acc32x2 neg() const { return {-hi, -lo}; }
  __device__ __forceinline__ Acc32x2 shfl_up(int o) const {
    return {__shfl_up_sync(0xffffffffu, hi, o), __shfl_up_sync(0xffffffffu, lo, o)};
  }
  // (hi + lo) (r2h + r2l) as a normalised pair (r2 split on the host side of
  // the loop)
  __device__ __forceinline__ float2 times2(float r2h, float r2l) const {
    const float ph = hi * r2h;
    const float pe = fmaf(hi, r2h, -ph) + fmaf(hi, r2l, lo * r2h);
    const float h = ph + pe;
    return make_float2(h, pe - (h - ph));
  }
  // (b0 + db) * dcp_j: the sum exactly by two-sum, the product by fma
  static __device__ __forceinline__ float2 term(const Params<float> &p, float b0, float db, int j) {
    const float2 b = two_sum(b0, db), d = p.t.dcp2[j];
    const float ph = b.x * d.x;
    return make_float2(ph, fmaf(b.x, d.x, -ph) + fmaf(b.x, d.y, b.y * d.x));
  }
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};
template <typename R> struct PsiAccOf { using T = Acc64; };
template <> struct PsiAccOf<float> { using T = Acc32x2; };

template <typename A>
__device__ __forceinline__ typename PsiOf<double>::T psi_out(const A &a, double r2) { return a.times(r2); }
__device__ __forceinline__ float2 psi_out(const Acc32x2 &a, double r2) {
  const float r2h = (float)r2, r2l = (float)(r2 - (double)r2h);
  return a.times2(r2h, r2l);
}

template <typename R>
__global__ void __launch_bounds__(kPsiThreads) k_psi(Params<R> p) {
  using A = typename PsiAccOf<R>::T;
  using T = typename A::Term;
  using P = typename PsiOf<R>::T;
  extern __shared__ __align__(16) unsigned char psmem[];
  T *row = reinterpret_cast<T *>(psmem);  // nt + 1 terms
  __shared__ A warp_tot[kPsiThreads / 32];
  const int i = blockIdx.x, nt = p.nt, tid = threadIdx.x;
  const R *br = p.f.br + (int64_t)i * nt;
  const R *br0 = p.f.br0 + (int64_t)i * nt;
  for (int j = tid; j < nt; j += kPsiThreads) row[psi_pad(j)] = A::term(p, br0[j], br[j], j);
  __syncthreads();
  const int chunk = (nt + kPsiThreads - 1) / kPsiThreads;
  const int j0 = min(tid * chunk, nt), j1 = min(j0 + chunk, nt);
  A acc{};
  for (int j = j0; j < j1; ++j) acc.add(row[psi_pad(j)]);
  // exclusive scan of the chunk totals over the block
  const int lane = tid & 31, wid = tid >> 5;
  A x = acc;
  for (int o = 1; o < 32; o <<= 1) {
    const A y = x.shfl_up(o);
    if (lane >= o) x.add(y);
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  A run = x;
  run.add(acc.neg());
  for (int w = 0; w < wid; ++w) run.add(warp_tot[w]);
  const double r2 = p.t.r2n[i];
  // rewrite the chunk in place with the prefix (inclusive, shifted by one;
  // a term and a Psi value have the same type), then store the row coalesced
  static_assert(sizeof(T) == sizeof(P), "term and Psi share the staged row");
  for (int j = j0; j < j1; ++j) {
    run.add(row[psi_pad(j)]);
    row[psi_pad(j)] = psi_out(run, r2);  // becomes Psi(i, j+1)
  }
  __syncthreads();
  P *psi = p.f.psi + (int64_t)i * (nt + 1);
  for (int j = tid; j <= nt; j += kPsiThreads) psi[j] = (j == 0) ? P{} : row[psi_pad(j - 1)];
}

// ----------------------------------------------------------- collocation
// Arithmetic means of the staggered neighbours at node (i, j) (Sect. 3);
// interior rows only; transverse components vanish on the axis.
template <typename R>
__device__ __forceinline__ void collocate(const Params<R> &p, int i, int j, R e[3], R b[3]) {
  const int nt = p.nt, n1 = nt + 1;
  const bool axis = (j == 0 || j == nt);
  const Fields<R> &f = p.f;
  e[0] = R(0.5) * (f.er[ix(i - 1, j, n1)] + f.er[ix(i, j, n1)]);
  e[1] = axis ? R(0) : R(0.5) * (f.et[ix(i, j - 1, nt)] + f.et[ix(i, j, nt)]);
  e[2] = axis ? R(0) : f.ep[ix(i, j, n1)];
  auto br = [&](int a, int c) { const int64_t k = ix(a, c, nt); return f.br0[k] + f.br[k]; };
  auto bt = [&](int a, int c) { const int64_t k = ix(a, c, n1); return f.bt0[k] + f.bt[k]; };
  auto bp = [&](int a, int c) { const int64_t k = ix(a, c, nt); return f.bp0[k] + f.bp[k]; };
  b[0] = (j == 0) ? br(i, 0) : (j == nt) ? br(i, nt - 1) : R(0.5) * (br(i, j - 1) + br(i, j));
  b[1] = axis ? R(0) : R(0.5) * (bt(i - 1, j) + bt(i, j));
  b[2] = axis ? R(0) : R(0.25) * (bp(i - 1, j - 1) + bp(i - 1, j) + bp(i, j - 1) + bp(i, j));
}

template <typename R> __device__ __forceinline__ R b2min();
template <> __device__ __forceinline__ float b2min<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double b2min<double>() { return 1e-30; }

// ----------------------------------------------------------- node pass A
// rho = div E / 4 pi over the node dual cell and J_perp = c rho E x B / B^2
// (first term of Eq. 24) from E^n, B^n; plus the per-cell pure force-free
// flag f(Psi_cell) >= 1 used to remove particles (Eq. 29: no particles).
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_node_a(Params<R> p) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  const Fields<R> &f = p.f;
  if (i < nr && j < nt) f.ffcell[ix(i, j, nt)] = ff_cell(p, i, j) ? 1 : 0;
  R jx = 0, jy = 0, jz = 0;
  if (i >= 1 && i < nr) {
    R e[3], b[3];
    collocate(p, i, j, e, b);
    R div = p.t.rho_a[i] * (p.t.rh2[i] * f.er[ix(i, j, n1)] - p.t.rh2[i - 1] * f.er[ix(i - 1, j, n1)]);
    R dt = 0;
    if (j < nt) dt += p.t.sh[j] * f.et[ix(i, j, nt)];
    if (j > 0) dt -= p.t.sh[j - 1] * f.et[ix(i, j - 1, nt)];
    const R rho = div + p.t.rho_b[i] * dt * p.t.inv_dch[j];
    const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (b2 > b2min<R>()) {
      const R s = rho / b2;
      jx = s * (e[1] * b[2] - e[2] * b[1]);
      jy = s * (e[2] * b[0] - e[0] * b[2]);
      jz = s * (e[0] * b[1] - e[1] * b[0]);
    }
  }
  f.jpr[ix(i, j, n1)] = jx;
  f.jpt[ix(i, j, n1)] = jy;
  f.jpp[ix(i, j, n1)] = jz;
}

// ---------------------------------------------------------------- Faraday
// Eq. 18 over the exact primary faces, dB -= h dt curl E; optionally the
// absorber B -= sigma (B - B_0), i.e. dB -= sigma dB, afterwards.
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_faraday(Params<R> p, R hdt, bool absorb) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  const Fields<R> &f = p.f;
  const Tables<R> &t = p.t;
  if (j < nt) {  // B_r(i, j+1/2), i = 0..nr
    const R c = t.inv_rn[i] * (t.sn[j + 1] * f.ep[ix(i, j + 1, n1)] - t.sn[j] * f.ep[ix(i, j, n1)]) *
                t.inv_dcp[j];
    R v = f.br[ix(i, j, nt)] - hdt * c;
    if (absorb) { const R sg = t.sig_n[i]; if (sg > R(0)) v -= sg * v; }
    f.br[ix(i, j, nt)] = v;
  }
  if (i < nr) {
    // B_th(i+1/2, j): zero on the axis
    R v = R(0);
    if (j > 0 && j < nt) {
      v = f.bt[ix(i, j, n1)] +
          hdt * t.c_b2[i] * (t.rn[i + 1] * f.ep[ix(i + 1, j, n1)] - t.rn[i] * f.ep[ix(i, j, n1)]);
      if (absorb) { const R sg = t.sig_h[i]; if (sg > R(0)) v -= sg * v; }
    }
    f.bt[ix(i, j, n1)] = v;
    if (j < nt) {  // B_ph(i+1/2, j+1/2)
      const R c = t.c_b2[i] * (t.rn[i + 1] * f.et[ix(i + 1, j, nt)] - t.rn[i] * f.et[ix(i, j, nt)]) -
                  t.c_bp2[i] * (f.er[ix(i, j + 1, n1)] - f.er[ix(i, j, n1)]);
      R w = f.bp[ix(i, j, nt)] - hdt * c;
      if (absorb) { const R sg = t.sig_h[i]; if (sg > R(0)) w -= sg * w; }
      f.bp[ix(i, j, nt)] = w;
    }
  }
}

// mean of a node quantity over the two nodes of a radial edge (interior
// nodes only: rows 0 and nr carry the boundary conditions)
template <typename R>
__device__ __forceinline__ R edge_r_mean(const R *a, int i, int j, int nr, int n1) {
  const bool lo = i >= 1, hi = i + 1 <= nr - 1;
  R v = R(0);
  if (lo) v += a[ix(i, j, n1)];
  if (hi) v += a[ix(i + 1, j, n1)];
  return (lo && hi) ? R(0.5) * v : v;
}

// ---------------------------------------------------------------- Ampere
// Eq. 19 over the exact dual faces, curl B = curl dB + curl B_0, with
// J = (1 - f) J_PIC + f J_FFE (Eq. 28);
// then the corotating star (tangential E fixed, Sect. 4), the conducting
// outer wall, E_ph = 0 on the axis, the absorber on E, and J_PIC cleared.
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_ampere(Params<R> p) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  const Fields<R> &f = p.f;
  const Tables<R> &t = p.t;
  const R dt = p.dt, fp = R(4.0 * kPi) * p.dt;
  if (i < nr) {  // E_r(i+1/2, j)
    R c = R(0);
    if (j < nt) c += t.sh[j] * f.bp[ix(i, j, nt)];
    if (j > 0) c -= t.sh[j - 1] * f.bp[ix(i, j - 1, nt)];
    c *= t.inv_rh[i] * t.inv_dch[j];
    const R fb = blend_redge(p, i, j);
    const int64_t k = ix(i, j, n1);
    const R jt = (R(1) - fb) * f.jr[k] + fb * edge_r_mean(f.jpr, i, j, nr, n1);
    f.er[k] = (f.er[k] + dt * (c + f.sr[k]) - fp * jt) * (R(1) - t.sig_h[i]);
    f.jr[k] = R(0);
  }
  if (j < nt) {  // E_th(i, j+1/2)
    const int64_t k = ix(i, j, nt);
    R v;
    if (i == 0) {
      v = -p.omega * t.rn[0] * t.sh[j] * (f.br0[ix(0, j, nt)] + f.br[ix(0, j, nt)]);
    } else if (i == nr) {
      v = R(0);
    } else {
      const R c = -t.c_e2[i] * (t.rh[i] * f.bp[ix(i, j, nt)] - t.rh[i - 1] * f.bp[ix(i - 1, j, nt)]);
      const R fb = blend_tedge(p, i, j);
      const R jt = (R(1) - fb) * f.jt[k] + fb * R(0.5) * (f.jpt[ix(i, j, n1)] + f.jpt[ix(i, j + 1, n1)]);
      v = (f.et[k] + dt * (c + f.st[k]) - fp * jt) * (R(1) - t.sig_n[i]);
    }
    f.et[k] = v;
    f.jt[k] = R(0);
  }
  {  // E_ph(i, j)
    const int64_t k = ix(i, j, n1);
    R v = R(0);
    if (i >= 1 && i < nr && j >= 1 && j < nt) {
      const R c = t.c_e2[i] * (t.rh[i] * f.bt[ix(i, j, n1)] - t.rh[i - 1] * f.bt[ix(i - 1, j, n1)]) -
                  t.c_ep2[i] * (f.br[ix(i, j, nt)] - f.br[ix(i, j - 1, nt)]);
      const R fb = blend_node(p, i, j);
      const R jt = (R(1) - fb) * f.jp[k] + fb * f.jpp[k];
      v = (f.ep[k] + dt * (c + f.sp[k]) - fp * jt) * (R(1) - t.sig_n[i]);
    }
    f.ep[k] = v;
    f.jp[k] = R(0);
  }
}

// ----------------------------------------------------------- node pass B
// Renormalisation at interior nodes from E^{n+1} and B^{n+1/2}:
// E' = E - (E.B) B/B^2 (Eq. 25), E'' = sqrt(B^2/E'^2) E' if E'^2 > B^2 (Eq. 26).
// Stores Delta E = E'' - E, or E'' itself when the corrected field returns to
// the edges (ff_interp_e = 1; 0 and 2 return the corrections, see
// k_correct).  With the optional fourth-difference filter it also
// stores sigma/16 D4 E_r (along r) at the E_r edge (i+1/2, j) and sigma/16
// D4 E_th (along theta) at the E_th edge (i, j+1/2), from the same
// uncorrected E, in the J_PIC arrays: those are zero between Ampere's law and
// the next deposit, and the correction reads and clears them.
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_node_b(Params<R> p) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  if (p.ff_sigma16 != R(0)) {
    const Fields<R> &f = p.f;
    if (i >= 2 && i <= nr - 3) {
      const R d4 = f.er[ix(i - 2, j, n1)] - R(4) * f.er[ix(i - 1, j, n1)] + R(6) * f.er[ix(i, j, n1)] -
                   R(4) * f.er[ix(i + 1, j, n1)] + f.er[ix(i + 2, j, n1)];
      f.jr[ix(i, j, n1)] = p.ff_sigma16 * d4;
    }
    if (i >= 1 && i <= nr - 1 && j >= 2 && j <= nt - 3) {
      const R d4 = f.et[ix(i, j - 2, nt)] - R(4) * f.et[ix(i, j - 1, nt)] + R(6) * f.et[ix(i, j, nt)] -
                   R(4) * f.et[ix(i, j + 1, nt)] + f.et[ix(i, j + 2, nt)];
      f.jt[ix(i, j, nt)] = p.ff_sigma16 * d4;
    }
  }
  R d0 = 0, d1 = 0, d2 = 0;
  bool clamped = false;
  if (i >= 1 && i < nr) {
    R e[3], b[3];
    collocate(p, i, j, e, b);
    // the stellar-row return needs row 1's collocated E_r before any edge
    // moves: kept in the (zero) J_PIC slot of the radial edge (0, j)
    if (i == 1 && p.ff_interp_e == 2) p.f.jr[ix(0, j, n1)] = e[0];
    const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (b2 > b2min<R>()) {
      const R s = (e[0] * b[0] + e[1] * b[1] + e[2] * b[2]) / b2;
      const R x = e[0] - s * b[0], y = e[1] - s * b[1], z = e[2] - s * b[2];
      const R e2 = x * x + y * y + z * z;
      const R sc = (e2 > b2) ? sqrt(b2 / e2) : R(1);
      d0 = sc * x - e[0];
      d1 = sc * y - e[1];
      d2 = sc * z - e[2];
      clamped = e2 > b2;
    }
    if (p.ff_interp_e == 1) { d0 += e[0]; d1 += e[1]; d2 += e[2]; }
  }
  // running count of Eq. 26 activations (failure detection: a force-free
  // region that keeps needing the clamp is going unstable)
  const unsigned act = __activemask(), m = __ballot_sync(act, clamped);
  if (m && (threadIdx.x & 31) == (unsigned)(__ffs(act) - 1)) atomicAdd(p.clamps, (unsigned long long)__popc(m));
  p.f.der[ix(i, j, n1)] = d0;
  p.f.det[ix(i, j, n1)] = d1;
  p.f.dep[ix(i, j, n1)] = d2;
}

// Delta E interpolated back to the staggered mesh by arithmetic means and
// applied with the blend weight f (Sect. 3, Eqs. 29-31); or, with
// ff_interp_e = 1, the corrected node field itself: E <- E + f (<E''> - E);
// with ff_interp_e = 2, Delta E everywhere except the radial edges at the
// star, which take E''(1) (their only interior node).
// The optional filter term (node pass B, in the J_PIC arrays) is subtracted
// with the same weight and its slot cleared for the next deposit.
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_correct(Params<R> p) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  const Fields<R> &f = p.f;
  const bool lit = p.ff_interp_e == 1;
  const bool filt = p.ff_sigma16 != R(0);
  if (i < nr) {
    const int64_t k = ix(i, j, n1);
    const R fb = blend_redge(p, i, j);
    // ff_interp_e = 2: the radial edge at the star (one interior node, row 1)
    // takes the corrected node field E''(1) = Delta E(1) + collocated E(1)
    const bool star = p.ff_interp_e == 2 && i == 0 && nr > 1;
    R g = R(0), e1 = R(0);
    if (star) { e1 = f.jr[k]; f.jr[k] = R(0); }
    else if (filt) { g = f.jr[k]; f.jr[k] = R(0); }
    if (fb != R(0)) {
      const R m = edge_r_mean(f.der, i, j, nr, n1) - g + e1;
      f.er[k] += fb * ((lit || star) ? m - f.er[k] : m);
    }
  }
  if (i >= 1 && i < nr) {
    if (j < nt) {
      const int64_t k = ix(i, j, nt);
      const R fb = blend_tedge(p, i, j);
      R g = R(0);
      if (filt) { g = f.jt[k]; f.jt[k] = R(0); }
      if (fb != R(0)) {
        const R m = R(0.5) * (f.det[ix(i, j, n1)] + f.det[ix(i, j + 1, n1)]) - g;
        f.et[k] += fb * (lit ? m - f.et[k] : m);
      }
    }
    if (j >= 1 && j < nt) {
      const R fb = blend_node(p, i, j);
      if (fb != R(0)) {
        const int64_t k = ix(i, j, n1);
        const R m = f.dep[k];
        f.ep[k] += fb * (lit ? m - f.ep[k] : m);
      }
    }
  }
}

// ------------------------------------------------------- fused field update
// The field update between the push and the injection -- J_perp at the
// nodes from E^n, B^n (first term of Eq. 24), Faraday's first half step
// (Eq. 18), Ampere's law with the blended current (Eqs. 19, 28) and the
// boundaries, the renormalisation at the nodes (Eqs. 25-26), the return to
// the edges with the blend weights, and Faraday's second half step with the
// absorber -- as one pass.  A block owns a strip of theta columns (with
// kFuseHalo columns recomputed on each side) and a segment of rows (with
// kFuseWarm rows of warm-up below it), and walks the rows upward.  Row step
// k has four phases separated by barriers:
//   0: F2, dB^{n+1} at node row k-4 (B_r) and half row k-5 (B_th, B_ph);
//      node row k and half row k (k+1/2) of E^n, dB^n, B_0, Psi and the
//      radial tables, loaded one step earlier, go to shared-memory rings,
//      and the loads of row k+1 are issued (they complete behind phases
//      1-3);
//   1: F1, B^{n+1/2} at node row k (B_r) and half row k-1 (B_th, B_ph), and
//      J_perp at node row k;
//   2: A, E^{n+1} at half row k-1 (E_r) and node row k-1 (E_th, E_ph), with
//      the blend weights f kept in registers for phase 3 two steps later;
//      N, Delta E (or E'') at node row k-2, and the filter terms;
//   3: C, the corrected E at half row k-3 and node row k-3.
// Every stage reads only what earlier phases produced, so E^n and dB^n are
// read once and every output written once; the arithmetic is that of
// k_node_a, k_faraday, k_ampere, k_node_b and k_correct, location by
// location.  Column and row ranges: F2 needs the corrected E at columns c,
// c+1; C (with the theta filter) the uncorrected E at c-2 .. c+2 and Delta E
// at c, c+1; N and A one column to the left, F1 and J_perp one more on
// either side, so three columns of halo suffice on each side, and likewise
// three rows of warm-up (C's radial filter reaches two rows down, A and F1
// one more each).
//
// The update is in place, and a block's halo columns and warm-up / trailing
// rows belong to its neighbours, which overwrite them during the same
// launch; so a block reads E^n and dB^n live only inside its own area (which
// no other block writes, and which it overwrites only rows below the one it
// is reading), and everywhere else from a snapshot of those regions taken
// just before (k_fuse_snap_cols, k_fuse_snap_rows).  J_PIC is only read, and
// the caller clears it after the launch.
constexpr int kFuseThreads = 128;     // columns of a strip, halo included
constexpr int kFuseHalo = 4;          // columns recomputed on each side
constexpr int kFuseWarm = 4;          // rows recomputed below a segment
constexpr int kFuseTrail = 5;         // rows above a segment the pipeline loads (up to i_e + 3)
constexpr int kFuseOwn = kFuseThreads - 2 * kFuseHalo;
constexpr int kFuseArrays = 6;        // E_r E_th E_ph dB_r dB_th dB_ph
// ring depths: rows live at once (see the phase order above)
constexpr int kDEn = 2, kDDbr = 1, kDDbn = 2, kDB0r = 3, kDB0h = 4, kDJp = 2, kDPsi = 2, kDBr = 4, kDBh = 4,
              kDE1r = 5, kDE1n = 3, kDD = 2, kDEc = 2, kDTab = 8;
constexpr int kFuseRingRows = 3 * kDEn + kDDbr + 2 * kDDbn + kDB0r + 2 * kDB0h + 3 * kDJp + kDBr + 2 * kDBh + kDE1r +
                              2 * kDE1n + 3 * kDD + 3 * kDEc;
// radial tables of a row, staged in shared memory by the first threads
enum FuseTab { TB_RN, TB_INV_RN, TB_C_E2, TB_C_EP2, TB_SIG_N, TB_RHO_A, TB_RHO_B, TB_RH, TB_INV_RH, TB_C_B2,
               TB_C_BP2, TB_SIG_H, TB_RH2, TB_COUNT };
constexpr int kTabN = 16;
static_assert(TB_COUNT <= kTabN && TB_COUNT <= kFuseThreads, "table row");

template <typename R>
size_t fuse_smem_bytes() {
  return ((size_t)kFuseRingRows * kFuseThreads + (size_t)kDTab * kTabN) * sizeof(R) +
         (size_t)kDPsi * kFuseThreads * sizeof(typename PsiOf<R>::T) + 16;
}

// Geometry of a launch: strips of kFuseOwn owned columns, segments of
// seg_rows owned rows.  Snapshot of E^n and dB^n (six arrays, every array
// addressed as (nr+1) x (nt+1)): for every strip boundary b = 1 .. strips-1
// the 2 kFuseHalo columns around column b kFuseOwn over all rows, and for
// every segment boundary b = 1 .. segs-1 the rows from b seg_rows - kFuseWarm
// to b seg_rows + kFuseTrail - 1 over all columns.
struct FuseGeom {
  int strips, segs, seg_rows;
};
__host__ __device__ inline FuseGeom fuse_geom(int nr, int nt, int seg_rows) {
  FuseGeom g;
  g.strips = (nt + 1 + kFuseOwn - 1) / kFuseOwn;
  g.seg_rows = seg_rows;
  g.segs = (nr + 1 + seg_rows - 1) / seg_rows;
  return g;
}
__host__ __device__ inline int64_t fuse_snap_cols(int nr, int strips) {
  return (int64_t)(strips > 1 ? strips - 1 : 0) * kFuseArrays * (nr + 1) * (2 * kFuseHalo);
}
__host__ __device__ inline int64_t fuse_snap_rows(int nt, int segs) {
  return (int64_t)(segs > 1 ? segs - 1 : 0) * kFuseArrays * (kFuseWarm + kFuseTrail) * (nt + 1);
}

template <typename R>
__device__ __forceinline__ const R *fuse_array(const Params<R> &p, int a, int &ld, int &rows, int &cols) {
  const int nr = p.nr, nt = p.nt;
  switch (a) {
    case 0: ld = nt + 1; rows = nr; cols = nt + 1; return p.f.er;
    case 1: ld = nt; rows = nr + 1; cols = nt; return p.f.et;
    case 2: ld = nt + 1; rows = nr + 1; cols = nt + 1; return p.f.ep;
    case 3: ld = nt; rows = nr + 1; cols = nt; return p.f.br;
    case 4: ld = nt + 1; rows = nr; cols = nt + 1; return p.f.bt;
    default: ld = nt; rows = nr; cols = nt; return p.f.bp;
  }
}

// the snapshot: halo columns (block 2 kFuseHalo x 32: column, row) ...
template <typename R>
__global__ void k_fuse_snap_cols(Params<R> p, R *snap_c) {
  const int cc = threadIdx.x, row = blockIdx.x * blockDim.y + threadIdx.y, ba = blockIdx.y;
  if (row > p.nr) return;
  const int a = ba % kFuseArrays, b = ba / kFuseArrays + 1;
  const int col = b * kFuseOwn - kFuseHalo + cc;
  int ld, rows, cols;
  const R *src = fuse_array(p, a, ld, rows, cols);
  const R v = (row < rows && col >= 0 && col < cols) ? src[(int64_t)row * ld + col] : R(0);
  snap_c[((int64_t)ba * (p.nr + 1) + row) * (2 * kFuseHalo) + cc] = v;
}
// ... and warm-up / trailing rows (grid: columns, row of the window, boundary x array)
template <typename R>
__global__ void k_fuse_snap_rows(Params<R> p, R *snap_r, int seg_rows) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x, rr = blockIdx.y, ba = blockIdx.z;
  if (col > p.nt) return;
  const int a = ba % kFuseArrays, b = ba / kFuseArrays + 1;
  const int row = b * seg_rows - kFuseWarm + rr;
  int ld, rows, cols;
  const R *src = fuse_array(p, a, ld, rows, cols);
  const R v = (row >= 0 && row < rows && col < cols) ? src[(int64_t)row * ld + col] : R(0);
  snap_r[((int64_t)ba * (kFuseWarm + kFuseTrail) + rr) * (p.nt + 1) + col] = v;
}

// a ring of rows in shared memory, one element per column of the strip
template <typename T, int D>
struct FRing {
  T *p;
  __device__ __forceinline__ T &operator()(int row, int c) const {
    return p[((unsigned)row % (unsigned)D) * kFuseThreads + c];
  }
};

// node row k and half row k of one column, in flight between phase 0 of
// step k-1 and phase 0 of step k
template <typename R>
struct FuseRow {
  R er, et, ep, br, bt, bp, b0r, b0t, b0p, tab;
  typename PsiOf<R>::T psi;
};
// J_PIC and curl B_0 of one column at the E locations of row k (half row
// for E_r, node row for E_th and E_ph), used by phase 2 of step k+1
template <typename R>
struct FuseSrc {
  R jr, sr, jt, st, jp, sp;
};

template <typename R>
__global__ void __launch_bounds__(kFuseThreads) k_field_fused(Params<R> p, R hdt, FuseGeom fg, const R *snap_c,
                                                              const R *snap_r) {
  using P = typename PsiOf<R>::T;
  constexpr int NC = kFuseThreads, H = kFuseHalo, W = kFuseWarm;
  extern __shared__ __align__(16) unsigned char fsmem[];
  const int nr = p.nr, nt = p.nt, n1 = nt + 1, seg_rows = fg.seg_rows;
  const int c = threadIdx.x, sx = blockIdx.x, sy = blockIdx.y;
  const int j = sx * kFuseOwn - H + c;                                 // global column of this thread
  const bool jn = j >= 0 && j <= nt, jh = j >= 0 && j < nt;           // node / half column exists
  const bool own = c >= H && c < NC - H;                              // column written by this block
  const int i_s = sy * seg_rows;                                      // first output row
  if (i_s > nr) return;
  const int i_e = min(i_s + seg_rows, nr + 1);                        // one past the last output node row
  const int k0 = max(0, i_s - W), kl = min(nr, i_e) + 3;              // row steps with phases 1-3
  const Fields<R> &f = p.f;
  const Tables<R> &t = p.t;
  // snapshot offset of a halo column (array 0, row 0); unused where the
  // column is outside the grid (the first strip's left and the last
  // strip's right halo)
  int64_t sc0 = 0;
  if (!own) {
    const int b = (c < H) ? sx : sx + 1;
    sc0 = (int64_t)(b - 1) * kFuseArrays * (nr + 1) * (2 * H) + (j - (b * kFuseOwn - H));
  }
  // the radial table this thread stages (threads 0 .. TB_COUNT-1)
  const R *tp = nullptr;
  int tlim = -1;
  switch (c) {
    case TB_RN: tp = t.rn; tlim = nr; break;
    case TB_INV_RN: tp = t.inv_rn; tlim = nr; break;
    case TB_C_E2: tp = t.c_e2; tlim = nr; break;
    case TB_C_EP2: tp = t.c_ep2; tlim = nr; break;
    case TB_SIG_N: tp = t.sig_n; tlim = nr; break;
    case TB_RHO_A: tp = t.rho_a; tlim = nr; break;
    case TB_RHO_B: tp = t.rho_b; tlim = nr; break;
    case TB_RH: tp = t.rh; tlim = nr - 1; break;
    case TB_INV_RH: tp = t.inv_rh; tlim = nr - 1; break;
    case TB_C_B2: tp = t.c_b2; tlim = nr - 1; break;
    case TB_C_BP2: tp = t.c_bp2; tlim = nr - 1; break;
    case TB_SIG_H: tp = t.sig_h; tlim = nr - 1; break;
    case TB_RH2: tp = t.rh2; tlim = nr - 1; break;
    default: break;
  }
  // Row steps come in two versions: interior steps, whose rows k-5 .. k+1
  // all lie inside this block's own rows and inside rows 2 .. nr-3 (every
  // row condition below holds), and the general one.  IN is true in the
  // former, where the compiler drops the row conditions.
  //
  // E^n and dB^n of node row k and half row k: live inside this block's own
  // area, from the snapshot in the halo columns and the warm-up / trailing
  // rows; then B_0, Psi and the radial table of the row
  auto fetch = [&](int k, FuseRow<R> &x, auto tag) {
    constexpr bool IN = decltype(tag)::value;
    const bool node = IN || k <= nr, half = IN || k < nr;
    const bool cer = half && jn, cet = node && jh, cep = node && jn, cbr = node && jh, cbt = half && jn,
               cbp = half && jh;
    const int64_t kn = (int64_t)k * n1 + j, kh = (int64_t)k * nt + j;
    if (own && (IN || (k >= i_s && k < i_e))) {
      x.er = cer ? f.er[kn] : R(0);
      x.et = cet ? f.et[kh] : R(0);
      x.ep = cep ? f.ep[kn] : R(0);
      x.br = cbr ? f.br[kh] : R(0);
      x.bt = cbt ? f.bt[kn] : R(0);
      x.bp = cbp ? f.bp[kh] : R(0);
    } else {
      // array a of the snapshot at s + a as (see k_fuse_snap_rows / _cols)
      const R *s;
      int64_t as;
      if (own) {
        const int b = (k < i_s) ? sy : sy + 1;
        s = snap_r + ((int64_t)(b - 1) * kFuseArrays * (W + kFuseTrail) + (k - (b * seg_rows - W))) * n1 + j;
        as = (int64_t)(W + kFuseTrail) * n1;
      } else {
        s = snap_c + sc0 + (int64_t)k * (2 * H);
        as = (int64_t)(nr + 1) * (2 * H);
      }
      x.er = cer ? s[0] : R(0);
      x.et = cet ? s[as] : R(0);
      x.ep = cep ? s[2 * as] : R(0);
      x.br = cbr ? s[3 * as] : R(0);
      x.bt = cbt ? s[4 * as] : R(0);
      x.bp = cbp ? s[5 * as] : R(0);
    }
    x.b0r = cbr ? __ldg(f.br0 + kh) : R(0);
    x.b0t = cbt ? __ldg(f.bt0 + kn) : R(0);
    x.b0p = cbp ? __ldg(f.bp0 + kh) : R(0);
    x.psi = cep ? __ldg(f.psi + kn) : P{};
    x.tab = (k <= tlim) ? __ldg(tp + k) : R(0);
  };
  auto fetch_src = [&](int k, FuseSrc<R> &y, auto tag) {
    constexpr bool IN = decltype(tag)::value;
    const bool node = IN || k <= nr, half = IN || k < nr;
    const int64_t kn = (int64_t)k * n1 + j, kh = (int64_t)k * nt + j;
    y.jr = (half && jn) ? __ldg(f.jr + kn) : R(0);
    y.sr = (half && jn) ? __ldg(f.sr + kn) : R(0);
    y.jt = (node && jh) ? __ldg(f.jt + kh) : R(0);
    y.st = (node && jh) ? __ldg(f.st + kh) : R(0);
    y.jp = (node && jn) ? __ldg(f.jp + kn) : R(0);
    y.sp = (node && jn) ? __ldg(f.sp + kn) : R(0);
  };
  // carve the rings
  FRing<R, kDEn> en_r, en_t, en_p;      // E^n            (half, node, node)
  FRing<R, kDDbr> dbr;                  // dB_r^n         (node)
  FRing<R, kDDbn> dbn_t, dbn_p;         // dB_th^n, dB_ph^n (half)
  FRing<R, kDB0r> b0_r;                 // B_0,r          (node)
  FRing<R, kDB0h> b0_t, b0_p;           // B_0,th, B_0,ph (half)
  FRing<R, kDJp> jp_r, jp_t, jp_p;      // J_perp         (node)
  FRing<R, kDBr> bh_r;                  // dB_r^{n+1/2}   (node)
  FRing<R, kDBh> bh_t, bh_p;            // dB^{n+1/2}     (half)
  FRing<R, kDE1r> e1_r;                 // E^{n+1} before the correction (half)
  FRing<R, kDE1n> e1_t, e1_p;           //                                (node)
  FRing<R, kDD> d_r, d_t, d_p;          // Delta E or E'' (node)
  FRing<R, kDEc> ec_r, ec_t, ec_p;      // corrected E    (half, node, node)
  FRing<P, kDPsi> psi;                  // Psi            (node)
  R *tab;                               // radial tables, kDTab rows of kTabN
  {
    R *q = reinterpret_cast<R *>(fsmem);
    auto take = [&](int rows) { R *r = q; q += rows * NC; return r; };
    en_r.p = take(kDEn); en_t.p = take(kDEn); en_p.p = take(kDEn);
    dbr.p = take(kDDbr); dbn_t.p = take(kDDbn); dbn_p.p = take(kDDbn);
    b0_r.p = take(kDB0r); b0_t.p = take(kDB0h); b0_p.p = take(kDB0h);
    jp_r.p = take(kDJp); jp_t.p = take(kDJp); jp_p.p = take(kDJp);
    bh_r.p = take(kDBr); bh_t.p = take(kDBh); bh_p.p = take(kDBh);
    e1_r.p = take(kDE1r); e1_t.p = take(kDE1n); e1_p.p = take(kDE1n);
    d_r.p = take(kDD); d_t.p = take(kDD); d_p.p = take(kDD);
    ec_r.p = take(kDEc); ec_t.p = take(kDEc); ec_p.p = take(kDEc);
    tab = q;
    q += kDTab * kTabN;
    uintptr_t a = reinterpret_cast<uintptr_t>(q);
    a = (a + 15) & ~uintptr_t(15);
    psi.p = reinterpret_cast<P *>(a);
  }
  auto T = [&](int row, int w) -> R { return tab[((unsigned)row % (unsigned)kDTab) * kTabN + w]; };
  // theta tables of this column
  const R sn0 = jn ? t.sn[j] : R(0), sn1 = jh ? t.sn[j + 1] : R(0), idcp = jh ? t.inv_dcp[j] : R(0);
  const R sh0 = jh ? t.sh[j] : R(0), shm = (j >= 1 && j <= nt) ? t.sh[j - 1] : R(0);
  const R idch = jn ? t.inv_dch[j] : R(0);
  const R dt = p.dt, fp4 = R(4.0 * kPi) * p.dt;
  const bool lit = p.ff_interp_e == 1, filt = p.ff_sigma16 != R(0);
  const bool axis = (j == 0 || j == nt);
  unsigned long long nclamp = 0;
  // blend weights of rows k-1, k-2, k-3 (E_r edge, E_th edge, node)
  R fr1 = 0, fr2 = 0, fr3 = 0, ft1 = 0, ft2 = 0, ft3 = 0, fn1 = 0, fn2 = 0, fn3 = 0;
  FuseRow<R> nx{};
  FuseSrc<R> js{}, jsn{};
  // F2: dB^{n+1} at node row k-4 and half row k-5 (own columns and rows)
  auto f2 = [&](int k, auto tag) {
    constexpr bool IN = decltype(tag)::value;
    if (!own) return;
    const int i = k - 4;  // B_r(i, j+1/2)
    if ((IN || (i >= i_s && i < i_e)) && jh) {
      const R cu = T(i, TB_INV_RN) * (sn1 * ec_p(i, c + 1) - sn0 * ec_p(i, c)) * idcp;
      R v = bh_r(i, c) - hdt * cu;
      const R sg = T(i, TB_SIG_N);
      if (sg > R(0)) v -= sg * v;
      f.br[(int64_t)i * nt + j] = v;
    }
    const int h = k - 5;  // B_th(h+1/2, j), B_ph(h+1/2, j+1/2)
    if (IN || (h >= i_s && h < i_e && h < nr)) {
      const R sg = T(h, TB_SIG_H), cb2 = T(h, TB_C_B2), rn0 = T(h, TB_RN), rn1 = T(h + 1, TB_RN);
      if (jn) {
        R v = R(0);
        if (j > 0 && j < nt) {
          v = bh_t(h, c) + hdt * cb2 * (rn1 * ec_p(h + 1, c) - rn0 * ec_p(h, c));
          if (sg > R(0)) v -= sg * v;
        }
        f.bt[(int64_t)h * n1 + j] = v;
      }
      if (jh) {
        const R cu = cb2 * (rn1 * ec_t(h + 1, c) - rn0 * ec_t(h, c)) - T(h, TB_C_BP2) * (ec_r(h, c + 1) - ec_r(h, c));
        R w = bh_p(h, c) - hdt * cu;
        if (sg > R(0)) w -= sg * w;
        f.bp[(int64_t)h * nt + j] = w;
      }
    }
  };
  auto step = [&](int k, auto tag) {
    constexpr bool IN = decltype(tag)::value;
    // ------------------------------------------------------------ phase 0
    f2(k, tag);
    en_r(k, c) = nx.er; en_t(k, c) = nx.et; en_p(k, c) = nx.ep;
    dbr(k, c) = nx.br; dbn_t(k, c) = nx.bt; dbn_p(k, c) = nx.bp;
    b0_r(k, c) = nx.b0r; b0_t(k, c) = nx.b0t; b0_p(k, c) = nx.b0p;
    psi(k, c) = nx.psi;
    if (c < TB_COUNT) tab[((unsigned)k % (unsigned)kDTab) * kTabN + c] = nx.tab;
    js = jsn;
    fetch_src(k, jsn, tag);
    if (IN || k + 1 <= kl) fetch(k + 1, nx, tag);
    __syncthreads();
    // ------------------------------------------------------------ phase 1
    if (IN || k <= nr) {
      // B_r(k, j+1/2)
      R v = dbr(k, c);
      if (jh && c < NC - 1) v -= hdt * (T(k, TB_INV_RN) * (sn1 * en_p(k, c + 1) - sn0 * en_p(k, c)) * idcp);
      bh_r(k, c) = v;
      // J_perp(k, j) = rho E x B / B^2 from E^n, B^n
      R jx = 0, jy = 0, jz = 0;
      if ((IN || (k >= 1 && k < nr)) && jn && c >= 1) {
        R e[3], b[3];
        e[0] = R(0.5) * (en_r(k - 1, c) + en_r(k, c));
        e[1] = axis ? R(0) : R(0.5) * (en_t(k, c - 1) + en_t(k, c));
        e[2] = axis ? R(0) : en_p(k, c);
        auto br = [&](int dc) { return b0_r(k, c + dc) + dbr(k, c + dc); };
        auto bt = [&](int row) { return b0_t(row, c) + dbn_t(row, c); };
        auto bp = [&](int row, int dc) { return b0_p(row, c + dc) + dbn_p(row, c + dc); };
        b[0] = (j == 0) ? br(0) : (j == nt) ? br(-1) : R(0.5) * (br(-1) + br(0));
        b[1] = axis ? R(0) : R(0.5) * (bt(k - 1) + bt(k));
        b[2] = axis ? R(0) : R(0.25) * (bp(k - 1, -1) + bp(k - 1, 0) + bp(k, -1) + bp(k, 0));
        const R div = T(k, TB_RHO_A) * (T(k, TB_RH2) * en_r(k, c) - T(k - 1, TB_RH2) * en_r(k - 1, c));
        R dth = 0;
        if (j < nt) dth += sh0 * en_t(k, c);
        if (j > 0) dth -= shm * en_t(k, c - 1);
        const R rho = div + T(k, TB_RHO_B) * dth * idch;
        const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        if (b2 > b2min<R>()) {
          const R s = rho / b2;
          jx = s * (e[1] * b[2] - e[2] * b[1]);
          jy = s * (e[2] * b[0] - e[0] * b[2]);
          jz = s * (e[0] * b[1] - e[1] * b[0]);
        }
      }
      jp_r(k, c) = jx; jp_t(k, c) = jy; jp_p(k, c) = jz;
      if (own && jn && (IN || (k >= i_s && k < i_e))) {
        const int64_t kk = (int64_t)k * n1 + j;
        f.jpr[kk] = jx; f.jpt[kk] = jy; f.jpp[kk] = jz;
      }
    }
    if (IN || (k >= 1 && k - 1 < nr)) {
      const int i = k - 1;
      const R cb2 = T(i, TB_C_B2), rn0 = T(i, TB_RN), rn1 = T(k, TB_RN);
      R v = R(0);  // B_th(i+1/2, j): zero on the axis
      if (j > 0 && j < nt) v = dbn_t(i, c) + hdt * cb2 * (rn1 * en_p(k, c) - rn0 * en_p(i, c));
      bh_t(i, c) = v;
      if (jh && c < NC - 1) {  // B_ph(i+1/2, j+1/2)
        const R cu = cb2 * (rn1 * en_t(k, c) - rn0 * en_t(i, c)) - T(i, TB_C_BP2) * (en_r(i, c + 1) - en_r(i, c));
        bh_p(i, c) = dbn_p(i, c) - hdt * cu;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------ phase 2
    fr3 = fr2; fr2 = fr1; ft3 = ft2; ft2 = ft1; fn3 = fn2; fn2 = fn1;
    fr1 = 0; ft1 = 0; fn1 = 0;
    if ((IN || (k >= 1 && k - 1 <= nr)) && c >= 1 && c < NC - 1) {  // A at row i = k-1
      const int i = k - 1;
      if ((IN || i < nr) && jn) {  // E_r(i+1/2, j)
        R cu = R(0);
        if (j < nt) cu += sh0 * bh_p(i, c);
        if (j > 0) cu -= shm * bh_p(i, c - 1);
        cu *= T(i, TB_INV_RH) * idch;
        const R fb = blend(p, psi_mean2(psi(i, c), psi(i + 1, c)));
        fr1 = fb;
        const bool lo = IN || i >= 1, hi = IN || i + 1 <= nr - 1;
        R jm = R(0);
        if (lo) jm += jp_r(i, c);
        if (hi) jm += jp_r(i + 1, c);
        if (lo && hi) jm *= R(0.5);
        const R jt = (R(1) - fb) * js.jr + fb * jm;
        e1_r(i, c) = (en_r(i, c) + dt * (cu + js.sr) - fp4 * jt) * (R(1) - T(i, TB_SIG_H));
      }
      if (jh) {  // E_th(i, j+1/2)
        R v;
        if (!IN && i == 0) {
          v = -p.omega * T(0, TB_RN) * sh0 * (b0_r(0, c) + bh_r(0, c));
        } else if (!IN && i == nr) {
          v = R(0);
        } else {
          const R cu = -T(i, TB_C_E2) * (T(i, TB_RH) * bh_p(i, c) - T(i - 1, TB_RH) * bh_p(i - 1, c));
          const R fb = blend(p, psi_mean2(psi(i, c), psi(i, c + 1)));
          ft1 = fb;
          const R jt = (R(1) - fb) * js.jt + fb * R(0.5) * (jp_t(i, c) + jp_t(i, c + 1));
          v = (en_t(i, c) + dt * (cu + js.st) - fp4 * jt) * (R(1) - T(i, TB_SIG_N));
        }
        e1_t(i, c) = v;
      }
      if (jn) {  // E_ph(i, j)
        R v = R(0);
        if ((IN || (i >= 1 && i < nr)) && j >= 1 && j < nt) {
          const R cu = T(i, TB_C_E2) * (T(i, TB_RH) * bh_t(i, c) - T(i - 1, TB_RH) * bh_t(i - 1, c)) -
                       T(i, TB_C_EP2) * (bh_r(i, c) - bh_r(i, c - 1));
          const R fb = blend(p, psi(i, c));
          fn1 = fb;
          const R jt = (R(1) - fb) * js.jp + fb * jp_p(i, c);
          v = (en_p(i, c) + dt * (cu + js.sp) - fp4 * jt) * (R(1) - T(i, TB_SIG_N));
        }
        e1_p(i, c) = v;
      }
    }
    if ((IN || (k >= 2 && k - 2 <= nr)) && c >= 1) {  // N at node row i = k-2
      const int i = k - 2;
      const bool orow = IN || (i >= i_s && i < i_e);
      R d0 = 0, d1 = 0, d2 = 0;
      if ((IN || (i >= 1 && i < nr)) && jn) {
        R e[3], b[3];
        e[0] = R(0.5) * (e1_r(i - 1, c) + e1_r(i, c));
        e[1] = axis ? R(0) : R(0.5) * (e1_t(i, c - 1) + e1_t(i, c));
        e[2] = axis ? R(0) : e1_p(i, c);
        auto br = [&](int dc) { return b0_r(i, c + dc) + bh_r(i, c + dc); };
        auto bt = [&](int row) { return b0_t(row, c) + bh_t(row, c); };
        auto bp = [&](int row, int dc) { return b0_p(row, c + dc) + bh_p(row, c + dc); };
        b[0] = (j == 0) ? br(0) : (j == nt) ? br(-1) : R(0.5) * (br(-1) + br(0));
        b[1] = axis ? R(0) : R(0.5) * (bt(i - 1) + bt(i));
        b[2] = axis ? R(0) : R(0.25) * (bp(i - 1, -1) + bp(i - 1, 0) + bp(i, -1) + bp(i, 0));
        const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        if (b2 > b2min<R>()) {
          const R sdot = (e[0] * b[0] + e[1] * b[1] + e[2] * b[2]) / b2;
          const R x = e[0] - sdot * b[0], y = e[1] - sdot * b[1], z = e[2] - sdot * b[2];
          const R e2 = x * x + y * y + z * z;
          const R sc = (e2 > b2) ? sqrt(b2 / e2) : R(1);
          d0 = sc * x - e[0];
          d1 = sc * y - e[1];
          d2 = sc * z - e[2];
          if (e2 > b2 && own && orow) ++nclamp;
        }
        if (lit) { d0 += e[0]; d1 += e[1]; d2 += e[2]; }
      }
      d_r(i, c) = d0; d_t(i, c) = d1; d_p(i, c) = d2;
      if (own && jn && orow) {
        const int64_t kk = (int64_t)i * n1 + j;
        f.der[kk] = d0; f.det[kk] = d1; f.dep[kk] = d2;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------ phase 3
    if ((IN || (k >= 3 && k - 3 <= nr)) && c >= 2 && c < NC - 2) {  // C at row i = k-3
      const int i = k - 3;
      const bool out = own && (IN || (i >= i_s && i < i_e));
      if ((IN || i < nr) && jn) {  // E_r(i+1/2, j)
        R v = e1_r(i, c);
        const R fb = fr3;
        if (fb != R(0)) {
          const bool lo = IN || i >= 1, hi = IN || i + 1 <= nr - 1;
          R m = R(0);
          if (lo) m += d_r(i, c);
          if (hi) m += d_r(i + 1, c);
          if (lo && hi) m *= R(0.5);
          if (filt && (IN || (i >= 2 && i <= nr - 3)))
            m -= p.ff_sigma16 * (e1_r(i - 2, c) - R(4) * e1_r(i - 1, c) + R(6) * v - R(4) * e1_r(i + 1, c) +
                                 e1_r(i + 2, c));
          v += fb * (lit ? m - v : m);
        }
        ec_r(i, c) = v;
        if (out) f.er[(int64_t)i * n1 + j] = v;
      }
      if (jh) {  // E_th(i, j+1/2)
        R v = e1_t(i, c);
        if (IN || (i >= 1 && i < nr)) {
          const R fb = ft3;
          if (fb != R(0)) {
            R m = R(0.5) * (d_t(i, c) + d_t(i, c + 1));
            if (filt && j >= 2 && j <= nt - 3)
              m -= p.ff_sigma16 * (e1_t(i, c - 2) - R(4) * e1_t(i, c - 1) + R(6) * v - R(4) * e1_t(i, c + 1) +
                                   e1_t(i, c + 2));
            v += fb * (lit ? m - v : m);
          }
        }
        ec_t(i, c) = v;
        if (out) f.et[(int64_t)i * nt + j] = v;
      }
      if (jn) {  // E_ph(i, j)
        R v = e1_p(i, c);
        if ((IN || (i >= 1 && i < nr)) && j >= 1 && j < nt) {
          const R fb = fn3;
          if (fb != R(0)) {
            const R m = d_p(i, c);
            v += fb * (lit ? m - v : m);
          }
        }
        ec_p(i, c) = v;
        if (out) f.ep[(int64_t)i * n1 + j] = v;
      }
    }
    __syncthreads();
  };
  // interior steps: rows k-5 .. k+1 own (k-5 >= i_s, k+1 < i_e) and inside
  // rows 2 .. nr-3 (k >= 7, k+4 <= nr)
  const int kin0 = max(i_s + 5, 7), kin1 = min(i_e - 2, nr - 4);
  fetch(k0, nx, std::false_type{});
  for (int k = k0; k <= kl; ++k) {
    if (k >= kin0 && k <= kin1) step(k, std::true_type{});
    else step(k, std::false_type{});
  }
  f2(kl + 1, std::false_type{});
  // running count of Eq. 26 activations (see k_node_b)
  unsigned long long tot = nclamp;
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(p.clamps, tot);
}

template <typename R> size_t field_fused_smem() { return fuse_smem_bytes<R>(); }
template <typename R> const void *field_fused_fn() { return reinterpret_cast<const void *>(&k_field_fused<R>); }
template <typename R> cudaError_t set_field_fused_smem(size_t bytes) { return raise_smem_limit<field_fused_fn<R>>(bytes); }
// rows per segment: as many segments as fit the strips into wave_blocks
// resident blocks (one wave: every block walks its rows once, none waits
// for a second wave), at least 32 rows so that the warm-up stays a small
// share
int fuse_seg_rows(int nr, int nt, int wave_blocks, size_t) {
  const int strips = (nt + 1 + kFuseOwn - 1) / kFuseOwn;
  const int segs = std::max(1, wave_blocks / strips);
  return std::max(32, (nr + 1 + segs - 1) / segs);
}
template <typename R> int field_fused_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_field_fused<R>, kFuseThreads, fuse_smem_bytes<R>()) !=
      cudaSuccess)
    return 0;
  return n;
}
int fuse_own_cols(size_t) { return kFuseOwn; }
size_t fuse_snap_bytes(int nr, int nt, int seg_rows, size_t real) {
  const FuseGeom fg = fuse_geom(nr, nt, seg_rows);
  return (size_t)(fuse_snap_cols(nr, fg.strips) + fuse_snap_rows(nt, fg.segs)) * real;
}
template <typename R> void launch_field_fused(const Params<R> &p, int seg_rows, void *snap, cudaStream_t s) {
  const FuseGeom fg = fuse_geom(p.nr, p.nt, seg_rows);
  R *sc = reinterpret_cast<R *>(snap);
  R *sr = sc + fuse_snap_cols(p.nr, fg.strips);
  if (fg.strips > 1)
    k_fuse_snap_cols<R><<<dim3((p.nr + 1 + 31) / 32, (fg.strips - 1) * kFuseArrays), dim3(2 * kFuseHalo, 32), 0, s>>>(
        p, sc);
  if (fg.segs > 1)
    k_fuse_snap_rows<R><<<dim3((p.nt + 1 + 255) / 256, kFuseWarm + kFuseTrail, (fg.segs - 1) * kFuseArrays), 256, 0,
                          s>>>(p, sr, seg_rows);
  k_field_fused<R><<<dim3(fg.strips, fg.segs), kFuseThreads, fuse_smem_bytes<R>(), s>>>(p, R(0.5) * p.dt, fg, sc, sr);
}

// The per-cell pure force-free flag f(Psi_cell) >= 1 (used to remove
// particles, Eq. 29) on its own, for the fused field update, which computes
// J_perp itself: a thread walks kFfRows cells of one column, reading every
// node row of Psi once (the arithmetic of ff_cell).
constexpr int kFfRows = 16;
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_ffcell(Params<R> p) {
  using P = typename PsiOf<R>::T;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i0 = blockIdx.y * kFfRows;
  if (j >= nt || i0 >= nr) return;
  const int i1 = min(i0 + kFfRows, nr);
  const P *psi = p.f.psi + j;
  P a = psi[(int64_t)i0 * n1], b = psi[(int64_t)i0 * n1 + 1];
  for (int i = i0; i < i1; ++i) {
    const P c = psi[(int64_t)(i + 1) * n1], d = psi[(int64_t)(i + 1) * n1 + 1];
    p.f.ffcell[(int64_t)i * nt + j] = blend(p, psi_mean4(a, c, b, d)) >= R(1) ? 1 : 0;
    a = c;
    b = d;
  }
}

// The blend weights of the last flux prefix, on request (hff_fields): f at
// the E_r and E_th edges and at the nodes, and the force-free cell flags
// (outputs passed as null are skipped).
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_blend_out(Params<R> p, R *fr, R *ft, R *fn, uint8_t *cells) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  if (fr && i < nr) fr[ix(i, j, n1)] = blend_redge(p, i, j);
  if (ft && j < nt) ft[ix(i, j, nt)] = blend_tedge(p, i, j);
  if (fn) fn[ix(i, j, n1)] = blend_node(p, i, j);
  if (cells && i < nr && j < nt) cells[ix(i, j, nt)] = ff_cell(p, i, j) ? 1 : 0;
}

static inline dim3 row_grid(int rows, int nt) { return dim3((nt + 1 + kRowThreads - 1) / kRowThreads, rows); }

template <typename R> size_t psi_smem(int nt) { return (size_t)(psi_pad(nt) + 2) * 8; }
template <typename R> void launch_psi(const Params<R> &p, cudaStream_t s) {
  const size_t smem = psi_smem<R>(p.nt);
  k_psi<R><<<p.nr + 1, kPsiThreads, smem, s>>>(p);
}
template <typename R> const void *psi_fn() { return reinterpret_cast<const void *>(&k_psi<R>); }
template <typename R> cudaError_t set_psi_smem(size_t bytes) { return raise_smem_limit<psi_fn<R>>(bytes); }
template <typename R> void launch_node_a(const Params<R> &p, cudaStream_t s) {
  k_node_a<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p);
}
template <typename R> void launch_ffcell(const Params<R> &p, cudaStream_t s) {
  k_ffcell<R><<<dim3((p.nt + kRowThreads - 1) / kRowThreads, (p.nr + kFfRows - 1) / kFfRows), kRowThreads, 0, s>>>(p);
}
template <typename R> void launch_faraday(const Params<R> &p, R half, bool absorb, cudaStream_t s) {
  k_faraday<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p, half * p.dt, absorb);
}
template <typename R> void launch_ampere(const Params<R> &p, cudaStream_t s) {
  k_ampere<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p);
}
template <typename R> void launch_correct(const Params<R> &p, cudaStream_t s) {
  k_node_b<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p);
  k_correct<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p);
}

template <typename R> void launch_blend_out(const Params<R> &p, R *fr, R *ft, R *fn, uint8_t *cells, cudaStream_t s) {
  k_blend_out<R><<<row_grid(p.nr + 1, p.nt), kRowThreads, 0, s>>>(p, fr, ft, fn, cells);
}

template <typename R>
__global__ void k_combine(R *dst, const R *a, const R *b, int64_t n, R sign) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = a[k] + sign * b[k];
}
template <typename R> void launch_combine(R *dst, const R *a, const R *b, int64_t n, int sign, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t blocks = (n + 255) / 256;
  k_combine<R><<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(dst, a, b, n, (R)sign);
}

#define HFF_INST(R)                                                            \
  template void launch_combine<R>(R *, const R *, const R *, int64_t, int, cudaStream_t); \
  template void launch_psi<R>(const Params<R> &, cudaStream_t);                \
  template cudaError_t set_psi_smem<R>(size_t);                                \
  template size_t psi_smem<R>(int);                                            \
  template void launch_node_a<R>(const Params<R> &, cudaStream_t);             \
  template void launch_ffcell<R>(const Params<R> &, cudaStream_t);             \
  template void launch_faraday<R>(const Params<R> &, R, bool, cudaStream_t);   \
  template void launch_ampere<R>(const Params<R> &, cudaStream_t);             \
  template void launch_correct<R>(const Params<R> &, cudaStream_t);            \
  template void launch_blend_out<R>(const Params<R> &, R *, R *, R *, uint8_t *, cudaStream_t); \
  template void launch_field_fused<R>(const Params<R> &, int, void *, cudaStream_t);            \
  template size_t field_fused_smem<R>();                                                         \
  template cudaError_t set_field_fused_smem<R>(size_t);                                          \
  template int field_fused_blocks_per_sm<R>();
HFF_INST(float)
HFF_INST(double)
#undef HFF_INST

}  // namespace hff
