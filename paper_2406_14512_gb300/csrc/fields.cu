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
// the edges (ff_interp_e).  With the optional fourth-difference filter it also
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
    if (p.ff_interp_e) { d0 += e[0]; d1 += e[1]; d2 += e[2]; }
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
// ff_interp_e, the corrected node field itself: E <- E + f (<E''> - E).
// The optional filter term (node pass B, in the J_PIC arrays) is subtracted
// with the same weight and its slot cleared for the next deposit.
template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_correct(Params<R> p) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  if (j > nt) return;
  const Fields<R> &f = p.f;
  const bool lit = p.ff_interp_e != 0;
  const bool filt = p.ff_sigma16 != R(0);
  if (i < nr) {
    const int64_t k = ix(i, j, n1);
    const R fb = blend_redge(p, i, j);
    R g = R(0);
    if (filt) { g = f.jr[k]; f.jr[k] = R(0); }
    if (fb != R(0)) {
      const R m = edge_r_mean(f.der, i, j, nr, n1) - g;
      f.er[k] += fb * (lit ? m - f.er[k] : m);
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
// The field update between the push and the injection -- Faraday's first
// half step (Eq. 18), Ampere's law with the blended current (Eqs. 19, 28) and
// the boundaries, the renormalisation at the nodes (Eqs. 25-26), the return to
// the edges with the blend weights, and Faraday's second half step with the
// absorber -- as one pass.  A block owns a strip of theta columns (with a
// halo of kFuseHalo columns on each side, recomputed) and a segment of rows
// (with kFuseWarm rows of warm-up below it, recomputed), and walks the rows
// upward.  At row step k it loads node row k and half row k (k+1/2) of E^n,
// dB^n, B_0, J_perp and Psi into ring buffers in shared memory, and then:
//   F1: B^{n+1/2} at node row k (B_r) and half row k-1 (B_th, B_ph);
//   A : E^{n+1} at half row k-1 (E_r) and node row k-1 (E_th, E_ph), J cleared;
//   N : Delta E (or E'') at node row k-1, and the filter terms;
//   C : the corrected E at half row k-3 and node row k-3;
//   F2: dB^{n+1} at node row k-3 (B_r) and half row k-4 (B_th, B_ph).
// Each stage reads only rows the earlier stages of this or previous steps
// produced, so every value is computed once per block from E^n and dB^n read
// once; the outputs are written once.  The arithmetic is that of k_faraday,
// k_ampere, k_node_b and k_correct, location by location.
//
// The update is in place, and a block's halo columns and warm-up / trailing
// rows belong to its neighbours, which overwrite them during the same
// launch; so a block reads E^n and dB^n live only inside its own area (which
// no other block writes, and which it overwrites only rows below the one it
// is reading), and everywhere else from a snapshot of those regions taken
// just before (k_fuse_snap).  J_PIC, read inside the halos too, is cleared by
// the caller after the launch.
constexpr int kFuseThreads = 128;     // columns of a strip, halo included
constexpr int kFuseHalo = 8;          // columns recomputed on each side
constexpr int kFuseWarm = 8;          // rows recomputed below a segment
// ring depths (rows live at once, see the step order above)
constexpr int kDEn = 2, kDBh = 4, kDB0n = 2, kDB0h = 3, kDJp = 2, kDPsi = 4, kDEnr = 5, kDEnn = 3, kDD = 3,
              kDEc = 2;

template <typename R>
struct FuseRings {
  R *en_r, *en_t, *en_p;        // E^n            (half, node, node)   kDEn
  R *dbn_t, *dbn_p;             // dB^n           (half, half)         kDEn
  R *b0_r, *b0_t, *b0_p;        // B_0            (node, half, half)   kDB0n, kDB0h
  R *jp_r, *jp_t, *jp_p;        // J_perp         (node)               kDJp
  typename PsiOf<R>::T *psi;    // Psi            (node)               kDPsi
  R *bh_r, *bh_t, *bh_p;        // dB^{n+1/2}     (node, half, half)   kDBh
  R *e1_r, *e1_t, *e1_p;        // E^{n+1} before the correction (half kDEnr, node kDEnn)
  R *d_r, *d_t, *d_p;           // Delta E or E'' (node)               kDD
  R *ec_r, *ec_t, *ec_p;        // corrected E    (half, node, node)   kDEc
};

template <typename R>
size_t fuse_smem_bytes() {
  const size_t rows = 3 * kDEn + 2 * kDEn + kDB0n + 2 * kDB0h + 3 * kDJp + 3 * kDBh + kDEnr + 2 * kDEnn + 3 * kDD +
                      3 * kDEc;
  return rows * kFuseThreads * sizeof(R) + (size_t)kDPsi * kFuseThreads * sizeof(typename PsiOf<R>::T) + 64;
}

// Geometry of a launch: strips of kFuseOwn owned columns, segments of
// seg_rows owned rows.  Snapshot of E^n and dB^n (six arrays, every array
// addressed as (nr+1) x (nt+1)): for every strip boundary b = 1 .. strips-1
// the 2 kFuseHalo columns around column b kFuseOwn over all rows, and for
// every segment boundary b = 1 .. segs-1 the rows from b seg_rows - kFuseWarm
// to b seg_rows + kFuseTrail - 1 over all columns.
constexpr int kFuseOwn = kFuseThreads - 2 * kFuseHalo;
constexpr int kFuseTrail = 5;   // rows above a segment the pipeline reads (k1 = i_e + 4)
constexpr int kFuseArrays = 6;  // E_r E_th E_ph dB_r dB_th dB_ph
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

// the snapshot (one thread per snapshot element)
template <typename R>
__global__ void k_fuse_snap(Params<R> p, R *snap_c, R *snap_r, FuseGeom fg) {
  const int nr = p.nr, nt = p.nt;
  const int64_t nc = fuse_snap_cols(nr, fg.strips), nrw = fuse_snap_rows(nt, fg.segs);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc + nrw; e += (int64_t)gridDim.x * blockDim.x) {
    int b, a, row, col;
    if (e < nc) {
      const int w = 2 * kFuseHalo;
      int64_t q = e;
      const int cc = (int)(q % w); q /= w;
      row = (int)(q % (nr + 1)); q /= (nr + 1);
      a = (int)(q % kFuseArrays); b = (int)(q / kFuseArrays) + 1;
      col = b * kFuseOwn - kFuseHalo + cc;
    } else {
      const int h = kFuseWarm + kFuseTrail;
      int64_t q = e - nc;
      col = (int)(q % (nt + 1)); q /= (nt + 1);
      const int rr = (int)(q % h); q /= h;
      a = (int)(q % kFuseArrays); b = (int)(q / kFuseArrays) + 1;
      row = b * fg.seg_rows - kFuseWarm + rr;
    }
    int ld, rows, cols;
    const R *src = fuse_array(p, a, ld, rows, cols);
    const R v = (row >= 0 && row < rows && col >= 0 && col < cols) ? src[(int64_t)row * ld + col] : R(0);
    if (e < nc) snap_c[e] = v;
    else snap_r[e - nc] = v;
  }
}

// ring slot of a row (rows may be negative for never-used slots)
__device__ __forceinline__ int rs(int row, int depth) { return ((row % depth) + depth) % depth; }

template <typename R>
__global__ void __launch_bounds__(kFuseThreads) k_field_fused(Params<R> p, R hdt, FuseGeom fg, const R *snap_c,
                                                              const R *snap_r) {
  using P = typename PsiOf<R>::T;
  extern __shared__ __align__(16) unsigned char fsmem[];
  const int nr = p.nr, nt = p.nt, n1 = nt + 1, NC = kFuseThreads, seg_rows = fg.seg_rows;
  const int c = threadIdx.x, sx = blockIdx.x, sy = blockIdx.y;
  const int j = sx * kFuseOwn - kFuseHalo + c;                          // global column of this thread
  const bool jn = j >= 0 && j <= nt, jh = j >= 0 && j < nt;          // node / half column exists
  const bool own = c >= kFuseHalo && c < NC - kFuseHalo;               // column written by this block
  const int i_s = sy * seg_rows;                                       // first output row
  if (i_s > nr) return;
  const int i_e = min(i_s + seg_rows, nr + 1);                         // one past the last output node row
  // E^n and dB^n at (row, column j): live inside this block's own area,
  // from the snapshot in the halo columns and the warm-up / trailing rows
  auto src = [&](int a, const R *live, int ld, int row) -> R {
    if (own && row >= i_s && row < i_e) return live[(int64_t)row * ld + j];
    if (!own) {
      const int b = (c < kFuseHalo) ? sx : sx + 1;                     // strip boundary
      const int cc = j - (b * kFuseOwn - kFuseHalo);
      return snap_c[(((int64_t)(b - 1) * kFuseArrays + a) * (nr + 1) + row) * (2 * kFuseHalo) + cc];
    }
    const int b = (row < i_s) ? sy : sy + 1;                           // segment boundary
    const int rr = row - (b * seg_rows - kFuseWarm);
    return snap_r[(((int64_t)(b - 1) * kFuseArrays + a) * (kFuseWarm + kFuseTrail) + rr) * (nt + 1) + j];
  };
  const int k0 = max(0, i_s - kFuseWarm), k1 = min(nr, i_e) + 4;
  // carve the rings
  FuseRings<R> g;
  {
    R *q = reinterpret_cast<R *>(fsmem);
    auto take = [&](int rows) { R *r = q; q += rows * NC; return r; };
    g.en_r = take(kDEn); g.en_t = take(kDEn); g.en_p = take(kDEn);
    g.dbn_t = take(kDEn); g.dbn_p = take(kDEn);
    g.b0_r = take(kDB0n); g.b0_t = take(kDB0h); g.b0_p = take(kDB0h);
    g.jp_r = take(kDJp); g.jp_t = take(kDJp); g.jp_p = take(kDJp);
    g.bh_r = take(kDBh); g.bh_t = take(kDBh); g.bh_p = take(kDBh);
    g.e1_r = take(kDEnr); g.e1_t = take(kDEnn); g.e1_p = take(kDEnn);
    g.d_r = take(kDD); g.d_t = take(kDD); g.d_p = take(kDD);
    g.ec_r = take(kDEc); g.ec_t = take(kDEc); g.ec_p = take(kDEc);
    uintptr_t a = reinterpret_cast<uintptr_t>(q);
    a = (a + 15) & ~uintptr_t(15);
    g.psi = reinterpret_cast<P *>(a);
  }
  // ring accessors: (array, depth, row, column offset)
  auto at = [&](R *ring, int depth, int row, int dc) -> R & { return ring[rs(row, depth) * NC + c + dc]; };
  const Fields<R> &f = p.f;
  const Tables<R> &t = p.t;
  const R dt = p.dt, fp = R(4.0 * kPi) * p.dt;
  const bool lit = p.ff_interp_e != 0, filt = p.ff_sigma16 != R(0);
  bool clamped_any = false;
  unsigned long long nclamp = 0;
  for (int k = k0; k <= k1; ++k) {
    // ---------------------------------------------------------------- load
    if (k <= nr) {
      const int64_t kn = ix(k, j, n1), kh = ix(k, j, nt);
      at(g.en_t, kDEn, k, 0) = jh ? src(1, f.et, nt, k) : R(0);
      at(g.en_p, kDEn, k, 0) = jn ? src(2, f.ep, n1, k) : R(0);
      at(g.b0_r, kDB0n, k, 0) = jh ? f.br0[kh] : R(0);
      at(g.bh_r, kDBh, k, 0) = jh ? src(3, f.br, nt, k) : R(0);  // dB_r^n, advanced in place by F1 below
      at(g.jp_r, kDJp, k, 0) = jn ? f.jpr[kn] : R(0);
      at(g.jp_t, kDJp, k, 0) = jn ? f.jpt[kn] : R(0);
      at(g.jp_p, kDJp, k, 0) = jn ? f.jpp[kn] : R(0);
      g.psi[rs(k, kDPsi) * NC + c] = jn ? f.psi[kn] : P{};
      if (k < nr) {
        at(g.en_r, kDEn, k, 0) = jn ? src(0, f.er, n1, k) : R(0);
        at(g.dbn_t, kDEn, k, 0) = jn ? src(4, f.bt, n1, k) : R(0);
        at(g.dbn_p, kDEn, k, 0) = jh ? src(5, f.bp, nt, k) : R(0);
        at(g.b0_t, kDB0h, k, 0) = jn ? f.bt0[kn] : R(0);
        at(g.b0_p, kDB0h, k, 0) = jh ? f.bp0[kh] : R(0);
      }
    }
    __syncthreads();
    // ------------------------------------------------------------------ F1
    if (k <= nr && jh && c < NC - 1) {  // B_r(k, j+1/2)
      const R cu = t.inv_rn[k] * (t.sn[j + 1] * at(g.en_p, kDEn, k, 1) - t.sn[j] * at(g.en_p, kDEn, k, 0)) *
                   t.inv_dcp[j];
      at(g.bh_r, kDBh, k, 0) -= hdt * cu;
    }
    if (k >= 1 && k - 1 < nr) {
      const int i = k - 1;
      R v = R(0);  // B_th(i+1/2, j): zero on the axis
      if (j > 0 && j < nt)
        v = at(g.dbn_t, kDEn, i, 0) +
            hdt * t.c_b2[i] * (t.rn[i + 1] * at(g.en_p, kDEn, i + 1, 0) - t.rn[i] * at(g.en_p, kDEn, i, 0));
      at(g.bh_t, kDBh, i, 0) = v;
      if (jh && c < NC - 1) {  // B_ph(i+1/2, j+1/2)
        const R cu = t.c_b2[i] * (t.rn[i + 1] * at(g.en_t, kDEn, i + 1, 0) - t.rn[i] * at(g.en_t, kDEn, i, 0)) -
                     t.c_bp2[i] * (at(g.en_r, kDEn, i, 1) - at(g.en_r, kDEn, i, 0));
        at(g.bh_p, kDBh, i, 0) = at(g.dbn_p, kDEn, i, 0) - hdt * cu;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------------- A
    if (k >= 1 && k - 1 <= nr && c >= 1 && c < NC - 1) {
      const int i = k - 1;
      auto psi_at = [&](int row, int dc) { return g.psi[rs(row, kDPsi) * NC + c + dc]; };
      if (i < nr && jn) {  // E_r(i+1/2, j)
        R cu = R(0);
        if (j < nt) cu += t.sh[j] * at(g.bh_p, kDBh, i, 0);
        if (j > 0) cu -= t.sh[j - 1] * at(g.bh_p, kDBh, i, -1);
        cu *= t.inv_rh[i] * t.inv_dch[j];
        const R fb = blend(p, psi_mean2(psi_at(i, 0), psi_at(i + 1, 0)));
        const bool lo = i >= 1, hi = i + 1 <= nr - 1;
        R jm = R(0);
        if (lo) jm += at(g.jp_r, kDJp, i, 0);
        if (hi) jm += at(g.jp_r, kDJp, i + 1, 0);
        if (lo && hi) jm *= R(0.5);
        const int64_t kk = ix(i, j, n1);
        const R jt = (R(1) - fb) * f.jr[kk] + fb * jm;
        at(g.e1_r, kDEnr, i, 0) = (at(g.en_r, kDEn, i, 0) + dt * (cu + f.sr[kk]) - fp * jt) * (R(1) - t.sig_h[i]);
      }
      if (jh) {  // E_th(i, j+1/2)
        const int64_t kk = ix(i, j, nt);
        R v;
        if (i == 0) {
          v = -p.omega * t.rn[0] * t.sh[j] * (at(g.b0_r, kDB0n, 0, 0) + at(g.bh_r, kDBh, 0, 0));
        } else if (i == nr) {
          v = R(0);
        } else {
          const R cu = -t.c_e2[i] * (t.rh[i] * at(g.bh_p, kDBh, i, 0) - t.rh[i - 1] * at(g.bh_p, kDBh, i - 1, 0));
          const R fb = blend(p, psi_mean2(psi_at(i, 0), psi_at(i, 1)));
          const R jt = (R(1) - fb) * f.jt[kk] + fb * R(0.5) * (at(g.jp_t, kDJp, i, 0) + at(g.jp_t, kDJp, i, 1));
          v = (at(g.en_t, kDEn, i, 0) + dt * (cu + f.st[kk]) - fp * jt) * (R(1) - t.sig_n[i]);
        }
        at(g.e1_t, kDEnn, i, 0) = v;
      }
      if (jn) {  // E_ph(i, j)
        const int64_t kk = ix(i, j, n1);
        R v = R(0);
        if (i >= 1 && i < nr && j >= 1 && j < nt) {
          const R cu = t.c_e2[i] * (t.rh[i] * at(g.bh_t, kDBh, i, 0) - t.rh[i - 1] * at(g.bh_t, kDBh, i - 1, 0)) -
                       t.c_ep2[i] * (at(g.bh_r, kDBh, i, 0) - at(g.bh_r, kDBh, i, -1));
          const R fb = blend(p, psi_at(i, 0));
          const R jt = (R(1) - fb) * f.jp[kk] + fb * at(g.jp_p, kDJp, i, 0);
          v = (at(g.en_p, kDEn, i, 0) + dt * (cu + f.sp[kk]) - fp * jt) * (R(1) - t.sig_n[i]);
        }
        at(g.e1_p, kDEnn, i, 0) = v;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------------- N
    if (k >= 1 && k - 1 <= nr && c >= 1 && c < NC - 1) {
      const int i = k - 1;
      R d0 = 0, d1 = 0, d2 = 0;
      if (i >= 1 && i < nr && jn) {
        const bool axis = (j == 0 || j == nt);
        R e[3], b[3];
        e[0] = R(0.5) * (at(g.e1_r, kDEnr, i - 1, 0) + at(g.e1_r, kDEnr, i, 0));
        e[1] = axis ? R(0) : R(0.5) * (at(g.e1_t, kDEnn, i, -1) + at(g.e1_t, kDEnn, i, 0));
        e[2] = axis ? R(0) : at(g.e1_p, kDEnn, i, 0);
        auto br = [&](int dc) { return at(g.b0_r, kDB0n, i, dc) + at(g.bh_r, kDBh, i, dc); };
        auto bt = [&](int row) { return at(g.b0_t, kDB0h, row, 0) + at(g.bh_t, kDBh, row, 0); };
        auto bp = [&](int row, int dc) { return at(g.b0_p, kDB0h, row, dc) + at(g.bh_p, kDBh, row, dc); };
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
          if (e2 > b2 && own && i >= i_s && i < i_e) { clamped_any = true; ++nclamp; }
        }
        if (lit) { d0 += e[0]; d1 += e[1]; d2 += e[2]; }
      }
      at(g.d_r, kDD, i, 0) = d0;
      at(g.d_t, kDD, i, 0) = d1;
      at(g.d_p, kDD, i, 0) = d2;
      if (own && jn && i >= i_s && i < i_e) {
        const int64_t kk = ix(i, j, n1);
        f.der[kk] = d0; f.det[kk] = d1; f.dep[kk] = d2;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------------- C
    if (k >= 3 && k - 3 <= nr && c >= 2 && c < NC - 2) {
      const int i = k - 3;
      auto psi_at = [&](int row, int dc) { return g.psi[rs(row, kDPsi) * NC + c + dc]; };
      if (i < nr && jn) {  // E_r(i+1/2, j)
        R v = at(g.e1_r, kDEnr, i, 0);
        const R fb = blend(p, psi_mean2(psi_at(i, 0), psi_at(i + 1, 0)));
        if (fb != R(0)) {
          const bool lo = i >= 1, hi = i + 1 <= nr - 1;
          R m = R(0);
          if (lo) m += at(g.d_r, kDD, i, 0);
          if (hi) m += at(g.d_r, kDD, i + 1, 0);
          if (lo && hi) m *= R(0.5);
          if (filt && i >= 2 && i <= nr - 3)
            m -= p.ff_sigma16 * (at(g.e1_r, kDEnr, i - 2, 0) - R(4) * at(g.e1_r, kDEnr, i - 1, 0) + R(6) * v -
                                 R(4) * at(g.e1_r, kDEnr, i + 1, 0) + at(g.e1_r, kDEnr, i + 2, 0));
          v += fb * (lit ? m - v : m);
        }
        at(g.ec_r, kDEc, i, 0) = v;
        if (own && i >= i_s && i < i_e) f.er[ix(i, j, n1)] = v;
      }
      if (jh) {  // E_th(i, j+1/2)
        R v = at(g.e1_t, kDEnn, i, 0);
        if (i >= 1 && i < nr) {
          const R fb = blend(p, psi_mean2(psi_at(i, 0), psi_at(i, 1)));
          if (fb != R(0)) {
            R m = R(0.5) * (at(g.d_t, kDD, i, 0) + at(g.d_t, kDD, i, 1));
            if (filt && j >= 2 && j <= nt - 3)
              m -= p.ff_sigma16 * (at(g.e1_t, kDEnn, i, -2) - R(4) * at(g.e1_t, kDEnn, i, -1) + R(6) * v -
                                   R(4) * at(g.e1_t, kDEnn, i, 1) + at(g.e1_t, kDEnn, i, 2));
            v += fb * (lit ? m - v : m);
          }
        }
        at(g.ec_t, kDEc, i, 0) = v;
        if (own && i >= i_s && i < i_e) f.et[ix(i, j, nt)] = v;
      }
      if (jn) {  // E_ph(i, j)
        R v = at(g.e1_p, kDEnn, i, 0);
        if (i >= 1 && i < nr && j >= 1 && j < nt) {
          const R fb = blend(p, psi_at(i, 0));
          if (fb != R(0)) {
            const R m = at(g.d_p, kDD, i, 0);
            v += fb * (lit ? m - v : m);
          }
        }
        at(g.ec_p, kDEc, i, 0) = v;
        if (own && i >= i_s && i < i_e) f.ep[ix(i, j, n1)] = v;
      }
    }
    __syncthreads();
    // ------------------------------------------------------------------ F2
    if (own) {
      if (k >= 3 && k - 3 <= nr && jh) {  // B_r(i, j+1/2), i = k-3
        const int i = k - 3;
        const R cu = t.inv_rn[i] * (t.sn[j + 1] * at(g.ec_p, kDEc, i, 1) - t.sn[j] * at(g.ec_p, kDEc, i, 0)) *
                     t.inv_dcp[j];
        R v = at(g.bh_r, kDBh, i, 0) - hdt * cu;
        const R sg = t.sig_n[i];
        if (sg > R(0)) v -= sg * v;
        if (i >= i_s && i < i_e) f.br[ix(i, j, nt)] = v;
      }
      if (k >= 4 && k - 4 < nr) {  // B_th, B_ph at half row i = k-4
        const int i = k - 4;
        if (i >= i_s && i < i_e) {
          if (jn) {
            R v = R(0);
            if (j > 0 && j < nt) {
              v = at(g.bh_t, kDBh, i, 0) +
                  hdt * t.c_b2[i] * (t.rn[i + 1] * at(g.ec_p, kDEc, i + 1, 0) - t.rn[i] * at(g.ec_p, kDEc, i, 0));
              const R sg = t.sig_h[i];
              if (sg > R(0)) v -= sg * v;
            }
            f.bt[ix(i, j, n1)] = v;
          }
          if (jh) {
            const R cu = t.c_b2[i] * (t.rn[i + 1] * at(g.ec_t, kDEc, i + 1, 0) - t.rn[i] * at(g.ec_t, kDEc, i, 0)) -
                         t.c_bp2[i] * (at(g.ec_r, kDEc, i, 1) - at(g.ec_r, kDEc, i, 0));
            R w = at(g.bh_p, kDBh, i, 0) - hdt * cu;
            const R sg = t.sig_h[i];
            if (sg > R(0)) w -= sg * w;
            f.bp[ix(i, j, nt)] = w;
          }
        }
      }
    }
    __syncthreads();  // the next step's loads reuse ring slots
  }
  // running count of Eq. 26 activations (see k_node_b)
  const unsigned m = __ballot_sync(0xffffffffu, clamped_any);
  unsigned long long tot = nclamp;
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
  if (m && (threadIdx.x & 31) == 0 && tot) atomicAdd(p.clamps, tot);
}

template <typename R> size_t field_fused_smem() { return fuse_smem_bytes<R>(); }
template <typename R> const void *field_fused_fn() { return reinterpret_cast<const void *>(&k_field_fused<R>); }
template <typename R> cudaError_t set_field_fused_smem(size_t bytes) { return raise_smem_limit<field_fused_fn<R>>(bytes); }
// rows per segment: enough blocks for the GPU (about eight per SM), at
// least 32 rows so that the warm-up stays a small share
int fuse_seg_rows(int nr, int nt, int n_sm) {
  const int strips = (nt + 1 + kFuseOwn - 1) / kFuseOwn;
  const int want = std::max(1, (8 * n_sm + strips - 1) / strips);
  return std::max(32, (nr + 1 + want - 1) / want);
}
size_t fuse_snap_bytes(int nr, int nt, int seg_rows, size_t real) {
  const FuseGeom fg = fuse_geom(nr, nt, seg_rows);
  return (size_t)(fuse_snap_cols(nr, fg.strips) + fuse_snap_rows(nt, fg.segs)) * real;
}
template <typename R> void launch_field_fused(const Params<R> &p, int seg_rows, void *snap, cudaStream_t s) {
  const FuseGeom fg = fuse_geom(p.nr, p.nt, seg_rows);
  R *sc = reinterpret_cast<R *>(snap);
  R *sr = sc + fuse_snap_cols(p.nr, fg.strips);
  const int64_t n = fuse_snap_cols(p.nr, fg.strips) + fuse_snap_rows(p.nt, fg.segs);
  if (n > 0) k_fuse_snap<R><<<(unsigned)std::min<int64_t>((n + 255) / 256, 16384), 256, 0, s>>>(p, sc, sr, fg);
  k_field_fused<R><<<dim3(fg.strips, fg.segs), kFuseThreads, fuse_smem_bytes<R>(), s>>>(p, R(0.5) * p.dt, fg, sc, sr);
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
  template void launch_faraday<R>(const Params<R> &, R, bool, cudaStream_t);   \
  template void launch_ampere<R>(const Params<R> &, cudaStream_t);             \
  template void launch_correct<R>(const Params<R> &, cudaStream_t);            \
  template void launch_blend_out<R>(const Params<R> &, R *, R *, R *, uint8_t *, cudaStream_t); \
  template void launch_field_fused<R>(const Params<R> &, int, void *, cudaStream_t);            \
  template size_t field_fused_smem<R>();                                                         \
  template cudaError_t set_field_fused_smem<R>(size_t);
HFF_INST(float)
HFF_INST(double)
#undef HFF_INST

}  // namespace hff
