// particles.cu -- particle side of the hybrid step: linear gather from the
// staggered mesh, modified Boris push with radiation reaction (Eqs. 15-17),
// removal of u_perp near the star (Sect. 5.1), straight-line move in the
// local Cartesian frame, charge-conserving (Esirkepov) deposit of J_PIC, and
// the surface pair injection (Sects. 4 and 5.1).
//
// Two drivers share one per-particle routine:
//  * k_push_tiled -- persistent blocks take (species, tile, chunk) work items
//    from a list built by the sort.  The block stages E, B and the force-free
//    flags of the tile plus a halo (the farthest a particle can drift between
//    sorts) into shared memory, accumulates J in shared memory with shared
//    atomics, and flushes the tile's J with one global atomic per nonzero
//    entry.  Particles of a tile are contiguous, so the particle stream is
//    read and written once, fully coalesced.
//  * k_push_tail -- particles appended since the last sort (injection) and
//    the no-sort configuration: gathers through L1/L2 and global atomics.
#include <type_traits>

#include "hff_common.cuh"

namespace hff {

// -------------------------------------------------------------- accessors
// Global-memory view of the mesh.
template <typename R>
struct GlobalMesh {
  const Params<R> &p;
  __device__ GlobalMesh(const Params<R> &pp) : p(pp) {}
  __device__ __forceinline__ R er(int i, int j) const { return p.f.er[ix(i, j, p.nt + 1)]; }
  __device__ __forceinline__ R et(int i, int j) const { return p.f.et[ix(i, j, p.nt)]; }
  __device__ __forceinline__ R ep(int i, int j) const { return p.f.ep[ix(i, j, p.nt + 1)]; }
  // B = B_0 + dB
  __device__ __forceinline__ R br(int i, int j) const { const int64_t k = ix(i, j, p.nt); return p.f.br0[k] + p.f.br[k]; }
  __device__ __forceinline__ R bt(int i, int j) const { const int64_t k = ix(i, j, p.nt + 1); return p.f.bt0[k] + p.f.bt[k]; }
  __device__ __forceinline__ R bp(int i, int j) const { const int64_t k = ix(i, j, p.nt); return p.f.bp0[k] + p.f.bp[k]; }
  __device__ __forceinline__ bool ff(int i, int j) const { return p.f.ffcell[ix(i, j, p.nt)] != 0; }
  // raw charge flux through a dual face (J_r, J_th) or charge x velocity at
  // a node (J_ph), converted to a current density with the face area or
  // node volume and dt here
  // (indices outside the arrays carry zero flux for every valid move; they
  // are still checked here, on the global path)
  __device__ __forceinline__ void add_jr(int i, int j, R v) const {
    if (i >= 0 && i < p.nr && j >= 0 && j <= p.nt)
      atomicAdd(&p.f.jr[ix(i, j, p.nt + 1)], v * p.t.dep_r[i] * p.t.inv_dch[j]);
  }
  __device__ __forceinline__ void add_jt(int i, int j, R v) const {
    if (i >= 0 && i <= p.nr && j >= 0 && j < p.nt)
      atomicAdd(&p.f.jt[ix(i, j, p.nt)], v * p.t.dep_t[i] * p.t.inv_sh[j]);
  }
  __device__ __forceinline__ void add_jp(int i, int j, R v) const {
    if (i >= 0 && i <= p.nr && j >= 0 && j <= p.nt)
      atomicAdd(&p.f.jp[ix(i, j, p.nt + 1)], v * p.t.dep_p[i] * p.t.inv_dch[j]);
  }
  __device__ __forceinline__ R rn(int i) const { return p.t.rn[i]; }
  __device__ __forceinline__ R sn(int j) const { return p.t.sn[j]; }
  __device__ __forceinline__ R cn(int j) const { return p.t.cn[j]; }
};

// Shared-memory view of a tile region [i0, i0 + LR) x [j0, j0 + LT) of every
// component (indices are global; the caller guarantees they fall inside).
template <typename R>
struct SharedMesh {
  R *s_er, *s_et, *s_ep, *s_br, *s_bt, *s_bp, *s_jr, *s_jt, *s_jp;
  R *s_rn, *s_sn, *s_cn;   // row / column tables of the region
  uint8_t *s_ff;
  int i0, j0, lt;
  __device__ __forceinline__ int o(int i, int j) const { return (i - i0) * lt + (j - j0); }
  __device__ __forceinline__ R er(int i, int j) const { return s_er[o(i, j)]; }
  __device__ __forceinline__ R et(int i, int j) const { return s_et[o(i, j)]; }
  __device__ __forceinline__ R ep(int i, int j) const { return s_ep[o(i, j)]; }
  __device__ __forceinline__ R br(int i, int j) const { return s_br[o(i, j)]; }
  __device__ __forceinline__ R bt(int i, int j) const { return s_bt[o(i, j)]; }
  __device__ __forceinline__ R bp(int i, int j) const { return s_bp[o(i, j)]; }
  __device__ __forceinline__ bool ff(int i, int j) const { return s_ff[o(i, j)] != 0; }
  __device__ __forceinline__ void add_jr(int i, int j, R v) const { atomicAdd(&s_jr[o(i, j)], v); }
  __device__ __forceinline__ void add_jt(int i, int j, R v) const { atomicAdd(&s_jt[o(i, j)], v); }
  __device__ __forceinline__ void add_jp(int i, int j, R v) const { atomicAdd(&s_jp[o(i, j)], v); }
  __device__ __forceinline__ R rn(int i) const { return s_rn[i - i0]; }
  __device__ __forceinline__ R sn(int j) const { return s_sn[j - j0]; }
  __device__ __forceinline__ R cn(int j) const { return s_cn[j - j0]; }
};

// 1D linear weights for a component at positions k + a (a = 0 or 1/2),
// k = 0 .. n-1, constant beyond the ends.
template <typename R>
__device__ __forceinline__ void stag(int c, R o, bool half, int n, int &k0, R &w) {
  if (!half) { k0 = c; w = o; }
  else if (o >= R(0.5)) { k0 = c; w = o - R(0.5); }
  else { k0 = c - 1; w = o + R(0.5); }
  if (k0 < 0) { k0 = 0; w = R(0); }
  if (k0 > n - 2) { k0 = n - 2; w = R(1); }
}

// Small-argument Taylor expansions about 0, for the per-step increments that
// the Courant condition keeps small; callers switch to the library functions
// outside |x| < kSmall, where every truncation error is below 1e-12.
constexpr double kSmall = 0.03;
template <typename R> __device__ __forceinline__ R sin_small(R x) {
  const R x2 = x * x;
  return x * (R(1) - x2 * R(1.0 / 6.0) * (R(1) - x2 * R(1.0 / 20.0) * (R(1) - x2 * R(1.0 / 42.0))));
}
template <typename R> __device__ __forceinline__ R cos_small(R x) {
  const R x2 = x * x;
  return R(1) - R(0.5) * x2 * (R(1) - x2 * R(1.0 / 12.0) * (R(1) - x2 * R(1.0 / 30.0)));
}
template <typename R> __device__ __forceinline__ R atan_small(R t) {
  const R t2 = t * t;
  return t * (R(1) - t2 * (R(1.0 / 3.0) - t2 * (R(0.2) - t2 * (R(1.0 / 7.0) - t2 * R(1.0 / 9.0)))));
}
template <typename R> __device__ __forceinline__ R log1p_small(R x) {
  return x * (R(1) - x * (R(0.5) - x * (R(1.0 / 3.0) - x * (R(0.25) - x * (R(0.2) - x * (R(1.0 / 6.0) - x * R(1.0 / 7.0)))))));
}
template <typename R> __device__ __forceinline__ R exp_small(R x) {
  return R(1) + x * (R(1) + x * R(0.5) * (R(1) + x * R(1.0 / 3.0) * (R(1) + x * R(0.25) * (R(1) + x * R(0.2) * (R(1) + x * R(1.0 / 6.0))))));
}
// FP32 reciprocal, reciprocal square root and division as the single
// approximate hardware instructions (about 1-2 ulp, denormals flushed): their
// arguments here are squared norms, radii and ratios of per-step increments,
// never denormal, and the results enter quantities compared with the FP64
// oracle at 1e-5 relative
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float fdiv(float a, float b) {
  float y;
  asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

template <typename R, typename M, typename Get>
__device__ __forceinline__ R interp(const M &m, Get g, int i, R wi, int j, R wj) {
  const R a0 = g(m, i, j), a1 = g(m, i, j + 1), b0 = g(m, i + 1, j), b1 = g(m, i + 1, j + 1);
  const R lo = a0 + wj * (a1 - a0), hi = b0 + wj * (b1 - b0);
  return lo + wi * (hi - lo);
}

template <typename R, typename M>
__device__ __forceinline__ void gather(const M &m, int nr, int nt, int i, int j, R xo, R yo, R e[3], R b[3]) {
  // the four (node | half) x (node | half) weight sets, each shared by the
  // components that live there
  int kin, kih, kjn, kjh;
  R win, wih, wjn, wjh;
  stag(i, xo, false, nr + 1, kin, win);
  stag(i, xo, true, nr, kih, wih);
  stag(j, yo, false, nt + 1, kjn, wjn);
  stag(j, yo, true, nt, kjh, wjh);
  e[0] = interp(m, [](const M &q, int a, int c) { return q.er(a, c); }, kih, wih, kjn, wjn);
  b[1] = interp(m, [](const M &q, int a, int c) { return q.bt(a, c); }, kih, wih, kjn, wjn);
  e[1] = interp(m, [](const M &q, int a, int c) { return q.et(a, c); }, kin, win, kjh, wjh);
  b[0] = interp(m, [](const M &q, int a, int c) { return q.br(a, c); }, kin, win, kjh, wjh);
  e[2] = interp(m, [](const M &q, int a, int c) { return q.ep(a, c); }, kin, win, kjn, wjn);
  b[2] = interp(m, [](const M &q, int a, int c) { return q.bp(a, c); }, kih, wih, kjh, wjh);
}

// Shared-memory versions of the gather and the deposit: every access is a
// constant offset from one base offset per weight set, and the staged
// region replicates the edge values of each array, which reproduces the
// constant extrapolation of stag() without clamping.
template <typename R>
__device__ __forceinline__ R lerp4(const R *a, int o, int lt, R wi, R wj) {
  const R a0 = a[o], a1 = a[o + 1], b0 = a[o + lt], b1 = a[o + lt + 1];
  const R lo = a0 + wj * (a1 - a0), hi = b0 + wj * (b1 - b0);
  return lo + wi * (hi - lo);
}

template <typename R>
__device__ __forceinline__ void gather_sh(const SharedMesh<R> &m, int i, int j, R xo, R yo, R e[3], R b[3]) {
  const bool hx = xo >= R(0.5), hy = yo >= R(0.5);
  const int oc = m.o(i, j);
  const int onn = oc, onh = oc - (hy ? 0 : 1), ohn = oc - (hx ? 0 : m.lt), ohh = ohn - (hy ? 0 : 1);
  const R win = xo, wjn = yo, wih = hx ? xo - R(0.5) : xo + R(0.5), wjh = hy ? yo - R(0.5) : yo + R(0.5);
  const int lt = m.lt;
  e[0] = lerp4(m.s_er, ohn, lt, wih, wjn);
  b[1] = lerp4(m.s_bt, ohn, lt, wih, wjn);
  e[1] = lerp4(m.s_et, onh, lt, win, wjh);
  b[0] = lerp4(m.s_br, onh, lt, win, wjh);
  e[2] = lerp4(m.s_ep, onn, lt, win, wjn);
  b[2] = lerp4(m.s_bp, ohh, lt, wih, wjh);
}

// Modified Boris step (Eqs. 15-17, c = 1): Lorentz Boris gives u_L, the
// radiation-reaction kick K F_RR is evaluated at the time-centred momentum
// (u + u_L)/2 and limited to half of |u_L| per step.  Bperp^2 of Eq. 17 is
// evaluated as |F x beta|^2 + |F|^2 / gamma^2 with F = E + beta x B, which
// equals |F|^2 - (beta.F)^2 = |F|^2 - (beta.E)^2 without cancellation.
template <typename R>
__device__ __forceinline__ void boris_rr(R qm, R krr, R dt, const R u[3], const R e[3], const R b[3],
                                         R out[3], R &dgam) {
  const R a = R(0.5) * qm * dt;
  const R um0 = u[0] + a * e[0], um1 = u[1] + a * e[1], um2 = u[2] + a * e[2];
  const R ig = rsq(R(1) + um0 * um0 + um1 * um1 + um2 * um2);
  const R t0 = a * b[0] * ig, t1 = a * b[1] * ig, t2 = a * b[2] * ig;
  const R sc = R(2) * rcp(R(1) + t0 * t0 + t1 * t1 + t2 * t2);
  const R s0 = sc * t0, s1 = sc * t1, s2 = sc * t2;
  const R v0 = um0 + (um1 * t2 - um2 * t1), v1 = um1 + (um2 * t0 - um0 * t2), v2 = um2 + (um0 * t1 - um1 * t0);
  const R ul0 = um0 + (v1 * s2 - v2 * s1) + a * e[0];
  const R ul1 = um1 + (v2 * s0 - v0 * s2) + a * e[1];
  const R ul2 = um2 + (v0 * s1 - v1 * s0) + a * e[2];
  out[0] = ul0; out[1] = ul1; out[2] = ul2;
  dgam = R(0);
  if (krr != R(0)) {
    const R ub0 = R(0.5) * (u[0] + ul0), ub1 = R(0.5) * (u[1] + ul1), ub2 = R(0.5) * (u[2] + ul2);
    const R g2 = R(1) + ub0 * ub0 + ub1 * ub1 + ub2 * ub2;
    const R ig2 = rsq(g2);
    const R be0 = ub0 * ig2, be1 = ub1 * ig2, be2 = ub2 * ig2;
    const R f0 = e[0] + (be1 * b[2] - be2 * b[1]);
    const R f1 = e[1] + (be2 * b[0] - be0 * b[2]);
    const R f2 = e[2] + (be0 * b[1] - be1 * b[0]);
    const R c0 = f1 * be2 - f2 * be1, c1 = f2 * be0 - f0 * be2, c2 = f0 * be1 - f1 * be0;
    const R ff = f0 * f0 + f1 * f1 + f2 * f2;
    const R bp2 = c0 * c0 + c1 * c1 + c2 * c2 + ff * ig2 * ig2;
    const R bdot = be0 * e[0] + be1 * e[1] + be2 * e[2];
    const R k = dt * krr;
    const R du0 = k * ((f1 * b[2] - f2 * b[1]) + bdot * e[0] - g2 * bp2 * be0);
    const R du1 = k * ((f2 * b[0] - f0 * b[2]) + bdot * e[1] - g2 * bp2 * be1);
    const R du2 = k * ((f0 * b[1] - f1 * b[0]) + bdot * e[2] - g2 * bp2 * be2);
    const R dn2 = du0 * du0 + du1 * du1 + du2 * du2, ul2s = ul0 * ul0 + ul1 * ul1 + ul2 * ul2;
    const R lim = (dn2 > R(0.25) * ul2s) ? R(0.5) * rsq(dn2 * rcp(ul2s)) : R(1);
    out[0] = ul0 + lim * du0;
    out[1] = ul1 + lim * du1;
    out[2] = ul2 + lim * du2;
    const R gl = R(1) + ul2s, go = R(1) + out[0] * out[0] + out[1] * out[1] + out[2] * out[2];
    dgam = gl * rsq(gl) - go * rsq(go);
  }
}

// Straight-line move x' = x + (u/gamma) c dt in the local Cartesian frame at
// azimuth 0; the azimuthal displacement is rotated away (axisymmetry) and u
// re-expressed in the basis of the new point.  Increments only, no
// subtraction of absolute radii.  General form (any displacement).
template <typename R>
__device__ __forceinline__ void move_general(R r, R sn, R cs, R dt, const R u[3], R &dr, R &dth, R uo[3]) {
  const R ig = dt / sqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const R d0 = u[0] * ig, d1 = u[1] * ig, d2 = u[2] * ig;
  const R x = (r + d0) * sn + d1 * cs;
  const R rc = sqrt(x * x + d2 * d2);
  const R dR = (x > R(0)) ? d2 * d2 / (rc + x) : rc - x;
  const R pa = d0 + dR * sn;
  const R a = r + pa, bb = d1 + dR * cs;
  const R rnew = sqrt(a * a + bb * bb);
  dr = (pa * (R(2) * r + pa) + bb * bb) / (rnew + r);
  const R al = atan2(bb, a);
  const R ph = atan2(d2, x);
  dth = al;
  const R uR = u[0] * sn + u[1] * cs;
  R sp, cp, sa, ca;
  sincos(ph, &sp, &cp);
  sincos(al, &sa, &ca);
  const R s1 = sn * ca + cs * sa, c1 = cs * ca - sn * sa;  // angle of the new point
  const R h = sin(R(0.5) * ph);
  const R duR = uR * (R(-2) * h * h) + u[2] * sp;
  uo[0] = u[0] * ca + u[1] * sa + duR * s1;
  uo[1] = -u[0] * sa + u[1] * ca + duR * c1;
  uo[2] = -uR * sp + u[2] * cp;
}

// The same move for the usual case of a displacement much smaller than the
// distance to the axis (|d_phi| < 0.03 X and |b| < 0.03 a), where both
// rotation angles are small: with t = tan(angle), cos = 1/sqrt(1+t^2),
// sin = t cos and 1 - cos = t^2 / (sqrt(1+t^2)(sqrt(1+t^2)+1)) exactly, and
// the angle itself from the Taylor series of atan.  Returns false (nothing
// written) when the displacement is not small.
template <typename R>
__device__ __forceinline__ bool move_small(R r, R sn, R cs, R dt, const R u[3], R &dr, R &dth, R uo[3]) {
  const R ig = dt * rsq(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const R d0 = u[0] * ig, d1 = u[1] * ig, d2 = u[2] * ig;
  const R x = (r + d0) * sn + d1 * cs;
  if (!(x > R(0)) || fabs(d2) >= R(kSmall) * x) return false;
  const R tp = fdiv(d2, x), qp = tp * tp;
  const R cp = rsq(R(1) + qp), sqp = (R(1) + qp) * cp;
  const R sp = tp * cp, omc = fdiv(qp, sqp * (sqp + R(1)));  // 1 - cos(phi)
  const R dR = x * omc * sqp;                                // sqrt(x^2+d2^2) - x
  const R pa = d0 + dR * sn;
  const R a = r + pa, bb = d1 + dR * cs;
  if (fabs(bb) >= R(kSmall) * a) return false;
  const R ta = fdiv(bb, a), qa = ta * ta;
  const R ca = rsq(R(1) + qa), sqa = (R(1) + qa) * ca, sa = ta * ca;
  const R rnew = a * sqa;
  dr = fdiv(pa * (R(2) * r + pa) + bb * bb, rnew + r);
  dth = atan_small(ta);
  const R uR = u[0] * sn + u[1] * cs;
  const R s1 = sn * ca + cs * sa, c1 = cs * ca - sn * sa;
  const R duR = -uR * omc + u[2] * sp;
  uo[0] = u[0] * ca + u[1] * sa + duR * s1;
  uo[1] = -u[0] * sa + u[1] * ca + duR * c1;
  uo[2] = -uR * sp + u[2] * cp;
  return true;
}

// Charge-conserving deposit for linear shapes (Esirkepov decomposition) in
// the logical (xi, eta) plane.  (x0, y0) in [0,1) is the start offset in cell
// (i0, j0) and (X1, Y1) the end point relative to node (i0, j0), in (-1, 2).
// With S0, S1 the start and end weights on the nodes i0-1 .. i0+2 and
// dS = S1 - S0, the charge through the radial dual face between nodes a and
// a+1 in row b is -q (dS_x[0] + .. + dS_x[a]) (S0_y[b] + S1_y[b]) / 2, and
// likewise in theta; J_ph uses the mid-point weights.  For linear weights the
// nonzero radial fluxes always lie in a 2-face x 3-row window (and the polar
// ones in a 3 x 2 window) placed by the direction of any cell crossing, so
// every particle runs the same 16 predicated updates, with no data-dependent
// loops.  The accessor receives raw charge fluxes (charge x velocity for
// J_ph); the face areas, node volumes and dt are applied where the flux
// reaches global memory.
template <typename R>
struct Axis {  // weights along one direction
  R f0, f1;       // prefix-summed dS on the two faces of the window
  R m0, m1, m2;   // (S0 + S1) / 2 on the three nodes of the window
  int a0;         // window start relative to node i0 - 1 (0 or 1)
};

template <typename R>
__device__ __forceinline__ Axis<R> axis_weights(R x0, R X1) {
  Axis<R> w;
  const bool lo = X1 < R(0), hi = X1 >= R(1);
  // end weights on the nodes -1, 0, 1, 2 (relative to the start node)
  const R e0 = lo ? -X1 : R(0);
  const R e1 = lo ? R(1) + X1 : (hi ? R(0) : R(1) - X1);
  const R e2 = lo ? R(0) : (hi ? R(2) - X1 : X1);
  const R e3 = hi ? X1 - R(1) : R(0);
  // prefix sums of dS = e - (0, 1 - x0, x0, 0) on the faces -1/2, 1/2, 3/2;
  // inside one cell the middle one is -(X1 - x0) exactly
  const R p0 = e0;
  const R p1 = (lo || hi) ? e0 + e1 - (R(1) - x0) : x0 - X1;
  const R p2 = hi ? p1 + e2 - x0 : R(0);  // zero without a crossing (exactly)
  // weights (S0 + S1)/2 on the nodes -1 .. 2
  const R n0 = R(0.5) * e0, n1 = R(0.5) * (e1 + R(1) - x0), n2 = R(0.5) * (e2 + x0), n3 = R(0.5) * e3;
  w.a0 = lo ? 0 : 1;
  w.f0 = lo ? p0 : p1;
  w.f1 = lo ? p1 : p2;
  w.m0 = lo ? n0 : n1;
  w.m1 = lo ? n1 : n2;
  w.m2 = lo ? n2 : n3;
  return w;
}

// With `runs` (a work item whose particles sit cell by cell, decided once
// per item), lanes of a warp that deposit into the same windows (equal J_r
// / J_th window base and equal J_ph base) and sit next to each other form a
// run; with at least kRunMin such neighbours in the warp, a segmented scan
// sums each run's 16 site values and only the run's last lane issues the
// shared atomics.  FP32 (and FP64) shared atomic adds are retry loops of
// about six instructions on this GPU, which serialise on equal addresses: particles of one
// cell next to each other in memory (co-located injected pairs, or any
// cell-coherent order) otherwise cost one retry per lane and site (a
// cell-ordered 4096^2 workload measured 2.7x the push time of a scattered
// order).
constexpr int kRunMin = 4;
constexpr int kRunItemMin = 16;  // equal neighbour cells among 256 sampled pairs of a work item
template <typename R>
__device__ __forceinline__ void deposit_sh_runs(const SharedMesh<R> &m, R qw, int i0, int j0, R x0, R y0, R X1,
                                                R Y1, R vphi) {
  const Axis<R> ax = axis_weights(x0, X1), ay = axis_weights(y0, Y1);
  const R nq = -qw;
  const int lt = m.lt;
  const int ob = m.o(i0 - 1 + ax.a0, j0 - 1 + ay.a0);
  R v[16];
  {
    const R g0 = nq * ax.f0, g1 = nq * ax.f1;
    v[0] = g0 * ay.m0; v[1] = g0 * ay.m1; v[2] = g0 * ay.m2;
    v[3] = g1 * ay.m0; v[4] = g1 * ay.m1; v[5] = g1 * ay.m2;
  }
  {
    const R g0 = nq * ay.f0, g1 = nq * ay.f1;
    v[6] = g0 * ax.m0; v[7] = g0 * ax.m1; v[8] = g0 * ax.m2;
    v[9] = g1 * ax.m0; v[10] = g1 * ax.m1; v[11] = g1 * ax.m2;
  }
  int op;
  {
    const R xm = R(0.5) * (x0 + X1), ym = R(0.5) * (y0 + Y1);
    const int km = (xm < R(0)) ? -1 : (xm < R(1) ? 0 : 1);
    const int lm = (ym < R(0)) ? -1 : (ym < R(1) ? 0 : 1);
    const R wx = xm - R(km), wy = ym - R(lm);
    const R qv = qw * vphi;
    const R a0 = qv * (R(1) - wx), a1 = qv * wx;
    v[12] = a0 * (R(1) - wy); v[13] = a0 * wy; v[14] = a1 * (R(1) - wy); v[15] = a1 * wy;
    op = m.o(i0 + km, j0 + lm);
  }
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  const int pob = __shfl_up_sync(act, ob, 1), pop = __shfl_up_sync(act, op, 1);
  const bool cont = lane > 0 && ((act >> (lane - 1)) & 1u) && pob == ob && pop == op;
  const unsigned conts = __ballot_sync(act, cont);
  if (__popc(conts) >= kRunMin) {  // the same decision in every lane of act
    // a run starts at every lane that does not continue its predecessor
    // (inactive lanes included), so a run holds active lanes only
    const unsigned upto = (lane == 31) ? 0xffffffffu : ((2u << lane) - 1u);
    const int start = 31 - __clz(~conts & upto);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const R y = __shfl_up_sync(act, v[k], d);
        if (lane - d >= start) v[k] += y;
      }
    }
    if (lane < 31 && ((conts >> (lane + 1)) & 1u)) return;  // not the run's last lane
  }
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (v[k] != R(0)) atomicAdd(&m.s_jr[ob + (k / 3) * lt + k % 3], v[k]);
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (v[6 + k] != R(0)) atomicAdd(&m.s_jt[ob + (k % 3) * lt + k / 3], v[6 + k]);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (v[12 + k] != R(0)) atomicAdd(&m.s_jp[op + (k / 2) * lt + k % 2], v[12 + k]);
}

template <typename R>
__device__ __forceinline__ void deposit_sh(const SharedMesh<R> &m, R qw, int i0, int j0, R x0, R y0, R X1, R Y1,
                                           R vphi, bool runs) {
  if (runs) {
    deposit_sh_runs<R>(m, qw, i0, j0, x0, y0, X1, Y1, vphi);
    return;
  }
  const Axis<R> ax = axis_weights(x0, X1), ay = axis_weights(y0, Y1);
  const R nq = -qw;
  const int lt = m.lt;
  const int ob = m.o(i0 - 1 + ax.a0, j0 - 1 + ay.a0);
  {
    const R g0 = nq * ax.f0, g1 = nq * ax.f1;
    const R v[6] = {g0 * ay.m0, g0 * ay.m1, g0 * ay.m2, g1 * ay.m0, g1 * ay.m1, g1 * ay.m2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (v[k] != R(0)) atomicAdd(&m.s_jr[ob + (k / 3) * lt + k % 3], v[k]);
  }
  {
    const R g0 = nq * ay.f0, g1 = nq * ay.f1;
    const R v[6] = {g0 * ax.m0, g0 * ax.m1, g0 * ax.m2, g1 * ax.m0, g1 * ax.m1, g1 * ax.m2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (v[k] != R(0)) atomicAdd(&m.s_jt[ob + (k % 3) * lt + k / 3], v[k]);
  }
  {
    const R xm = R(0.5) * (x0 + X1), ym = R(0.5) * (y0 + Y1);
    const int km = (xm < R(0)) ? -1 : (xm < R(1) ? 0 : 1);
    const int lm = (ym < R(0)) ? -1 : (ym < R(1) ? 0 : 1);
    const R wx = xm - R(km), wy = ym - R(lm);
    const R qv = qw * vphi;
    const R a0 = qv * (R(1) - wx), a1 = qv * wx;
    const R v[4] = {a0 * (R(1) - wy), a0 * wy, a1 * (R(1) - wy), a1 * wy};
    const int op = m.o(i0 + km, j0 + lm);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (v[k] != R(0)) atomicAdd(&m.s_jp[op + (k / 2) * lt + k % 2], v[k]);
  }
}

template <typename R, typename M>
__device__ __forceinline__ void deposit(const M &m, R qw, int i0, int j0, R x0, R y0, R X1, R Y1, R vphi) {
  const Axis<R> ax = axis_weights(x0, X1), ay = axis_weights(y0, Y1);
  const R nq = -qw;
  const int ib = i0 - 1 + ax.a0, jb = j0 - 1 + ay.a0;
  // radial faces ib, ib+1 (E_r rows) x nodes jb .. jb+2
  {
    const R g0 = nq * ax.f0, g1 = nq * ax.f1;
    const R v[6] = {g0 * ay.m0, g0 * ay.m1, g0 * ay.m2, g1 * ay.m0, g1 * ay.m1, g1 * ay.m2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (v[k] != R(0)) m.add_jr(ib + k / 3, jb + k % 3, v[k]);
  }
  // polar faces jb, jb+1 (E_th columns) x nodes ib .. ib+2
  {
    const R g0 = nq * ay.f0, g1 = nq * ay.f1;
    const R v[6] = {g0 * ax.m0, g0 * ax.m1, g0 * ax.m2, g1 * ax.m0, g1 * ax.m1, g1 * ax.m2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (v[k] != R(0)) m.add_jt(ib + k % 3, jb + k / 3, v[k]);
  }
  // J_ph at the mid-point
  {
    const R xm = R(0.5) * (x0 + X1), ym = R(0.5) * (y0 + Y1);
    const int km = (xm < R(0)) ? -1 : (xm < R(1) ? 0 : 1);
    const int lm = (ym < R(0)) ? -1 : (ym < R(1) ? 0 : 1);
    const R wx = xm - R(km), wy = ym - R(lm);
    const R qv = qw * vphi;
    const R a0 = qv * (R(1) - wx), a1 = qv * wx;
    const R v[4] = {a0 * (R(1) - wy), a0 * wy, a1 * (R(1) - wy), a1 * wy};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (v[k] != R(0)) m.add_jp(i0 + km + k / 2, j0 + lm + k % 2, v[k]);
  }
}

template <typename R> __device__ __forceinline__ R one_minus_ulp();
template <> __device__ __forceinline__ float one_minus_ulp<float>() { return 0.99999994f; }
template <> __device__ __forceinline__ double one_minus_ulp<double>() { return 0.99999999999999989; }

// per-thread counters in the working precision (FP64 only in the warp and
// global sums)
template <typename R>
struct Tally {
  R killed, radiated;
  unsigned nonfinite;
  unsigned pushed;
};

// per-species constants of a push, loaded once per work item.  In (read)
// and S (written) are the same arrays, except in the first push after a sort,
// which reads the unsorted parity through the sorted order sidx.
template <typename R>
struct SpeciesConst {
  Species<R> S, In;
  const uint32_t *sidx;
  R qm, krr, q, m;
  uint32_t key_hi;   // species in the top bit of a pair-creation event key
  bool creates;      // a lepton of a run with pair creation
  __device__ __forceinline__ SpeciesConst(const Params<R> &p, int s, bool gather = false)
      : S(p.sp[s]), In(gather ? p.src[s] : p.sp[s]), sidx(p.sidx[s]), qm(p.qm[s]),
        krr(p.krr[s] * (R)(*p.rr_scale)), q(p.q[s]), m(p.m[s]), key_hi((uint32_t)s << 31),
        creates(p.pairs != 0 && s < 2) {}
};

// Sect. 5.1: a lepton above the threshold Lorentz factor creates a pair at
// its new position, along its direction of motion, with gamma_s.  Recorded
// as an event here (slot order of the atomic is arbitrary; the key restores
// the parent order when the pairs are appended).
template <typename R>
__device__ __forceinline__ void record_pair(const Params<R> &p, const SpeciesConst<R> &K, int q, int cell, R xn,
                                            R yn, const R uo[3], R w) {
  const R u2 = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
  if (!(R(1) + u2 > p.gamma_th2)) return;
  const unsigned e = atomicAdd(p.pe_count, 1u);
  if ((int64_t)e >= p.pe_cap) { atomicOr(p.status, kStCapacity); return; }
  const R a = p.u_s * rsq(u2);
  p.ev_key[e] = K.key_hi | (uint32_t)q;
  p.ev_cell[e] = cell;
  p.ev_xo[e] = xn; p.ev_yo[e] = yn;
  p.ev_ur[e] = a * uo[0]; p.ev_ut[e] = a * uo[1]; p.ev_up[e] = a * uo[2];
  p.ev_w[e] = w;
}

// One particle: gather, push, move, kill rules, deposit, store.  Reads
// particle qi of K.In and writes slot q of K.S (the same particle unless the
// push also performs a sort's payload gather, kGather, which writes w too).
template <typename R, bool kGather, typename M>
__device__ __forceinline__ void push_one(const M &m, const Params<R> &p, const SpeciesConst<R> &K, int q,
                                         int qi, int i, int j, Tally<R> &tl, bool runs = false) {
  constexpr bool kShared = std::is_same<M, SharedMesh<R>>::value;
  const Species<R> &S = K.S;
  const Species<R> &In = K.In;
  const int nt = p.nt, nr = p.nr;
  const R xo = In.xo[qi], yo = In.yo[qi], w = In.w[qi];
  R u[3] = {In.ur[qi], In.ut[qi], In.up[qi]};
  R e[3], b[3], un[3], dg;
  tl.pushed += 1;
  if constexpr (kShared) gather_sh<R>(m, i, j, xo, yo, e, b);
  else gather<R>(m, nr, nt, i, j, xo, yo, e, b);
  boris_rr<R>(K.qm, K.krr, p.dt, u, e, b, un, dg);
  tl.radiated += w * K.m * dg;
  // position of the particle: r = r_i exp(xo D), theta = theta_j + yo dtheta
  const R xl = xo * p.dlog, ya = yo * p.dth;
  R ex, sa0, ca0;
  if (p.small_grid) {
    ex = exp_small(xl);
    sa0 = sin_small(ya);
    ca0 = cos_small(ya);
  } else {
    ex = exp(xl);
    sincos(ya, &sa0, &ca0);
  }
  const R r = m.rn(i) * ex;
  const R snj = m.sn(j), cnj = m.cn(j);
  const R sn = snj * ca0 + cnj * sa0, cs = cnj * ca0 - snj * sa0;
  if (r * r < p.shell_r2) {  // Sect. 5.1: no momentum across B near the star
    const R b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (b2 > R(1e-30)) {
      const R ub = (un[0] * b[0] + un[1] * b[1] + un[2] * b[2]) * rcp(b2);
      un[0] = ub * b[0]; un[1] = ub * b[1]; un[2] = ub * b[2];
    }
  }
  R dr, dth, uo[3];
  if (!move_small<R>(r, sn, cs, p.dt, un, dr, dth, uo)) move_general<R>(r, sn, cs, p.dt, un, dr, dth, uo);
  const R ginv = rsq(R(1) + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
  const R xr = dr * rcp(r);
  R X1 = xo + ((fabs(xr) < R(kSmall)) ? log1p_small(xr) : log1p(xr)) * p.inv_dlog;
  R Y1 = yo + dth * p.inv_dth;
  if (!isfinite(X1) || !isfinite(Y1) || !isfinite(uo[0] + uo[1] + uo[2])) {
    S.cell[q] = -1;
    tl.nonfinite += 1;
    return;
  }
  if (R(j) + Y1 < R(0)) Y1 = R(-2 * j) - Y1;
  if (R(j) + Y1 > R(nt)) Y1 = R(2 * (nt - j)) - Y1;
  bool dead = false;
  if (R(i) + X1 < R(0)) { X1 = -R(i); dead = true; }
  else if (R(i) + X1 > p.xi_abs) dead = true;
  int di = (int)floor(X1), dj = (int)floor(Y1);
  R xn = X1 - R(di), yn = Y1 - R(dj);
  if (xn >= R(1)) { xn -= R(1); di += 1; }
  if (yn >= R(1)) { yn -= R(1); dj += 1; }
  const int i1 = i + di;
  int j1 = j + dj;
  if (j1 >= nt) { j1 = nt - 1; yn = one_minus_ulp<R>(); }
  if (!dead && m.ff(i1, j1)) dead = true;
  if constexpr (kShared) deposit_sh<R>(m, K.q * w, i, j, xo, yo, X1, Y1, un[2] * ginv, runs);
  else deposit<R>(m, K.q * w, i, j, xo, yo, X1, Y1, un[2] * ginv);
  if (dead) {
    S.cell[q] = -1;
    tl.killed += w;
    return;
  }
  S.cell[q] = i1 * nt + j1;
  S.xo[q] = xn; S.yo[q] = yn;
  S.ur[q] = uo[0]; S.ut[q] = uo[1]; S.up[q] = uo[2];
  if constexpr (kGather) S.w[q] = w;
  if (i1 == 0 && p.inject) atomicAdd(&p.surf[j1], 1);
  if (K.creates) record_pair(p, K, q, i1 * nt + j1, xn, yn, uo, w);
}

// out-of-region fallback of the tiled kernel.  It returns its counts by
// value and takes the species index rather than the species constants:
// arguments passed by reference to an out-of-line call would have to live
// in local memory for the whole work item.
template <typename R, bool kGather>
__device__ __forceinline__ Tally<R> push_one_global(const Params<R> &p, int s, int q, int qi, int i, int j) {
  const SpeciesConst<R> K(p, s, kGather);
  GlobalMesh<R> g(p);
  Tally<R> tl{R(0), R(0), 0u, 0u};
  push_one<R, kGather>(g, p, K, q, qi, i, j, tl);
  return tl;
}

template <typename R>
__device__ __forceinline__ void flush_tally(const Tally<R> &tl, double *acc, unsigned *status,
                                            unsigned long long *pushed) {
  double k = tl.killed, r = tl.radiated;  // FP64 only for the warp and global sums
  unsigned nf = tl.nonfinite, np = tl.pushed;
  for (int o = 16; o > 0; o >>= 1) {
    k += __shfl_down_sync(0xffffffffu, k, o);
    r += __shfl_down_sync(0xffffffffu, r, o);
    nf += __shfl_down_sync(0xffffffffu, nf, o);
    np += __shfl_down_sync(0xffffffffu, np, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (k != 0.0) atomicAdd(&acc[1], k);
    if (r != 0.0) atomicAdd(&acc[2], r);
    if (nf) { atomicAdd(&acc[3], (double)nf); atomicOr(status, kStNonfinite); }
    if (np) atomicAdd(pushed, (unsigned long long)np);
  }
}

// ----------------------------------------------------------- tail kernel
template <typename R>
__global__ void __launch_bounds__(256) k_push_tail(Params<R> p) {
  GlobalMesh<R> m(p);
  Tally<R> tl{R(0), R(0), 0u, 0u};
  for (int s = 0; s < p.n_species; ++s) {
    const SpeciesConst<R> K(p, s);
    const int64_t n0 = p.count_sorted[s], n1 = p.count[s];
    for (int64_t q = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n1;
         q += (int64_t)gridDim.x * blockDim.x) {
      const int c = p.sp[s].cell[q];
      if (c < 0) continue;
      int i, j;
      decode_cell(p, c, i, j);
      push_one<R, false>(m, p, K, (int)q, (int)q, i, j, tl);
    }
  }
  flush_tally(tl, p.acc, p.status, &p.pushed[1]);
}

// ---------------------------------------------------------- tiled kernel
// Region of a tile: cells [ti*TR - H, (ti+1)*TR + H) (and likewise in theta)
// widened by the stencil: one node below, two above.
// Register budget: five blocks of 256 per SM in FP32 (48 registers, a few
// spilled values in L1; the region of a 16 x 24 tile fits five times in
// shared memory), three in FP64, whose doubled region leaves room for no more.
template <typename R> constexpr int push_tiled_min_blocks() { return sizeof(R) == 4 ? 5 : 3; }
template <typename R, bool kGather>
__global__ void __launch_bounds__(256, push_tiled_min_blocks<R>())
    k_push_tiled(const __grid_constant__ Params<R> p, WorkList wl, int halo) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lr = p.tile_r + 2 * halo + 4, lt = p.tile_t + 2 * halo + 4, area = lr * lt;
  R *base = reinterpret_cast<R *>(smem);
  SharedMesh<R> m;
  m.s_er = base; m.s_et = base + area; m.s_ep = base + 2 * area;
  m.s_br = base + 3 * area; m.s_bt = base + 4 * area; m.s_bp = base + 5 * area;
  m.s_jr = base + 6 * area; m.s_jt = base + 7 * area; m.s_jp = base + 8 * area;
  m.s_rn = base + 9 * area; m.s_sn = m.s_rn + lr; m.s_cn = m.s_sn + lt;
  m.s_ff = reinterpret_cast<uint8_t *>(m.s_cn + lt);
  m.lt = lt;
  __shared__ int s_item;
  const int nr = p.nr, nt = p.nt, n1 = nt + 1;
  Tally<R> tl{R(0), R(0), 0u, 0u};
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(wl.next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= *wl.n_items) break;
    const int4 item = wl.items[it];
    const int s = item.x, tile = item.y;
    const int ti = tile / p.ntt, tj = tile - ti * p.ntt;
    m.i0 = ti * p.tile_r - halo - 1;
    m.j0 = tj * p.tile_t - halo - 1;
    // stage E, B, flags (edge values replicated outside each array); clear J
    for (int k = threadIdx.x; k < area; k += blockDim.x) {
      const int a = k / lt, c = k - a * lt;
      const int gi = m.i0 + a, gj = m.j0 + c;
      const int in = min(max(gi, 0), nr), ih = min(max(gi, 0), nr - 1);   // node / half rows
      const int jn = min(max(gj, 0), nt), jh = min(max(gj, 0), nt - 1);   // node / half columns
      m.s_er[k] = p.f.er[ix(ih, jn, n1)];
      m.s_et[k] = p.f.et[ix(in, jh, nt)];
      m.s_ep[k] = p.f.ep[ix(in, jn, n1)];
      const int64_t kb = ix(in, jh, nt), kt = ix(ih, jn, n1), kp = ix(ih, jh, nt);
      m.s_br[k] = p.f.br0[kb] + p.f.br[kb];   // B = B_0 + dB
      m.s_bt[k] = p.f.bt0[kt] + p.f.bt[kt];
      m.s_bp[k] = p.f.bp0[kp] + p.f.bp[kp];
      m.s_ff[k] = (gi >= 0 && gj >= 0 && gi < nr && gj < nt) ? p.f.ffcell[ix(gi, gj, nt)] : 1;
      m.s_jr[k] = R(0); m.s_jt[k] = R(0); m.s_jp[k] = R(0);
    }
    for (int k = threadIdx.x; k < lr; k += blockDim.x) {
      const int gi = m.i0 + k;
      m.s_rn[k] = (gi >= 0 && gi <= nr) ? p.t.rn[gi] : R(1);
    }
    for (int k = threadIdx.x; k < lt; k += blockDim.x) {
      const int gj = m.j0 + k;
      m.s_sn[k] = (gj >= 0 && gj <= nt) ? p.t.sn[gj] : R(0);
      m.s_cn[k] = (gj >= 0 && gj <= nt) ? p.t.cn[gj] : R(1);
    }
    const SpeciesConst<R> K(p, s, kGather);
    const int q0 = item.z, q1 = item.z + item.w;
    // particles of one cell next to each other (co-located injected pairs
    // keep their order through the stable sort)?  Decided once per item from
    // blockDim.x neighbour pairs spread over it, so a scattered item pays
    // nothing in the deposit.
    int same = 0;
    {
      const int stride = max(1, (q1 - q0 - 1) / (int)blockDim.x);
      const int qa = q0 + 1 + (int)threadIdx.x * stride;
      if (qa < q1) {
        const int ca = K.In.cell[kGather ? (int)K.sidx[qa] : qa];
        const int cb = K.In.cell[kGather ? (int)K.sidx[qa - 1] : qa - 1];
        same = (ca == cb && ca >= 0) ? 1 : 0;
      }
    }
    const bool runs = __syncthreads_count(same) >= kRunItemMin;
    // the particles this thread visits: block-strided in a scattered item;
    // in a cell-coherent one every warp walks its own contiguous slice, so
    // that its lanes stay consecutive (the runs) while the warps work on
    // different cells (their atomics then rarely meet)
    int qs = q0 + (int)threadIdx.x, qe = q1, qstep = (int)blockDim.x;
    if (runs) {
      const int nw = (int)blockDim.x >> 5, w = (int)threadIdx.x >> 5;
      const int slice = ((q1 - q0 + nw - 1) / nw + 31) & ~31;
      qs = q0 + w * slice + ((int)threadIdx.x & 31);
      qe = min(q1, q0 + (w + 1) * slice);
      qstep = 32;
    }
    // a particle is handled in shared memory when its whole stencil (start
    // cell -1 .. +2 in both directions) lies inside the region
    for (int q = qs; q < qe; q += qstep) {
      const int qi = kGather ? (int)K.sidx[q] : q;
      const int c = K.In.cell[qi];
      if (c < 0) {
        if (kGather) K.S.cell[q] = -1;
        continue;
      }
      int i, j;
      decode_cell(p, c, i, j);
      if (i - 1 >= m.i0 && i + 2 < m.i0 + lr && j - 1 >= m.j0 && j + 2 < m.j0 + lt)
        push_one<R, kGather>(m, p, K, q, qi, i, j, tl, runs);
      else {
        const Tally<R> t = push_one_global<R, kGather>(p, s, q, qi, i, j);
        tl.killed += t.killed; tl.radiated += t.radiated;
        tl.nonfinite += t.nonfinite; tl.pushed += t.pushed;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < area; k += blockDim.x) {
      const int a = k / lt, c = k - a * lt;
      const int gi = m.i0 + a, gj = m.j0 + c;
      if (gi < 0 || gj < 0) continue;
      // raw fluxes -> current densities (face areas, node volumes, dt)
      if (m.s_jr[k] != R(0) && gi < nr && gj <= nt)
        atomicAdd(&p.f.jr[ix(gi, gj, n1)], m.s_jr[k] * p.t.dep_r[gi] * p.t.inv_dch[gj]);
      if (m.s_jt[k] != R(0) && gi <= nr && gj < nt)
        atomicAdd(&p.f.jt[ix(gi, gj, nt)], m.s_jt[k] * p.t.dep_t[gi] * p.t.inv_sh[gj]);
      if (m.s_jp[k] != R(0) && gi <= nr && gj <= nt)
        atomicAdd(&p.f.jp[ix(gi, gj, n1)], m.s_jp[k] * p.t.dep_p[gi] * p.t.inv_dch[gj]);
    }
    __syncthreads();
  }
  flush_tally(tl, p.acc, p.status, &p.pushed[0]);
}

template <typename R> size_t push_tiled_smem(const Params<R> &p, int halo) {
  const size_t lr = p.tile_r + 2 * halo + 4, lt = p.tile_t + 2 * halo + 4, area = lr * lt;
  return area * (9 * sizeof(R) + 1) + (lr + 2 * lt) * sizeof(R);
}

template <typename R> void launch_push_tail(const Params<R> &p, cudaStream_t s, int grid) {
  k_push_tail<R><<<grid, 256, 0, s>>>(p);
}
template <typename R> void launch_push_tiled(const Params<R> &p, const WorkList &wl, int halo,
                                             cudaStream_t s, int grid, bool gather) {
  if (gather) k_push_tiled<R, true><<<grid, 256, push_tiled_smem(p, halo), s>>>(p, wl, halo);
  else k_push_tiled<R, false><<<grid, 256, push_tiled_smem(p, halo), s>>>(p, wl, halo);
}

// ------------------------------------------------------------- injection
// Top-up of each eligible surface cell to its target (fixed at init from
// kappa n_GJ V / w, Sects. 4 and 5.1): n_new(j) = max(0, target_j - surf_j/2)
// co-located pairs, offsets from Philox4x32-10 keyed (seed; step, j, k),
// corotating momentum, appended in (j, k) order.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// one block: exclusive scan of the per-cell counts, reserve slots
template <typename R>
__global__ void __launch_bounds__(1024) k_inject_scan(Params<R> p) {
  __shared__ int s_w[32];
  __shared__ int s_carry;
  const int nt = p.nt;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int seg = 0; seg < nt; seg += blockDim.x) {
    const int j = seg + threadIdx.x;
    int v = 0;
    if (j < nt) {
      const int need = p.target[j] - p.surf[j] / 2;
      v = need > 0 ? need : 0;
      p.surf[j] = 0;  // consumed: cleared for the next step
    }
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    int off = s_carry;
    for (int w = 0; w < wid; ++w) off += s_w[w];
    if (j < nt) p.inj_prefix[j] = off + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = off + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int total = s_carry;
    p.inj_prefix[nt] = total;
    for (int k = 0; k < p.n_inj; ++k) {
      const int s = p.inj_sp[k];
      const long long base = p.count[s];
      p.inj_base[s] = base;
      long long end = base + total;
      if (end > p.cap) { end = p.cap; atomicOr(p.status, kStCapacity); }
      p.count[s] = end;
    }
    atomicAdd(&p.acc[0], (double)total * (double)p.w_inj * p.n_inj);
  }
}

template <typename R>
__global__ void __launch_bounds__(128) k_inject_write(Params<R> p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nt = p.nt;
  if (j < nt) {
    const int k0 = p.inj_prefix[j], n = p.inj_prefix[j + 1] - k0;
    const long long step = *p.step;
    for (int k = 0; k < n; ++k) {
      uint32_t c[4] = {(uint32_t)step, (uint32_t)((unsigned long long)step >> 32), (uint32_t)j, (uint32_t)k};
      philox4x32_10(c, p.seed_lo, p.seed_hi);
      const R ox = (R)(c[0] >> 8) * R(1.0 / 16777216.0);
      const R oy = (R)(c[1] >> 8) * R(1.0 / 16777216.0);
      const R r = p.t.rn[0] * exp(ox * p.dlog);
      const R v = p.omega * r * sin((R(j) + oy) * p.dth);
      const R uphi = v / sqrt(R(1) - v * v);
      for (int k2 = 0; k2 < p.n_inj; ++k2) {
        const int s = p.inj_sp[k2];
        const long long q = p.inj_base[s] + k0 + k;
        if (q >= p.count[s]) continue;  // capacity reached (flagged by the scan)
        Species<R> S = p.sp[s];
        S.cell[q] = j;
        S.xo[q] = ox; S.yo[q] = oy;
        S.ur[q] = R(0); S.ut[q] = R(0); S.up[q] = uphi;
        S.w[q] = p.w_inj;
      }
    }
  }
}

// The pairs of this step's events, appended to species 0 and 1 after the
// injected particles, in parent order (species 0 by slot, then species 1):
// each event is ranked by counting the smaller keys, for up to kRankMax
// events (a larger number, far beyond the parity cases, keeps the arbitrary
// event order).  One block.
constexpr int kRankMax = 4096;
template <typename R>
__global__ void __launch_bounds__(1024) k_pairs_append(Params<R> p) {
  __shared__ uint32_t skey[kRankMax];
  __shared__ long long base[2];
  __shared__ double wsum[32];
  const unsigned n_raw = *p.pe_count;
  const int64_t n = (int64_t)n_raw < p.pe_cap ? (int64_t)n_raw : p.pe_cap;
  const bool ranked = n <= kRankMax;
  if (threadIdx.x < 2) base[threadIdx.x] = p.count[threadIdx.x];
  if (ranked)
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) skey[e] = p.ev_key[e];
  __syncthreads();
  double ws = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int64_t rank = e;
    if (ranked) {
      const uint32_t k = skey[e];
      rank = 0;
      for (int64_t f = 0; f < n; ++f) rank += skey[f] < k;
    }
    ws += (double)p.ev_w[e];
    for (int s = 0; s < 2; ++s) {
      const int64_t q = base[s] + rank;
      if (q >= p.cap) continue;
      Species<R> S = p.sp[s];
      S.cell[q] = p.ev_cell[e];
      S.xo[q] = p.ev_xo[e]; S.yo[q] = p.ev_yo[e];
      S.ur[q] = p.ev_ur[e]; S.ut[q] = p.ev_ut[e]; S.up[q] = p.ev_up[e];
      S.w[q] = p.ev_w[e];
    }
  }
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_down_sync(0xffffffffu, ws, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
    for (int s = 0; s < 2; ++s) {
      long long end = base[s] + n;
      if (end > p.cap) { end = p.cap; atomicOr(p.status, kStCapacity); }
      p.count[s] = end;
    }
    p.acc[4] += 2.0 * t;
    *p.pe_count = 0u;
  }
}

template <typename R>
__global__ void k_step_done(Params<R> p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p.step += 1;
}

template <typename R> void launch_inject(const Params<R> &p, cudaStream_t s) {
  if (p.inject) {
    k_inject_scan<R><<<1, 1024, 0, s>>>(p);
    k_inject_write<R><<<(p.nt + 127) / 128, 128, 0, s>>>(p);
  }
  if (p.pairs) k_pairs_append<R><<<1, 1024, 0, s>>>(p);
  k_step_done<R><<<1, 32, 0, s>>>(p);
}
template <typename R> void launch_step_done(const Params<R> &p, cudaStream_t s) {
  k_step_done<R><<<1, 32, 0, s>>>(p);
}
template <typename R, bool G> const void *push_tiled_fn() { return reinterpret_cast<const void *>(&k_push_tiled<R, G>); }
template <typename R> cudaError_t set_push_smem(size_t bytes) {
  const cudaError_t e = raise_smem_limit<push_tiled_fn<R, false>>(bytes);
  return e != cudaSuccess ? e : raise_smem_limit<push_tiled_fn<R, true>>(bytes);
}
// resident blocks of the tiled push per SM with `bytes` of shared memory
// (registers and shared memory both counted); 0 on error
template <typename R> int push_tiled_blocks_per_sm(size_t bytes) {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_push_tiled<R, false>, 256, bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_push_tiled<R, true>, 256, bytes) != cudaSuccess)
    return 0;
  return a < b ? a : b;
}

#define HFF_INST(R)                                                                         \
  template size_t push_tiled_smem<R>(const Params<R> &, int);                               \
  template void launch_push_tail<R>(const Params<R> &, cudaStream_t, int);                  \
  template void launch_push_tiled<R>(const Params<R> &, const WorkList &, int, cudaStream_t, int, bool); \
  template void launch_inject<R>(const Params<R> &, cudaStream_t);                          \
  template void launch_step_done<R>(const Params<R> &, cudaStream_t);                       \
  template cudaError_t set_push_smem<R>(size_t);                                            \
  template int push_tiled_blocks_per_sm<R>(size_t);
HFF_INST(float)
HFF_INST(double)
#undef HFF_INST

}  // namespace hff
