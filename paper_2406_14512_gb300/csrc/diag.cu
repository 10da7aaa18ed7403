// diag.cu -- FP64 diagnostics of Sect. 4, on request only (not in the step):
// Psi in FP64 (Eq. 27), spin-down power L(r) through each half-node sphere
// (Eq. 35), Gauss's-law residual div E / 4 pi - rho on interior nodes, field
// energies, kinetic energy and live counts per species.
#include "diag.cuh"

namespace hff {

// Psi in FP64 at every node (one block per row)
template <typename R>
__global__ void __launch_bounds__(256) k_psi64(Params<R> p, double *out) {
  const int i = blockIdx.x, nt = p.nt;
  const R *br = p.f.br + (int64_t)i * nt, *br0 = p.f.br0 + (int64_t)i * nt;
  double *psi = out + (int64_t)i * (nt + 1);
  const double r2 = p.t.r2n[i];
  __shared__ double warp_tot[8];
  __shared__ double carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry = 0.0; psi[0] = 0.0; }
  __syncthreads();
  for (int seg = 0; seg < nt; seg += 256) {
    const int j = seg + threadIdx.x;
    double v = (j < nt) ? ((double)br0[j] + (double)br[j]) * p.t.dcp[j] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    double off = carry;
    for (int w = 0; w < wid; ++w) off += warp_tot[w];
    if (j < nt) psi[j + 1] = r2 * (off + v);
    __syncthreads();
    if (threadIdx.x == 255) carry = off + v;
    __syncthreads();
  }
}

// CIC node charges of the live particles (FP64 accumulation)
template <typename R>
__global__ void __launch_bounds__(256) k_node_charge(Params<R> p, double *q, double *kin, double *cnt) {
  const int nt = p.nt, n1 = nt + 1;
  for (int s = 0; s < p.n_species; ++s) {
    double ke = 0.0, c = 0.0;
    const int64_t n = p.count[s];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
      const int cell = p.sp[s].cell[k];
      if (cell < 0) continue;
      const int i = cell / nt, j = cell - (cell / nt) * nt;
      const double x = p.sp[s].xo[k], y = p.sp[s].yo[k], w = p.sp[s].w[k];
      const double qw = (double)p.q[s] * w;
      atomicAdd(&q[ix(i, j, n1)], qw * (1 - x) * (1 - y));
      atomicAdd(&q[ix(i + 1, j, n1)], qw * x * (1 - y));
      atomicAdd(&q[ix(i, j + 1, n1)], qw * (1 - x) * y);
      atomicAdd(&q[ix(i + 1, j + 1, n1)], qw * x * y);
      const double u0 = p.sp[s].ur[k], u1 = p.sp[s].ut[k], u2 = p.sp[s].up[k];
      ke += w * (double)p.m[s] * (sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2) - 1.0);
      c += 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      ke += __shfl_down_sync(0xffffffffu, ke, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(&kin[s], ke); atomicAdd(&cnt[s], c); }
  }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;
}
__device__ __forceinline__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, sh[w]);
  __syncthreads();
  return t;
}

// per row i (0..nr): [L(r_{i+1/2}), U_E part, U_B part, gauss max, gauss sum2,
// gauss count, rho max, unused], all FP64.  Geometry in FP64 from the row and
// column tables of the working precision, which were themselves rounded from
// FP64 (the relative error is that of R).
template <typename R>
__global__ void __launch_bounds__(256) k_diag_rows(Params<R> p, DiagGeom g, const double *q, double *rows) {
  __shared__ double sh[8];
  const int i = blockIdx.x, nr = p.nr, nt = p.nt, n1 = nt + 1;
  const Fields<R> &f = p.f;
  // B = B_0 + dB, summed in FP64
  auto Bt = [&](int64_t k) { return (double)f.bt0[k] + (double)f.bt[k]; };
  auto Bp = [&](int64_t k) { return (double)f.bp0[k] + (double)f.bp[k]; };
  auto Br = [&](int64_t k) { return (double)f.br0[k] + (double)f.br[k]; };
  double L = 0, ue = 0, ub = 0, gmax = 0, g2 = 0, gcnt = 0, rmax = 0, bad = 0;
  for (int j = threadIdx.x; j <= nt; j += blockDim.x) {
    // non-finite field values owned by (i, j) (failure detection)
    if (i < nr) {
      bad += !isfinite((double)f.er[ix(i, j, n1)]) + !isfinite((double)f.bt[ix(i, j, n1)]);
      if (j < nt) bad += !isfinite((double)f.bp[ix(i, j, nt)]);
    }
    if (j < nt) bad += !isfinite((double)f.et[ix(i, j, nt)]) + !isfinite((double)f.br[ix(i, j, nt)]);
    bad += !isfinite((double)f.ep[ix(i, j, n1)]);
    if (i < nr) {
      const double r = g.rh[i];
      if (j < nt) {
        const double et = 0.5 * ((double)f.et[ix(i, j, nt)] + (double)f.et[ix(i + 1, j, nt)]);
        L += et * Bp(ix(i, j, nt)) * 2 * kPi * r * r * g.dcp[j];
      }
      const double epm = 0.5 * ((double)f.ep[ix(i, j, n1)] + (double)f.ep[ix(i + 1, j, n1)]);
      L -= epm * Bt(ix(i, j, n1)) * 2 * kPi * r * r * g.dch[j];
      const double er = f.er[ix(i, j, n1)];
      ue += er * er * 2 * kPi * r * r * g.dch[j] * (g.rn[i + 1] - g.rn[i]);
      const double bt = Bt(ix(i, j, n1));
      ub += bt * bt * kPi * g.sn[j] * (g.rn[i + 1] * g.rn[i + 1] - g.rn[i] * g.rn[i]) * r * (g.thi[j] - g.tlo[j]);
      if (j < nt) {
        const double bp = Bp(ix(i, j, nt));
        ub += bp * bp * 0.5 * (g.rn[i + 1] * g.rn[i + 1] - g.rn[i] * g.rn[i]) * g.dth * 2 * kPi * r * g.sh[j];
      }
    }
    const double rlo = g.rlo[i], rhi = g.rhi[i], rni = g.rn[i];
    if (j < nt) {
      const double et = f.et[ix(i, j, nt)], br = Br(ix(i, j, nt));
      ue += et * et * kPi * g.sh[j] * (rhi * rhi - rlo * rlo) * rni * g.dth;
      ub += br * br * 2 * kPi * rni * rni * g.dcp[j] * (rhi - rlo);
    }
    const double ep = f.ep[ix(i, j, n1)];
    ue += ep * ep * 0.5 * (rhi * rhi - rlo * rlo) * (g.thi[j] - g.tlo[j]) * 2 * kPi * rni * g.sn[j];
    if (i >= 2 && i <= g.imax) {
      double flux = (double)f.er[ix(i, j, n1)] * 2 * kPi * g.rh[i] * g.rh[i] * g.dch[j] -
                    (double)f.er[ix(i - 1, j, n1)] * 2 * kPi * g.rh[i - 1] * g.rh[i - 1] * g.dch[j];
      if (j < nt) flux += (double)f.et[ix(i, j, nt)] * kPi * g.sh[j] * (rhi * rhi - rlo * rlo);
      if (j > 0) flux -= (double)f.et[ix(i, j - 1, nt)] * kPi * g.sh[j - 1] * (rhi * rhi - rlo * rlo);
      const double v = 2.0 * kPi / 3.0 * (rhi * rhi * rhi - rlo * rlo * rlo) * g.dch[j];
      const double qq = q[ix(i, j, n1)];
      const double res = (flux / (4 * kPi) - qq) / v;
      gmax = fmax(gmax, fabs(res));
      rmax = fmax(rmax, fabs(qq / v));
      g2 += res * res;
      gcnt += 1;
    }
  }
  L = block_sum(L, sh);
  ue = block_sum(ue, sh);
  ub = block_sum(ub, sh);
  g2 = block_sum(g2, sh);
  gcnt = block_sum(gcnt, sh);
  gmax = block_max(gmax, sh);
  rmax = block_max(rmax, sh);
  bad = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    double *o = rows + (int64_t)i * 8;
    o[0] = L / (4 * kPi); o[1] = ue; o[2] = ub; o[3] = gmax; o[4] = g2; o[5] = gcnt; o[6] = rmax; o[7] = bad;
  }
}

// Sect. 5.2 maps: sums of w and w m (gamma - 1) per cell, then divided by
// the exact cell volume (2 pi / 3)(r_{i+1}^3 - r_i^3)(cos th_j - cos th_{j+1})
template <typename R>
__global__ void __launch_bounds__(256) k_species_sums(Params<R> p, int s, double m, double *dens, double *ener) {
  const int64_t n = p.count[s];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int c = p.sp[s].cell[k];
    if (c < 0) continue;
    const double w = p.sp[s].w[k], u0 = p.sp[s].ur[k], u1 = p.sp[s].ut[k], u2 = p.sp[s].up[k];
    const double uu = u0 * u0 + u1 * u1 + u2 * u2;
    atomicAdd(&dens[c], w);
    atomicAdd(&ener[c], w * m * uu / (sqrt(1.0 + uu) + 1.0));  // gamma - 1 without cancellation
  }
}
template <typename R>
__global__ void __launch_bounds__(256) k_per_volume(Params<R> p, DiagGeom g, double *dens, double *ener) {
  const int64_t n = (int64_t)p.nr * p.nt;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c / p.nt), j = (int)(c - (int64_t)i * p.nt);
    const double a = g.rn[i], b = g.rn[i + 1];
    const double v = 2.0 * kPi / 3.0 * (b * b * b - a * a * a) * g.dcp[j];
    dens[c] /= v;
    ener[c] /= v;
  }
}
template <typename R>
__global__ void __launch_bounds__(256) k_spectrum(Params<R> p, int s, int nbins, double lg0, double inv,
                                                  double *out) {
  extern __shared__ double hist[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const int64_t n = p.count[s];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (p.sp[s].cell[k] < 0) continue;
    const double u0 = p.sp[s].ur[k], u1 = p.sp[s].ut[k], u2 = p.sp[s].up[k];
    const double lg = log10(sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2));
    double x = floor((lg - lg0) * inv);
    x = x < 0.0 ? 0.0 : (x > nbins - 1 ? (double)(nbins - 1) : x);
    atomicAdd(&hist[(int)x], (double)p.sp[s].w[k]);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (hist[b] != 0.0) atomicAdd(&out[b], hist[b]);
}

template <typename R> void launch_maps(const Params<R> &p, const DiagGeom &g, int species, double mass,
                                       double *dens, double *ener, cudaStream_t s) {
  const size_t n = (size_t)p.nr * p.nt;
  cudaMemsetAsync(dens, 0, n * sizeof(double), s);
  cudaMemsetAsync(ener, 0, n * sizeof(double), s);
  k_species_sums<R><<<1216, 256, 0, s>>>(p, species, mass, dens, ener);
  k_per_volume<R><<<1216, 256, 0, s>>>(p, g, dens, ener);
}
template <typename R> void launch_spectrum(const Params<R> &p, int species, int nbins, double lg_min,
                                           double lg_max, double *out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, (size_t)nbins * sizeof(double), s);
  k_spectrum<R><<<608, 256, (size_t)nbins * sizeof(double), s>>>(p, species, nbins, lg_min,
                                                                  nbins / (lg_max - lg_min), out);
}

template <typename R> void launch_psi64(const Params<R> &p, double *out, cudaStream_t s) {
  k_psi64<R><<<p.nr + 1, 256, 0, s>>>(p, out);
}
template <typename R> void launch_diag(const Params<R> &p, const DiagGeom &g, double *q, double *kin,
                                       double *cnt, double *rows, cudaStream_t s) {
  cudaMemsetAsync(q, 0, sizeof(double) * (size_t)(p.nr + 1) * (p.nt + 1), s);
  cudaMemsetAsync(kin, 0, sizeof(double) * 2 * kMaxSpecies, s);
  k_node_charge<R><<<1216, 256, 0, s>>>(p, q, kin, cnt);
  k_diag_rows<R><<<p.nr + 1, 256, 0, s>>>(p, g, q, rows);
}

template void launch_maps<float>(const Params<float> &, const DiagGeom &, int, double, double *, double *,
                                 cudaStream_t);
template void launch_maps<double>(const Params<double> &, const DiagGeom &, int, double, double *, double *,
                                  cudaStream_t);
template void launch_spectrum<float>(const Params<float> &, int, int, double, double, double *, cudaStream_t);
template void launch_spectrum<double>(const Params<double> &, int, int, double, double, double *, cudaStream_t);
template void launch_psi64<float>(const Params<float> &, double *, cudaStream_t);
template void launch_psi64<double>(const Params<double> &, double *, cudaStream_t);
template void launch_diag<float>(const Params<float> &, const DiagGeom &, double *, double *, double *,
                                 double *, cudaStream_t);
template void launch_diag<double>(const Params<double> &, const DiagGeom &, double *, double *, double *,
                                  double *, cudaStream_t);

}  // namespace hff
