// diag.cuh -- FP64 geometry used by the on-request diagnostics.
#pragma once
#include "hff_common.cuh"

namespace hff {

struct DiagGeom {
  const double *rn, *rh, *rlo, *rhi;          // rows: nr+1, nr, nr+1, nr+1
  const double *sn, *sh, *dcp, *dch, *tlo, *thi;  // columns: nt+1, nt, nt, nt+1, nt+1, nt+1
  double dth;
  int imax;                                   // last row of the Gauss check
};

template <typename R> void launch_psi64(const Params<R> &p, double *out, cudaStream_t s);
template <typename R> void launch_diag(const Params<R> &p, const DiagGeom &g, double *q, double *kin,
                                       double *cnt, double *rows, cudaStream_t s);
// per-cell number and kinetic-energy densities of one species (nr x nt, FP64)
template <typename R> void launch_maps(const Params<R> &p, const DiagGeom &g, int species, double mass,
                                       double *dens, double *ener, cudaStream_t s);
// weights of one species in nbins bins uniform in log10(gamma) (clamped ends)
template <typename R> void launch_spectrum(const Params<R> &p, int species, int nbins, double lg_min,
                                           double lg_max, double *out, cudaStream_t s);

}  // namespace hff
