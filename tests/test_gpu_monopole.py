"""The hybrid monopole of Sect. 4 (northern hemisphere PIC with kappa = 10
surface injection, southern hemisphere force-free, sharp cut at the equator)
for two spin periods at 512^2 and 1024^2: a KNOWN DEVIATION from the paper,
held as a regression of the measured behaviour.

The paper quotes eps < 1% at 1024^2 (Eq. 36) and about 0.15% at 4096^2.  This
implementation, with the corrected field returned literally to the mesh every
step (the stable reading of Sect. 3's "interpolate these back"), measures
6.9% at 512^2, 3.7% at 1024^2, 2.0% at 2048^2 and 1.36% at 4096^2: first-order
convergence, from the per-step averaging of that return.  The second-order
return of the corrections alone grows a mode next to the force-free / PIC
interface; returning the corrected field on the stellar row of radial edges
as well (ff_delta_only = 2) keeps the run finite but lets the force-free
solution drift away from Michel's at 1024^2 and 2048^2.  What is checked: the run stays finite and clean, eps falls with
resolution at no worse than first order and stays within 15% of the values
measured above (a regression in either direction fails), the spin-down near
the star is within 3% of Michel's L_M = 2 Psi*^2 Omega^2 / 3c at 1024^2, and
the force-free B_phi at 1.5 R_LC within 3% of Michel's."""
import pytest

pytestmark = pytest.mark.gpu

MEASURED_EPS = {512: 0.0686, 1024: 0.0373}


def test_monopole_known_first_order_deviation_from_the_paper():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import monopole
    res = {n: monopole.run(n, periods=2.0, chunk=20000) for n in (512, 1024)}
    for n, r in res.items():
        assert r["status"] == 0 and r["nonfinite"] == 0, r
        assert abs(r["L_in_over_L_M"] - 1.0) < 0.05, r
        assert r["bphi_rel_err_1p5_rlc"]["south_ff"] < 0.05, r
        assert abs(r["eps"] / MEASURED_EPS[n] - 1.0) < 0.15, (n, r["eps"])
    lo, hi = res[512], res[1024]
    assert hi["eps"] < 0.6 * lo["eps"], (lo["eps"], hi["eps"])   # at least first order
    assert abs(hi["L_in_over_L_M"] - 1.0) < 0.03
    assert hi["bphi_rel_err_1p5_rlc"]["south_ff"] < 0.03
