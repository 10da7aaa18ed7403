"""Pins of the oracle's FP64 diagnostics against closed forms:

* Psi_open, the flux through the northern hemisphere at r = 2 R_LC (Psi at the
  equator node), equals Psi* for the monopole of Eq. 32 and mu / r for the
  dipole of Eq. 37 (the discrete Psi is exact at nodes);
* the field energies of a uniform B_z and of a uniform E_z converge at second
  order to B^2 (r_max^3 - r_min^3) / 6 (the energy density B^2 / 8 pi over the
  spherical shell);
* the kinetic energy and the live count of given particles are
  sum w m (gamma - 1) and their number."""
import math

import numpy as np

from test_oracle_fields import grid, mk


def test_psi_open_exact_for_monopole_and_dipole(oracle_mod):
    nr, nt, r_max, r_lc = 64, 32, 30.0, 3.0
    d = math.log(r_max) / nr
    i_out = int(math.floor(math.log(2.0 * r_lc) / d + 0.5))
    r_out = math.exp(i_out * d)
    for geom, exact in (("monopole", 1.0), ("dipole", 1.0 / r_out)):
        o = oracle_mod.Oracle(mk(nr, nt, geom, r_max=r_max, r_lc=r_lc))
        dg, _ = o.diagnostics()
        assert abs(dg.psi_open / exact - 1.0) < 1e-13, (geom, dg.psi_open, exact)


def shell_energy(r_max):
    return (r_max ** 3 - 1.0) / 6.0


def test_magnetic_energy_of_uniform_field_second_order(oracle_mod):
    errs = []
    for n in (16, 32, 64):
        o = oracle_mod.Oracle(mk(n, n, "uniform", r_max=4.0, r_lc=1e6, r_abs=3.9))
        dg, _ = o.diagnostics()
        errs.append(abs(dg.u_b / shell_energy(4.0) - 1.0))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 1e-3 and min(rates) > 1.9, (errs, rates)


def test_electric_energy_of_uniform_field_second_order(oracle_mod):
    """E = z-hat at the edge points: E_r = cos(theta), E_th = -sin(theta)."""
    errs = []
    for n in (16, 32, 64):
        o = oracle_mod.Oracle(mk(n, n, "uniform", r_max=4.0, r_lc=1e6, r_abs=3.9))
        rn, rh, tn, th = grid(o)
        o.set("E_r", np.repeat(np.cos(tn)[None, :], n, axis=0))
        o.set("E_th", np.repeat(-np.sin(th)[None, :], n + 1, axis=0))
        o.set("E_ph", np.zeros(o.shape("E_ph")))
        dg, _ = o.diagnostics()
        errs.append(abs(dg.u_e / shell_energy(4.0) - 1.0))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 1e-3 and min(rates) > 1.9, (errs, rates)


def test_kinetic_energy_and_count(oracle_mod):
    c = mk(16, 16, "dipole", r_max=4.0, r_lc=2.0, capacity=8)
    c["m"] = [1.0, 3.0]
    o = oracle_mod.Oracle(c)
    u = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [1.0, -2.0, 2.0]])
    w = np.array([2.0, 0.5, 1.5])
    for s in range(2):
        o.set_particles(s, dict(cell=np.array([5 * 16 + 3, 7 * 16 + 8, -1], np.int32), xo=np.full(3, 0.5),
                                yo=np.full(3, 0.5), ur=u[:, 0].copy(), ut=u[:, 1].copy(), up=u[:, 2].copy(), w=w))
    dg, _ = o.diagnostics()
    # live: the first two (the third is removed); gamma = 1 and sqrt(26)
    for s, m in ((0, 1.0), (1, 3.0)):
        assert dg.count[s] == 2
        assert abs(dg.kinetic[s] - m * 0.5 * (math.sqrt(26.0) - 1.0)) < 1e-14
