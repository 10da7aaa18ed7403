"""Scale helpers against the numbers the paper prints for its reference
millisecond pulsar (Sect. 2: P = 1 ms, B* = 1e7 G, r* = 1e6 cm; Sect. 5.1 and
Table 1 for the 8192^2 run with R_LC = 5e6 cm, r_max = (10/3) R_LC), and the
monopole run's B_ph diagnostic against Michel's solution (Sect. 4)."""
import math

import pytest

from paper_2406_14512_gb300 import scales as S

R_STAR, B_STAR, P = 1e6, 1e7, 1e-3
RLC = 5e6          # the run of Sect. 5.1 fixes R_LC = 5e6 cm (P = 1 ms gives 4.77e6)


def close(x, ref, tol):
    return abs(x / ref - 1.0) < tol


def test_light_cylinder_and_spindown():
    assert close(S.r_lc(P), 5.0 * R_STAR, 0.05)                   # "R_LC ~ 5 r* (P / 1 ms)"
    assert close(S.b_lc(B_STAR, R_STAR, RLC), 8e4, 0.01)           # Sect. 5.1: B_LC ~ 8e4 G
    assert close(S.spindown(B_STAR, R_STAR, RLC), 4.8e33, 0.01)    # L_0 = 4.8e33 erg/s


def test_energy_scales():
    assert close(S.gamma_pc(B_STAR, R_STAR, S.r_lc(P)), 2.6e8, 0.05)
    assert close(S.gamma_th(B_STAR), 1e6, 0.15)                    # gamma_th ~ 1e6
    assert close(S.gamma_s(B_STAR), 2.2e5, 0.02)                   # gamma_s ~ 2.2e5
    assert close(S.gamma_rad(B_STAR, B_STAR), 3e4, 0.1)            # E_par = B_perp = 1e7 G
    blc = S.b_lc(B_STAR, R_STAR, RLC)
    assert close(S.gamma_rad(blc, blc), 3.3e5, 0.1)                # at the light cylinder


def test_length_scales():
    n = 100.0 * S.n_gj(B_STAR, S.r_lc(P))                          # kappa = 1e2
    assert close(S.skin_depth(n), 2.0, 0.1)                        # d_e* ~ 2 cm
    assert close(S.skin_depth(n, S.gamma_s(B_STAR)) / R_STAR, 1e-3, 0.1)  # d_e^s ~ 1e3 cm
    assert close(S.sheet_thickness(S.r_lc(P), 100.0), 2.4e4, 0.02)        # delta ~ 2.4e4 cm


def test_grid_of_the_dipole_run():
    """Table 1: dr = 3.4e2 cm and dt = 4.3e-9 s on 8192^2 cells over
    [r*, (10/3) R_LC] at half the 2D Courant limit."""
    dr, dt = S.grid_steps(R_STAR, 10.0 / 3.0 * RLC, 8192, courant=0.5)
    assert close(dr, 3.4e2, 0.02)
    assert close(dt, 4.3e-9, 0.02)


def test_resolution_ratios_of_section_5_1():
    """Sect. 5.1: d_e^s / dr ~ 3 and omega_pe^-1 / dt ~ 8 at the surface,
    rho_s / (R_LC dr / r*) ~ 3, rho_s / (c dt) ~ 36, t_syn^LC ~ 85 dt."""
    dr, dt = S.grid_steps(R_STAR, 10.0 / 3.0 * RLC, 8192, courant=0.5)
    n = 100.0 * S.n_gj(B_STAR, RLC)
    gs = S.gamma_s(B_STAR)
    assert 2.0 < S.skin_depth(n, gs) / dr < 4.0
    assert 6.0 < 1.0 / S.plasma_frequency(n, gs) / dt < 9.0
    blc = S.b_lc(B_STAR, R_STAR, RLC)
    rho = S.larmor_radius(gs, blc)
    assert 2.5 < rho / (RLC * dr / R_STAR) < 3.5
    assert close(rho / (S.C * dt), 36.0, 0.05)
    assert close(S.synchrotron_time(gs, blc) / dt, 85.0, 0.05)


def test_code_units():
    cu = S.code_units(B_STAR, P, R_STAR)
    assert close(cu["r_lc"], 4.77, 0.01)
    # e Phi_pc / m_e = gamma_pc in code units
    assert close((1.0 / cu["r_lc"] ** 2) / cu["m_e"], cu["gamma_pc"], 1e-12)
    assert cu["gamma_th"] > cu["gamma_s"] > 1.0


def test_monopole_bphi_error_against_michel():
    """The monopole run's B_ph diagnostic: zero for Michel's own field
    -(Psi*/R_LC) sin(theta)/r at the half nodes, 0.1 for a field 10% too
    strong in one hemisphere, per hemisphere."""
    import numpy as np
    from paper_2406_14512_gb300 import monopole
    cfg = monopole.config(64)
    nr, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    rh = cfg["r_min"] * np.exp((np.arange(nr) + 0.5) * d)
    th = (np.arange(nt) + 0.5) * math.pi / nt
    psi_star = cfg["b_star"] * cfg["r_min"] ** 2
    exact = -(psi_star / cfg["r_lc"]) * np.sin(th)[None, :] / rh[:, None]

    class Fake:
        def __init__(self, f):
            self.f = f

        def get(self, name):
            assert name == "B_ph"
            return self.f

    e = monopole.bphi_error(Fake(exact.astype(np.float32)), cfg)
    assert e["north_pic"] < 1e-6 and e["south_ff"] < 1e-6
    f = exact.copy()
    f[:, th > math.pi / 2] *= 1.1
    e = monopole.bphi_error(Fake(f), cfg)
    assert e["north_pic"] < 1e-12 and abs(e["south_ff"] - 0.1) < 1e-12
