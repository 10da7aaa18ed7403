"""The seeded synthetic inputs have the structure the design states for the
paper's workloads (no data set exists; these inputs stand in for its runs):
neutral co-located pairs inside the Table 1 PIC band and inside r_abs, a
fifth of them in the thin equatorial sheet beyond R_LC, weights giving the
density kappa n_GJ* (r*/r)^2, momenta either Maxwellian (sigma = 1 per
component) or isotropic with dN/dgamma ~ gamma^-2 on [1, 1e6], and the same
arrays for a given seed whatever the thread count."""
import math

import numpy as np

from paper_2406_14512_gb300 import workloads

N = 200_000


def gen(name, **kw):
    cfg = workloads.config(name)
    cfg.update(kw)
    return cfg, workloads.particles(cfg, n_pairs=N, seed=77, threads=1)


def test_pairs_are_colocated_and_placed_in_the_pic_band():
    """The synthetic field of the hybrid workloads: a dipole inside R_LC
    blended into a split monopole outside, s(r) = (1 - tanh((r - R_LC) /
    (0.2 R_LC))) / 2, Psi = s mu sin^2(theta)/r + (1 - s) Psi_open
    (1 - |cos theta|); every pair sits in a cell whose centre lies in the
    Table 1 PIC band and below r_abs."""
    cfg, (e, p) = gen("small_rr")
    for k in ("cell", "xo", "yo", "w"):
        assert np.array_equal(e[k], p[k]), k
    nr, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    i, j = e["cell"] // nt, e["cell"] % nt
    assert i.min() >= 1 and ((i + 1) * d < math.log(cfg["r_abs"] / cfg["r_min"])).all()
    r = cfg["r_min"] * np.exp((i + 0.5) * d)
    th = (j + 0.5) * math.pi / nt
    mu = cfg["b_star"] * cfg["r_min"] ** 3
    unit = mu / cfg["r_lc"]
    s = 0.5 * (1.0 - np.tanh((r - cfg["r_lc"]) / (0.2 * cfg["r_lc"])))
    psi = s * mu * np.sin(th) ** 2 / r + (1 - s) * cfg["synth_psi_open"] * unit * (1 - np.abs(np.cos(th)))
    assert (psi > cfg["psi_break"][0] * unit).all() and (psi < cfg["psi_break"][-1] * unit).all()
    assert ((e["xo"] >= 0) & (e["xo"] < 1) & (e["yo"] >= 0) & (e["yo"] < 1)).all()


def test_sheet_fraction():
    cfg, (e, _) = gen("c2")
    nt = cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
    i, j = e["cell"] // nt, e["cell"] % nt
    r = cfg["r_min"] * np.exp((i + 0.5) * d)
    sheet = (r > cfg["r_lc"]) & (np.abs(j + 0.5 - nt / 2) < 6)
    assert abs(sheet.mean() - 0.2) < 0.02, sheet.mean()


def test_weights_give_the_goldreich_julian_density():
    """With the configured number of pairs, the pairs (both species) stand
    for the density kappa n_GJ* (r*/r)^2, n_GJ* = B*/(2 pi e R_LC) (code units
    e = r* = B* = 1): a cell holds kappa/R_LC (r_{i+1} - r_i)(cos theta_j -
    cos theta_{j+1}) physical particles, so the placement region (rows 1 to
    i_abs - 1, every theta) holds 2 kappa (r_{i_abs} - r_1) / R_LC, and its
    inner and outer halves in proportion."""
    cfg = workloads.config("c1")
    e, p = workloads.particles(cfg, threads=1)
    nr, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    i_abs = int(math.floor(math.log(cfg["r_abs"] / cfg["r_min"]) / d)) - 1
    rk = lambda k: cfg["r_min"] * math.exp(k * d)
    w = e["w"].astype(np.float64) + p["w"].astype(np.float64)
    row = e["cell"] // nt
    mid = (1 + i_abs) // 2
    for lo, hi in ((1, i_abs), (1, mid), (mid, i_abs)):
        sel = (row >= lo) & (row < hi)
        expect = 2 * cfg["kappa_inj"] * (rk(hi) - rk(lo)) / cfg["r_lc"]
        assert abs(w[sel].sum() / expect - 1.0) < 0.02, (lo, hi, w[sel].sum(), expect)


def test_power_law_momenta():
    _, (e, p) = gen("small_rr")
    for s in (e, p):
        u = np.stack([s["ur"], s["ut"], s["up"]]).astype(np.float64)
        g = np.sqrt(1.0 + (u * u).sum(0))
        assert g.min() >= 1.0 and g.max() <= 1.0e6 * (1 + 1e-5)
        # P(gamma > x) = (1/x - 1e-6)/(1 - 1e-6) for dN/dgamma ~ gamma^-2
        for x in (2.0, 10.0, 100.0):
            expect = (1 / x - 1e-6) / (1 - 1e-6)
            got = (g > x).mean()
            assert abs(got - expect) < 5 * math.sqrt(expect * (1 - expect) / N), (x, got, expect)
        # isotropic: each direction cosine has mean 0 and mean square 1/3
        n = u / np.maximum(np.linalg.norm(u, axis=0), 1e-30)
        live = g > 1.0 + 1e-6
        for k in range(3):
            assert abs(n[k][live].mean()) < 0.01
            assert abs((n[k][live] ** 2).mean() - 1 / 3) < 0.01
    # the two species draw independently
    assert not np.array_equal(e["ur"], p["ur"])


def test_maxwellian_momenta():
    _, (e, _) = gen("small_pic")
    for k in ("ur", "ut", "up"):
        v = e[k].astype(np.float64)
        assert abs(v.mean()) < 0.01 and abs(v.std() - 1.0) < 0.01


def test_deterministic_for_a_seed_whatever_the_threads():
    cfg = workloads.config("small_rr")
    a = workloads.particles(cfg, n_pairs=50_000, seed=5, threads=1, chunk=10_000)
    b = workloads.particles(cfg, n_pairs=50_000, seed=5, threads=4, chunk=10_000)
    for s in range(2):
        for k in a[s]:
            assert np.array_equal(a[s][k], b[s][k]), k
