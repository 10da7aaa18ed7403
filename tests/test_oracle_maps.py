"""Pins of the oracle's density / energy maps and energy spectra (Sect. 5.2
figures): totals, a lone particle against its closed form, and spectrum bins
of particles with known Lorentz factors."""
import math

import numpy as np

from paper_2406_14512_gb300 import workloads


def cfg_small(**kw):
    cfg = workloads.config("small_pic")
    cfg.update(capacity=20000, inject=False, sort_every=0)
    cfg.update(kw)
    return cfg


def volumes(cfg):
    nr, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    rn = cfg["r_min"] * np.exp(np.arange(nr + 1) * d)
    tn = np.arange(nt + 1) * math.pi / nt
    return (2 * math.pi / 3) * (rn[1:] ** 3 - rn[:-1] ** 3)[:, None] * (np.cos(tn[:-1]) - np.cos(tn[1:]))[None, :]


def test_map_totals_match_the_particles(oracle_mod):
    cfg = cfg_small()
    o = oracle_mod.Oracle(cfg)
    ps = workloads.particles(cfg, n_pairs=3000, seed=3)
    for s in range(2):
        o.set_particles(s, ps[s])
    v = volumes(cfg)
    for s in range(2):
        dens, ener = o.species_maps(s)
        p = o.particles(s)
        assert abs((dens * v).sum() - p["w"].sum()) < 1e-12 * p["w"].sum()
        u2 = p["ur"] ** 2 + p["ut"] ** 2 + p["up"] ** 2
        ke = (p["w"] * cfg["m"][s] * (np.sqrt(1 + u2) - 1)).sum()
        assert abs((ener * v).sum() - ke) < 1e-10 * ke


def test_lone_particle_closed_form(oracle_mod):
    cfg = cfg_small()
    o = oracle_mod.Oracle(cfg)
    nt = cfg["nt"]
    i, j, w, u = 11, 7, 2.5, (3.0, -4.0, 12.0)          # |u| = 13, gamma = sqrt(170)
    p = dict(cell=np.array([i * nt + j], np.int32), xo=np.array([0.3]), yo=np.array([0.8]),
             ur=np.array([u[0]]), ut=np.array([u[1]]), up=np.array([u[2]]), w=np.array([w]))
    o.set_particles(0, p)
    dens, ener = o.species_maps(0)
    vol = volumes(cfg)[i, j]
    assert abs(dens[i, j] - w / vol) < 1e-14 * w / vol
    assert abs(ener[i, j] - w * cfg["m"][0] * (math.sqrt(170.0) - 1.0) / vol) < 1e-12 * ener[i, j]
    dens[i, j] = ener[i, j] = 0
    assert not dens.any() and not ener.any()


def test_spectrum_bins(oracle_mod):
    cfg = cfg_small()
    o = oracle_mod.Oracle(cfg)
    # gamma = 10^0.25, 10^1.25, 10^2.25, 10^3.25 and one far above / below the range
    lg = np.array([0.25, 1.25, 2.25, 3.25, 9.0, 0.0])
    gam = 10.0 ** lg
    u = np.sqrt(gam ** 2 - 1.0)
    w = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    p = dict(cell=np.full(6, 5 * cfg["nt"] + 3, np.int32), xo=np.full(6, 0.5), yo=np.full(6, 0.5),
             ur=u, ut=np.zeros(6), up=np.zeros(6), w=w)
    o.set_particles(1, p)
    h = o.spectrum(1, 8, 0.5, 4.5)       # bins of width 0.5 in log10(gamma) from 0.5
    expect = np.zeros(8)
    expect[0] += 1.0 + 6.0               # 0.25 and 0.0 lie below: first bin
    expect[1] += 2.0                     # 1.25 -> (1.25 - 0.5) / 0.5 = 1.5
    expect[3] += 3.0                     # 2.25 -> 3.5
    expect[5] += 4.0                     # 3.25 -> 5.5
    expect[7] += 5.0                     # above the range: last bin
    assert np.array_equal(h, expect)
