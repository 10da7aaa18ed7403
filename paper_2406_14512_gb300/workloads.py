"""Seeded synthetic workloads: configuration dicts and particle generators.

This module describes INPUTS only.  It holds none of the scheme's arithmetic
(no flux prefix, no blending, no push, no deposit): it writes down the grid and
physical parameters of each workload and draws macro-particles with numpy from
a fixed seed.  Both the CUDA library and the FP64 oracle consume exactly these
inputs.

Workloads (shaped like the runs of Sects. 4-5; the paper uses no dataset):
  c1  256 x 128, r in [1, 30], R_LC = 3, dipole, PIC everywhere, 2e5 e+-,
      kappa-mode surface injection, FP64 (200 steps)
  c2  1024 x 1024, r in [1, 60], R_LC = 6, synthetic dipole / split monopole,
      Table 1 flux bands, 5e7 e+- with Maxwellian momenta (sigma = 1)
  c3  4096 x 4096, r in [1, 100], R_LC = 10, same field construction, 3e8 e+-,
      gamma ~ dN/dgamma ~ gamma^-2 on [1, 1e6], radiation reaction on,
      Goldreich-Julian top-up injection
  c4  8192 x 8192, r in [1, 200], R_LC = 20, 1e9 e+- (precision stress)
  c5  an ensemble of 32 independent c2-like instances (seeds 1234..1265):
      N_r in {256, 512, 1024}, N_theta in {128, 256, 512}, R_LC uniform in
      [3, 10] with r_max = 10 R_LC, 1e5 - 5e6 e+- log-uniform (ensemble())
Plus small variants of each for parity tests.

Units: c = 1, r_star = 1, B_star = 1, e = 1 (species 0 = electrons q = -1,
species 1 = positrons q = +1).  The electron mass sets the scale separation;
it is chosen so that the surface plasma frequency at kappa n_GJ is resolved as
in Sect. 5.1 (omega_pe dt ~ 1/8).
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# Table 1 flux bands in units of Psi_pc = mu / R_LC: FF-I below 0.85 -> 0.9,
# PIC between, FF-II from 2.3 -> 2.4 upwards.
TABLE1_PSI = [0.85, 0.9, 2.3, 2.4]
TABLE1_F = [1.0, 0.0, 0.0, 1.0]


def _dt_estimate(nr, nt, r_min, r_max, courant):
    d = math.log(r_max / r_min) / nr
    dth = math.pi / nt
    dr = r_min * (math.exp(d) - 1.0)
    return courant / math.sqrt(1.0 / dr ** 2 + 1.0 / (r_min * dth) ** 2)


def _base(nr, nt, r_max, r_lc, geom, kappa=10.0, ppc_inj=4.0, courant=0.5, seed=1234):
    r_min = 1.0
    dt = _dt_estimate(nr, nt, r_min, r_max, courant)
    omega = 1.0 / r_lc
    # electron mass from omega_pe dt = 1/8 at n = kappa n_GJ*, n_GJ* = Omega B*/(2 pi e c)
    wpe = 1.0 / (8.0 * dt)
    m_e = 4.0 * math.pi * kappa * (omega / (2.0 * math.pi)) / wpe ** 2
    dlog, dth = math.log(r_max / r_min) / nr, math.pi / nt
    # injected weight: largest surface target count is ppc_inj pairs
    w_inj = kappa * omega * dlog * dth / ppc_inj
    r_abs = min(3.0 * r_lc, r_min * math.exp(dlog * (nr - 4)))
    return dict(nr=nr, nt=nt, r_min=r_min, r_max=r_max, r_lc=r_lc, b_star=1.0, geom=geom,
                courant=courant, r_abs=r_abs, absorb_strength=0.1, psi_break=[], f_break=[],
                q=[-1.0, 1.0], m=[m_e, m_e], inject=True, kappa_inj=kappa, w_inj=w_inj,
                gamma_rad=0.0, b_ref=1.0 / r_lc ** 3, rr_scale=1.0, shell_r=2.0 * r_min,
                synth_psi_open=1.25, seed=seed, capacity=0, tile_r=16, tile_t=32,
                sort_every=8, dt_estimate=dt, gamma_th=0.0, gamma_s=0.0)


def config(name: str) -> dict:
    """Workload configuration by name (see the module docstring)."""
    if name == "c1":
        c = _base(256, 128, 30.0, 3.0, "dipole", seed=1234)
        c.update(n_pairs=100_000, steps=200, precision="fp64", place="uniform", momenta="maxwell")
    elif name == "c2":
        c = _base(1024, 1024, 60.0, 6.0, "synth", seed=1235)
        c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=25_000_000,
                 steps=2000, precision="fp32", place="band", sheet_frac=0.2, momenta="maxwell",
                 tile_r=16, tile_t=24, sort_every=12)  # the autotuner's choice on this grid
    elif name == "c3":
        c = _base(4096, 4096, 100.0, 10.0, "synth", kappa=1.0, seed=1236)
        c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=150_000_000,
                 steps=1000, precision="fp32", place="band", sheet_frac=0.2, momenta="powerlaw")
        c["gamma_rad"] = 0.05 * (c["r_lc"] ** -2) / c["m"][0]  # 5% of gamma_pc = e Phi_pc / m c^2
        c.update(tile_r=0, tile_t=0, sort_every=-1)  # launch shape measured by the autotuner at init
    elif name == "c4":
        c = _base(8192, 8192, 200.0, 20.0, "synth", kappa=1.0, seed=1237)
        c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=500_000_000,
                 steps=500, precision="fp32", place="band", sheet_frac=0.2, momenta="maxwell",
                 tile_r=0, tile_t=0, sort_every=-1)  # launch shape measured by the autotuner at init
    elif name.startswith("small_"):
        # reduced-size parity variants, spanning several tiles and a ragged tail
        kind = name[len("small_"):]
        if kind == "pic":        # c1-like, PIC everywhere
            c = _base(70, 52, 30.0, 3.0, "dipole", seed=11)
            c.update(n_pairs=3000, steps=10, precision="fp64", place="uniform", momenta="maxwell")
        elif kind == "hybrid":   # c2-like with Table 1 bands
            c = _base(96, 80, 60.0, 6.0, "synth", seed=12)
            c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=6000,
                     steps=10, precision="fp32", place="band", sheet_frac=0.2, momenta="maxwell")
        elif kind == "rr":       # c3-like with radiation reaction
            c = _base(80, 72, 100.0, 10.0, "synth", kappa=1.0, seed=13)
            c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=6000,
                     steps=10, precision="fp32", place="band", sheet_frac=0.2, momenta="powerlaw")
            c["gamma_rad"] = 0.05 * (c["r_lc"] ** -2) / c["m"][0]
        elif kind == "fine":     # hybrid, fine enough for the small-increment series (D, dtheta < 0.03)
            c = _base(200, 120, 20.0, 4.0, "synth", seed=15)
            c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=8000,
                     steps=10, precision="fp32", place="band", sheet_frac=0.2, momenta="powerlaw")
            c["gamma_rad"] = 0.05 * (c["r_lc"] ** -2) / c["m"][0]
        elif kind == "pairs":    # PIC everywhere with threshold pair creation (Sect. 5.1)
            c = _base(72, 56, 30.0, 3.0, "dipole", seed=16)
            # gamma ~ gamma^-2 up to 1e6, so about 2% of the leptons start above
            # gamma_th; gamma_th / gamma_s = 1e6 / 2.2e5 as in Table 1
            c.update(n_pairs=4000, steps=10, precision="fp32", place="uniform", momenta="powerlaw",
                     gamma_th=50.0, gamma_s=50.0 * 2.2e5 / 1e6)
            c["gamma_rad"] = 0.05 * (c["r_lc"] ** -2) / c["m"][0]
        elif kind == "crust":    # e-, e+, protons: crust extraction of e- and p, pair creation (Sect. 5.1)
            c = _base(72, 56, 30.0, 3.0, "synth", seed=17)
            me = c["m"][0]
            c.update(q=[-1.0, 1.0, 1.0], m=[me, me, 1836.0 * me], inject_species=[0, 2],
                     psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=4000, steps=10,
                     precision="fp32", place="band", sheet_frac=0.2, momenta="powerlaw",
                     gamma_th=50.0, gamma_s=50.0 * 2.2e5 / 1e6)
            c["gamma_rad"] = 0.05 * (c["r_lc"] ** -2) / me
        elif kind == "michel":   # monopole, south hemisphere force-free (Sect. 4)
            c = _base(64, 64, 50.0 / 3.0, 5.0, "michel", seed=14)
            # sharp cut at the equator (Psi = Psi*), placed a hair below Psi* so
            # that the equatorial nodes fall deterministically on the force-free side
            c.update(psi_break=[1.0 - 1e-4, 1.0 - 1e-4], f_break=[0.0, 1.0], n_pairs=0, steps=10,
                     precision="fp32", place="uniform", momenta="maxwell")
        else:
            raise KeyError(name)
    else:
        raise KeyError(name)
    return c


def ensemble(name: str = "c5", n_inst: int | None = None) -> list[dict]:
    """Configurations of the independent instances of an ensemble workload.

    c5: 32 c2-like instances (synthetic dipole / split monopole, Table 1 flux
    bands, Maxwellian momenta, kappa-mode surface injection, FP32), instance k
    drawn from seed 1234 + k.  small_c5: 4 instances of the same kind on grids
    small enough for the oracle (parity tests)."""
    if name == "c5":
        n_inst = 32 if n_inst is None else n_inst
        rows, cols, lo, hi = [256, 512, 1024], [128, 256, 512], 1e5, 5e6
    elif name == "small_c5":
        n_inst = 4 if n_inst is None else n_inst
        rows, cols, lo, hi = [40, 56, 72], [32, 48, 64], 2e3, 8e3
    else:
        raise KeyError(name)
    out = []
    for k in range(n_inst):
        seed = 1234 + k
        rng = np.random.default_rng(seed)
        nr, nt = int(rng.choice(rows)), int(rng.choice(cols))
        r_lc = float(rng.uniform(3.0, 10.0))
        n_part = float(np.exp(rng.uniform(math.log(lo), math.log(hi))))
        c = _base(nr, nt, 10.0 * r_lc, r_lc, "synth", seed=seed)
        n_pairs = max(1, int(round(n_part / 2)))
        c.update(psi_break=list(TABLE1_PSI), f_break=list(TABLE1_F), n_pairs=n_pairs, steps=1000,
                 precision="fp32", place="band", sheet_frac=0.2, momenta="maxwell",
                 capacity=int(n_pairs * 1.2) + 20_000)
        out.append(c)
    return out


def sample(name: str, n: int) -> dict:
    """The workload `name` on an n x n grid with the same particles per cell
    (a bounded sample for timing the CPU oracle)."""
    c = config(name)
    scale = (n * n) / float(c["nr"] * c["nt"])
    small = _base(n, n, c["r_max"], c["r_lc"], c["geom"], kappa=c["kappa_inj"], seed=c["seed"])
    for k in ("psi_break", "f_break", "precision", "place", "sheet_frac", "momenta", "steps", "tile_r", "tile_t",
              "sort_every"):
        if k in c:
            small[k] = c[k]
    if c.get("gamma_rad", 0.0) > 0:
        small["gamma_rad"] = 0.05 * (small["r_lc"] ** -2) / small["m"][0]
    small["n_pairs"] = max(1, int(round(c["n_pairs"] * scale)))
    return small


# ---------------------------------------------------------------- particles
def _psi_analytic_cells(cfg: dict) -> np.ndarray:
    """Analytic flux function of the initial field at cell centres (input
    construction only: decides where the synthetic plasma is placed)."""
    nr, nt = cfg["nr"], cfg["nt"]
    dlog = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    r = cfg["r_min"] * np.exp((np.arange(nr) + 0.5) * dlog)[:, None]
    th = ((np.arange(nt) + 0.5) * math.pi / nt)[None, :]
    mu = cfg["b_star"] * cfg["r_min"] ** 3
    psi_d = mu * np.sin(th) ** 2 / r
    if cfg["geom"] == "synth":
        popen = cfg["synth_psi_open"] * mu / cfg["r_lc"]
        s = 0.5 * (1.0 - np.tanh((r - cfg["r_lc"]) / (0.2 * cfg["r_lc"])))
        return s * psi_d + (1.0 - s) * popen * (1.0 - np.abs(np.cos(th)))
    return np.broadcast_to(psi_d, (nr, nt))


def placement_cells(cfg: dict):
    """Cells eligible for the synthetic plasma and the thin-sheet subset."""
    nr, nt = cfg["nr"], cfg["nt"]
    dlog = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    i_abs = int(math.floor(math.log(cfg["r_abs"] / cfg["r_min"]) / dlog)) - 1
    rows = np.arange(nr)
    inside = (rows >= 1) & (rows < i_abs)
    if cfg.get("place") == "band" and cfg.get("psi_break"):
        unit = cfg["b_star"] * cfg["r_min"] ** 3 / cfg["r_lc"]
        lo, hi = cfg["psi_break"][0] * unit, cfg["psi_break"][-1] * unit
        psi = _psi_analytic_cells(cfg)
        ok = (psi > lo) & (psi < hi) & inside[:, None]
    else:
        ok = np.broadcast_to(inside[:, None], (nr, nt)).copy()
    cells = np.flatnonzero(ok.ravel()).astype(np.int64)
    r_row = cfg["r_min"] * np.exp((rows + 0.5) * dlog)
    half = 6
    sheet = np.zeros((nr, nt), bool)
    sheet[(r_row > cfg["r_lc"]) & inside, nt // 2 - half:nt // 2 + half] = True
    sheet_cells = np.flatnonzero((sheet & ok).ravel()).astype(np.int64)
    return cells, sheet_cells


def _draw_chunk(args):
    cfg, seed_seq, n, cells, sheet_cells, sheet_frac = args
    rng = np.random.default_rng(seed_seq)
    nt = cfg["nt"]
    dlog = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
    dth = math.pi / nt
    n_sheet = int(round(n * sheet_frac)) if len(sheet_cells) else 0
    pick = np.empty(n, np.int64)
    pick[:n - n_sheet] = cells[rng.integers(0, len(cells), n - n_sheet)]
    if n_sheet:
        pick[n - n_sheet:] = sheet_cells[rng.integers(0, len(sheet_cells), n_sheet)]
    xo = rng.random(n, dtype=np.float32)
    yo = rng.random(n, dtype=np.float32)
    i = pick // nt
    j = pick % nt
    r = cfg["r_min"] * np.exp((i + xo) * dlog)
    th = (j + yo) * dth
    # weight: density kappa n_GJ* (r_star/r)^2 at a uniform count per cell
    ppc = max(1.0, 2.0 * cfg["n_pairs"] / max(1, len(cells)))
    w = (cfg["kappa_inj"] * (1.0 / cfg["r_lc"]) * dlog * dth * r * np.maximum(np.sin(th), 0.5 * dth)
         / ppc).astype(np.float32)
    out = []
    for _ in range(2):
        if cfg.get("momenta") == "powerlaw":
            # dN/dgamma ~ gamma^-2 on [1, 1e6], isotropic
            g = 1.0 / (1.0 - rng.random(n) * (1.0 - 1e-6))
            pm = np.sqrt(np.maximum(g * g - 1.0, 0.0))
            mu = 2.0 * rng.random(n) - 1.0
            ph = 2.0 * math.pi * rng.random(n)
            st = np.sqrt(1.0 - mu * mu)
            u = np.stack([pm * mu, pm * st * np.cos(ph), pm * st * np.sin(ph)])
        else:
            u = rng.normal(0.0, 1.0, (3, n))
        out.append(u.astype(np.float32))
    return pick.astype(np.int32), xo, yo, w, out


def particles(cfg: dict, n_pairs: int | None = None, seed: int | None = None,
              threads: int = 8, chunk: int = 4_000_000) -> list[dict]:
    """Co-located e-/e+ pairs (neutral at t = 0), FP32 SoA per species.

    Returns ``[electrons, positrons]``, each a dict of numpy arrays
    ``cell`` (int32, i * nt + j), ``xo``, ``yo`` (offsets in [0, 1)),
    ``ur``, ``ut``, ``up`` (u = gamma v / c in the local spherical basis) and
    ``w`` (macro-particle weight).  The weights are those of the configured
    count ``cfg["n_pairs"]`` (the pairs then stand for the density
    kappa n_GJ* (r*/r)^2); drawing another ``n_pairs`` keeps the per-pair
    weight, so the represented density scales with the number drawn.
    Deterministic for a given seed whatever the thread count."""
    n = int(cfg["n_pairs"] if n_pairs is None else n_pairs)
    seed = int(cfg["seed"] if seed is None else seed)
    cells, sheet_cells = placement_cells(cfg)
    sizes = [min(chunk, n - k) for k in range(0, n, chunk)] if n else []
    seqs = np.random.SeedSequence(seed).spawn(max(1, len(sizes)))
    args = [(cfg, seqs[k], sizes[k], cells, sheet_cells, cfg.get("sheet_frac", 0.0))
            for k in range(len(sizes))]
    if len(args) > 1 and threads > 1:
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(_draw_chunk, args))
    else:
        parts = [_draw_chunk(a) for a in args]
    res = []
    for s in range(2):
        d = {}
        if parts:
            d["cell"] = np.concatenate([p[0] for p in parts])
            d["xo"] = np.concatenate([p[1] for p in parts])
            d["yo"] = np.concatenate([p[2] for p in parts])
            d["w"] = np.concatenate([p[3] for p in parts])
            u = np.concatenate([p[4][s] for p in parts], axis=1)
            d["ur"], d["ut"], d["up"] = u[0].copy(), u[1].copy(), u[2].copy()
        else:
            for k in ("xo", "yo", "w", "ur", "ut", "up"):
                d[k] = np.zeros(0, np.float32)
            d["cell"] = np.zeros(0, np.int32)
        res.append(d)
    return res


def random_fields(shapes: dict, seed: int, scale: float = 1.0) -> dict:
    """Smooth-plus-noise FP32 field arrays for stand-alone field-update tests."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in shapes.items():
        a = rng.normal(0.0, scale, shp)
        out[name] = a.astype(np.float32)
    return out
