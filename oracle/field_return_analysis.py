"""Stability analysis of the return of the corrected field (Sect. 3, "interpolate
these back") on the FP64 oracle.  TEST INFRASTRUCTURE: it drives only the
oracle in this folder, never the CUDA library.

Two measurements, each from finite differences through the oracle:

* `stage`: the Jacobian of one correction stage (node pass A for Psi, node
  pass B, the return to the edges) around Michel's monopole (Eqs. 32-35),
  force-free everywhere, on an n x n mesh.  Its largest singular value in the
  field-energy norm sum E^2 V_e (V_e = an E component's edge length times its
  dual face: the weights under which the Yee pair conserves vacuum energy),
  restricted to a region of edges, says whether the stage can raise the energy
  of a perturbation there (> 1) or not (<= 1).
* `step`: the Jacobian of one whole field step of the Sect. 4 monopole set-up
  (r in [r*, (10/3) R_LC], R_LC = 5 r*, a sharp cut at the equator, force-free
  south) with the northern hemisphere left in vacuum (f = 0, no particles),
  linearised `pre` steps into the run; its eigenvalues of largest modulus and
  where their eigenvectors sit.

    python -m oracle.field_return_analysis stage --n 16 --reading 1
    python -m oracle.field_return_analysis step --n 24 --reading 1 --pre 100
"""
from __future__ import annotations

import argparse
import math

import numpy as np

from . import Oracle

E_NAMES = ["E_r", "E_th", "E_ph"]
ALL_NAMES = ["E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph"]
ST_NODE, ST_CORRECT = 1, 2


def sect4_config(n: int, reading: int, geom: str = "monopole", allff: bool = False, r_abs: float = 0.0) -> dict:
    """The Sect. 4 monopole mesh without particles; `allff` makes the whole
    domain force-free, otherwise f jumps from 0 (north) to 1 (south) a hair
    below Psi* so that the equatorial nodes are force-free.  The absorber
    starts at 3 R_LC, or 4 cells inside r_max where 3 R_LC is closer to it
    (the library's limit), unless `r_abs` is given."""
    r_lc, r_max = 5.0, 50.0 / 3.0
    dlog = math.log(r_max) / n
    cut = 1.0 - 1e-4
    brk = dict(psi_break=[-1.0], f_break=[1.0]) if allff else dict(psi_break=[cut, cut], f_break=[0.0, 1.0])
    return dict(nr=n, nt=n, r_min=1.0, r_max=r_max, r_lc=r_lc, b_star=1.0, geom=geom, courant=0.5,
                r_abs=r_abs or min(3.0 * r_lc, r_max * math.exp(-4 * dlog)), absorb_strength=0.1,
                inject=False, capacity=0, seed=1, ff_delta_only=reading, **brk)


def energy_weights(cfg: dict):
    """V_e of E_r, E_th, E_ph on the staggered log-r mesh (edge length x dual face)."""
    n, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / n
    dth = math.pi / nt
    rn = cfg["r_min"] * np.exp(np.arange(n + 1) * d)
    rh = cfg["r_min"] * np.exp((np.arange(n) + 0.5) * d)
    tn = np.arange(nt + 1) * dth
    th = (np.arange(nt) + 0.5) * dth
    tlo, thi = np.concatenate([[0.0], th]), np.concatenate([th, [math.pi]])
    rlo, rhi = np.concatenate([[rn[0]], rh]), np.concatenate([rh, [rn[-1]]])
    dch = np.cos(tlo) - np.cos(thi)
    w_r = ((rn[1:] - rn[:-1]) * 2 * math.pi * rh ** 2)[:, None] * dch[None, :]
    w_t = (rn * dth)[:, None] * (math.pi * np.sin(th)[None, :] * (rhi ** 2 - rlo ** 2)[:, None])
    w_p = (2 * math.pi * rn[:, None] * np.sin(tn)[None, :]) * (0.5 * (rhi ** 2 - rlo ** 2)[:, None] * (thi - tlo)[None, :])
    return [w_r, w_t, w_p]


def _jacobian(f, x0: np.ndarray, eps: float = 1e-7) -> np.ndarray:
    y0 = f(x0)
    jac = np.empty((y0.size, x0.size))
    for q in range(x0.size):
        x = x0.copy()
        h = eps * max(1.0, abs(x0[q]))
        x[q] += h
        jac[:, q] = (f(x) - y0) / h
    return jac


def stage(n: int, reading: int) -> dict:
    """Largest singular value of one correction stage in the energy norm, by
    region: interior edges, the band of three columns at the north axis, the
    outer three rows (where the absorber acts) and the inner three rows."""
    cfg = sect4_config(n, reading, geom="michel", allff=True)
    o = Oracle(cfg)
    shapes = [o.shape(k) for k in E_NAMES]
    sizes = [int(np.prod(s)) for s in shapes]
    base_b = {k: o.get(k) for k in ("B_r", "B_th", "B_ph")}

    def f(x):
        for k, part, s in zip(E_NAMES, np.split(x, np.cumsum(sizes)[:-1]), shapes):
            o.set(k, part.reshape(s))
        for k, v in base_b.items():
            o.set(k, v)
        o.step(1, ST_NODE | ST_CORRECT)
        return np.concatenate([o.get(k).ravel() for k in E_NAMES])

    x0 = np.concatenate([o.get(k).ravel() for k in E_NAMES])
    jac = _jacobian(f, x0)
    w = np.concatenate([a.ravel() for a in energy_weights(cfg)])

    def region(r0, r1, j0, j1):
        m = []
        for s in shapes:
            i, j = np.meshgrid(np.arange(s[0]), np.arange(s[1]), indexing="ij")
            m.append(((i >= r0) & (i <= r1) & (j >= j0) & (j <= j1)).ravel())
        return np.concatenate(m) & (w > 0)

    out = {}
    for name, m in (("interior", region(3, n - 4, 3, n - 3)), ("axis band", region(3, n - 4, 0, 2)),
                    ("outer rows", region(n - 3, n, 3, n - 3)), ("inner rows", region(0, 2, 3, n - 3))):
        wh = np.sqrt(w[m])
        s = (wh[:, None] * jac[np.ix_(m, m)]) / wh[None, :]
        out[name] = float(np.linalg.svd(s, compute_uv=False)[0])
    return out


def step(n: int, reading: int, pre: int, top: int = 6, r_abs: float = 0.0) -> list:
    """Eigenvalues of largest modulus of one whole field step of the Sect. 4
    set-up, with the three largest entries of each eigenvector (field name
    and index)."""
    return spectrum(sect4_config(n, reading, r_abs=r_abs), pre, top)


def spectrum(cfg: dict, pre: int, top: int = 6) -> list:
    """Eigenvalues of largest modulus of one whole step of the oracle
    configured by `cfg` (no particles), linearised `pre` steps in."""
    o = Oracle(cfg)
    o.step(pre)
    shapes = [o.shape(k) for k in ALL_NAMES]
    sizes = [int(np.prod(s)) for s in shapes]
    step0 = o.step_index

    def f(x):
        for k, part, s in zip(ALL_NAMES, np.split(x, np.cumsum(sizes)[:-1]), shapes):
            o.set(k, part.reshape(s))
        o.step_index = step0
        o.step(1)
        return np.concatenate([o.get(k).ravel() for k in ALL_NAMES])

    x0 = np.concatenate([o.get(k).ravel() for k in ALL_NAMES])
    ev, vec = np.linalg.eig(_jacobian(f, x0))
    bounds = np.cumsum([0] + sizes)
    out = []
    for k in np.argsort(-np.abs(ev))[:top]:
        where = []
        for q in np.argsort(-np.abs(vec[:, k]))[:3]:
            fi = int(np.searchsorted(bounds, q, side="right") - 1)
            where.append(f"{ALL_NAMES[fi]}{tuple(int(v) for v in np.unravel_index(q - bounds[fi], shapes[fi]))}")
        out.append((float(abs(ev[k])), float(np.angle(ev[k])), where))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", choices=["stage", "step"])
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--reading", type=int, default=1, help="hff_config.ff_delta_only: 0, 1 or 2")
    ap.add_argument("--pre", type=int, default=100, help="steps before the linearisation (step)")
    ap.add_argument("--r-abs", type=float, default=0.0, help="start of the absorber (step; default: see sect4_config)")
    a = ap.parse_args()
    if a.what == "stage":
        for k, v in stage(a.n, a.reading).items():
            print(f"reading {a.reading}, {a.n}^2, {k:10s}: largest singular value {v:.5f}")
    else:
        for mod, arg, where in step(a.n, a.reading, a.pre, r_abs=a.r_abs):
            print(f"reading {a.reading}, {a.n}^2, {a.pre} steps in: |lambda| {mod:.6f} arg {arg:+.4f}  {' '.join(where)}")


if __name__ == "__main__":
    main()
