"""The monopole convergence run of Sect. 4 on the GPU.

Set-up (Sect. 4): r in [r*, (10/3) R_LC] with R_LC = 5 r*, log-spaced in r,
uniform in theta over [0, pi]; a vacuum radial field B = B* (r*/r)^2; the
corotating star; the absorber from 3 R_LC; the northern hemisphere in PIC
(f = 0 below Psi*) with electron-positron pairs injected at the surface at
kappa = 10, the southern one force-free (f = 1 above Psi*), a sharp cut at
the equator; no pair creation.  After `periods` spin periods the run reports
the dissipation rate of Eq. 36 (L averaged over [r*, 2 r*] and [2, 3] R_LC),
both averages against Michel's spin-down L_M = 2 Psi*^2 Omega^2 / 3c, and the
relative L2 distance of the toroidal field at 1.5 R_LC from Michel's
B_ph = -(Psi*/R_LC) sin(theta) / r in each hemisphere.

    python -m paper_2406_14512_gb300.monopole --n 1024 --periods 2
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def config(n: int, layer: float = 0.0, ppc: float = 4.0, **kw) -> dict:
    """layer = 0: the sharp cut at Psi = Psi* (placed a hair below it so that
    the equatorial nodes fall deterministically on the force-free side);
    layer > 0: f rises linearly from 0 at (1 - layer) Psi* to 1 there.
    ppc: injected pairs in the fullest surface cell (sets the macro weight)."""
    from . import workloads
    r_lc = 5.0
    c = workloads._base(n, n, 10.0 / 3.0 * r_lc, r_lc, "monopole", kappa=10.0, ppc_inj=ppc, seed=4242)
    c["ppc"] = ppc
    cut = 1.0 - 1e-4
    c.update(psi_break=[cut - layer, cut], f_break=[0.0, 1.0], n_pairs=0, precision="fp32",
             r_abs=3.0 * r_lc, inject=True, place="uniform", momenta="maxwell")
    c["capacity"] = int(kw.pop("capacity", int(8 * ppc) * n * n))
    c.update(kw)
    return c


def michel(cfg) -> dict:
    psi_star = cfg["b_star"] * cfg["r_min"] ** 2
    omega = 1.0 / cfg["r_lc"]
    return {"L_M": 2.0 * psi_star ** 2 * omega ** 2 / 3.0, "psi_star": psi_star}


def bphi_error(sim, cfg) -> dict:
    """Relative L2 distance of B_ph at the half-node row nearest 1.5 R_LC
    from Michel's solution, per hemisphere."""
    nr, nt = cfg["nr"], cfg["nt"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    i = int(round(math.log(1.5 * cfg["r_lc"] / cfg["r_min"]) / d - 0.5))
    r = cfg["r_min"] * math.exp((i + 0.5) * d)
    th = (np.arange(nt) + 0.5) * math.pi / nt
    exact = -(michel(cfg)["psi_star"] / cfg["r_lc"]) * np.sin(th) / r
    bp = sim.get("B_ph")[i].astype(np.float64)
    north, south = th < math.pi / 2, th > math.pi / 2
    err = {}
    for name, m in (("north_pic", north), ("south_ff", south)):
        err[name] = float(np.linalg.norm(bp[m] - exact[m]) / np.linalg.norm(exact[m]))
    return err


def run(n: int = 1024, periods: float = 2.0, chunk: int = 2000, log=None, layer: float = 0.0, **kw) -> dict:
    import torch
    from . import hff
    cfg = config(n, layer=layer, **kw)
    sim = hff.Sim(cfg)
    dt = sim.info().dt
    steps = int(round(periods * 2.0 * math.pi * cfg["r_lc"] / dt))
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        sim.step(k)
        done += k
        if log:
            torch.cuda.synchronize()
            d, _ = sim.diagnostics()
            log(f"[monopole {n}^2] step {done}/{steps}: eps {d.eps:.4f} "
                f"L_in/L_M {d.l_in / michel(cfg)['L_M']:.4f} live {d.count[0] + d.count[1]:.3g}")
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    d, prof = sim.diagnostics()
    lm = michel(cfg)["L_M"]
    out = {"n": n, "periods": periods, "layer": layer, "precision": cfg["precision"],
           "ff_delta_only": cfg.get("ff_delta_only", 0),
           "ff_filter": cfg.get("ff_filter", 0.0),
           "ppc": cfg["ppc"],
           "steps": steps, "dt": dt, "wall_s": wall,
           "eps": d.eps, "L_in_over_L_M": d.l_in / lm, "L_out_over_L_M": d.l_out / lm,
           "bphi_rel_err_1p5_rlc": bphi_error(sim, cfg), "live_particles": d.count[0] + d.count[1],
           "status": sim.status(), "nonfinite": d.nonfinite}
    sim.close()
    return out


def main():
    import sys
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--periods", type=float, default=2.0)
    ap.add_argument("--chunk", type=int, default=2000)
    ap.add_argument("--layer", type=float, default=0.0, help="transition layer width in Psi* (0 = sharp cut)")
    ap.add_argument("--ff-delta-only", type=int, default=0,
                    help="0: the corrected E returns to the edges (Sect. 3); 1: only the corrections "
                         "Delta E; 2: the corrections, the corrected E on the radial edges at the star")
    ap.add_argument("--ppc", type=float, default=4.0, help="largest injected pairs per surface cell")
    ap.add_argument("--ff-filter", type=float, default=0.0,
                    help="sigma of the fourth-difference filter of E_r, E_th (0 = off)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32",
                    help="fields and particles in FP32 (production) or FP64")
    a = ap.parse_args()
    kw = {"ff_delta_only": a.ff_delta_only, "ppc": a.ppc, "ff_filter": a.ff_filter, "precision": a.precision}
    print(json.dumps(run(a.n, a.periods, a.chunk, log=lambda m: print(m, file=sys.stderr, flush=True),
                         layer=a.layer, **kw)))


if __name__ == "__main__":
    main()
