"""Long-run precision: the FP32 and FP64 instantiations of the same kernels
run the 1024 x 1024 hybrid workload (5e7 e+-, Table 1 flux bands, 2000
steps) from the same inputs; the spin-down power L(r) inside 3 R_LC, the
open flux Psi(2 R_LC, pi/2), the field and kinetic energies and the live
count must stay within 2% of each other at every checkpoint (the tolerance
for long runs; particle trajectories decorrelate at face ties, so element
comparisons no longer apply)."""
import gc
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STEPS, EVERY = 2000, 500


def run(hff, cfg, ps, precision):
    import torch
    sim = hff.Sim(dict(cfg, precision=precision))
    for s in range(2):
        sim.load(s, ps[s])
    out = []
    for _ in range(STEPS // EVERY):
        sim.step(EVERY)
        d, prof = sim.diagnostics()
        out.append(dict(psi_open=d.psi_open, u_e=d.u_e, u_b=d.u_b, kin=d.kinetic[0] + d.kinetic[1],
                        count=d.count[0] + d.count[1], prof=prof.copy(), nonfinite=d.nonfinite))
    status = sim.status()
    sim.close()
    del sim.mem
    gc.collect()
    torch.cuda.empty_cache()
    return out, status


def test_c2_fp32_vs_fp64_long_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_14512_gb300 import hff, workloads
    cfg = workloads.config("c2")
    cfg["capacity"] = int(cfg["n_pairs"] * 1.3) + 100_000
    ps = workloads.particles(cfg, threads=16)
    a, sa = run(hff, cfg, ps, "fp32")
    b, sb = run(hff, cfg, ps, "fp64")
    assert sa == 0 and sb == 0
    nr = cfg["nr"]
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    rh = cfg["r_min"] * np.exp((np.arange(nr) + 0.5) * d)
    inside = rh <= 3 * cfg["r_lc"]
    for x, y in zip(a, b):
        assert x["nonfinite"] == 0 and y["nonfinite"] == 0
        for k in ("psi_open", "u_e", "u_b", "kin", "count"):
            assert abs(x[k] - y[k]) <= 0.02 * abs(y[k]), (k, x[k], y[k])
        lp, lq = x["prof"][inside], y["prof"][inside]
        assert np.linalg.norm(lp - lq) <= 0.02 * np.linalg.norm(lq)
