"""The force-free / PIC decision of Eqs. 29-31 at near-ties, through the C ABI.

On a monopole every equatorial node has Psi = Psi* up to the rounding of the
B_r it is summed from, so the nodes and radial edges of the equator sit within
about 1e-8 of each other.  Jumps of f placed between adjacent values of the
oracle's FP64 Psi there make every one of those decisions depend on the
precision of Psi: the library's flags and weights must equal the oracle's
exactly, in FP32 instances (Psi as a float pair summed from exact products)
as in FP64 ones.  A Psi rounded to FP32 (6e-8 relative) would put many of
them on the wrong side.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ST_NODE = 1


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2406_14512_gb300 import hff, workloads
    return hff, workloads, oracle


def _shared_b(sim, ref, real):
    """The same B in both codes: the oracle's, rounded through FP32 (exact in
    either precision), which also spreads the equatorial Psi over ~1e-8."""
    for name in ("B_r", "B_th", "B_ph"):
        v = ref.get(name).astype(np.float32)
        ref.set(name, v.astype(np.float64))
        sim.set(name, v.astype(real))


def _oracle_weights(ref):
    """f at the E_r edges, E_th edges and nodes, and the cell flags, from the
    oracle's Psi with the oracle's own blend (edge and cell means as its
    correction and push take them)."""
    psi = ref.get("psi")
    bl = np.vectorize(ref.blend)
    f_r = bl(0.5 * (psi[:-1, :] + psi[1:, :]))
    f_th = bl(0.5 * (psi[:, :-1] + psi[:, 1:]))
    f_n = bl(psi)
    cell = 0.25 * (psi[:-1, :-1] + psi[1:, :-1] + psi[:-1, 1:] + psi[1:, 1:])
    return f_r, f_th, f_n, (bl(cell) >= 1.0).astype(np.uint8), psi


def _near_tie_breaks(psi_eq):
    """Two jumps (0 -> 1 -> 0) at mid-points between adjacent distinct values
    near the 30% and 70% quantiles of the equatorial values."""
    v = np.unique(psi_eq)
    ks = [int(0.3 * (len(v) - 1)), int(0.7 * (len(v) - 1))]
    out = []
    for k in ks:
        while v[k + 1] - v[k] < 1e-13 * abs(v[k]):  # a gap the rounding cannot bridge
            k += 1
        out.append(0.5 * (v[k] + v[k + 1]))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_blend_decisions_at_near_ties_equal_the_oracle(env, prec):
    hff, workloads, oracle = env
    base = workloads.config("small_michel")
    base.update(precision=prec, capacity=0, inject=False, psi_break=[], f_break=[])
    real = np.float64 if prec == "fp64" else np.float32
    # the oracle's Psi from the shared (instance-precision) B
    probe_sim, probe = hff.Sim(base), oracle.Oracle(base)
    _shared_b(probe_sim, probe, real)
    probe.step(1, stages=ST_NODE)
    psi = probe.get("psi")
    nt = base["nt"]
    eq = np.concatenate([psi[:, nt // 2], 0.5 * (psi[:-1, nt // 2] + psi[1:, nt // 2])])
    a, b = _near_tie_breaks(eq)
    unit = probe.psi_unit
    # the test is only meaningful if many decisions are close calls
    close = np.sum(np.minimum(np.abs(eq - a), np.abs(eq - b)) < 1e-7 * abs(a))
    assert close >= 20, close
    probe_sim.close()

    cfg = dict(base, psi_break=[a / unit, a / unit, b / unit, b / unit], f_break=[0.0, 1.0, 1.0, 0.0])
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    _shared_b(sim, ref, real)
    ref.step(1, stages=ST_NODE)
    f_r, f_th, f_n, cells, _ = _oracle_weights(ref)
    assert 0 < f_r.sum() < f_r.size and 0 < f_n.sum() < f_n.size
    for name, want in (("f_r", f_r), ("f_th", f_th), ("f_node", f_n)):
        got = sim.get(name).astype(np.float64)
        bad = np.argwhere(got != want)
        assert len(bad) == 0, (name, len(bad), bad[:5])
    assert np.array_equal(sim.get("ff_cell"), cells)
    sim.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_blend_ramps_of_table1_match_the_oracle(env, prec):
    """The Table 1 bands (linear ramps) on the synthetic dipole: weights within
    FP32 (or FP64) rounding, force-free cell flags identical."""
    hff, workloads, oracle = env
    cfg = workloads.config("small_hybrid")
    cfg.update(precision=prec, capacity=0, inject=False)
    real = np.float64 if prec == "fp64" else np.float32
    sim, ref = hff.Sim(cfg), oracle.Oracle(cfg)
    _shared_b(sim, ref, real)
    ref.step(1, stages=ST_NODE)
    f_r, f_th, f_n, cells, _ = _oracle_weights(ref)
    tol = 1e-12 if prec == "fp64" else 2e-6
    for name, want in (("f_r", f_r), ("f_th", f_th), ("f_node", f_n)):
        got = sim.get(name).astype(np.float64)
        assert np.abs(got - want).max() <= tol, name
        assert ((0 < want) & (want < 1)).sum() > 50  # the ramps are exercised
    assert np.array_equal(sim.get("ff_cell"), cells)
    sim.close()
