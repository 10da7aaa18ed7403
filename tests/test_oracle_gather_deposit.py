"""Pins of the oracle's on-mesh gather and of the azimuthal part of its
deposit (Sect. 3: linear weights on the staggered mesh; J_phi at the nodes
from the mid-point of the move).

The gather is pinned by the interpolation error: fields given by smooth
closed forms at their staggered locations are gathered at fixed physical
points and must converge to the closed forms at second order (a misplaced
stagger or weight leaves a first-order or O(1) error).  The uniform B_z the
oracle builds from its flux function gives B_r = B cos(theta),
B_theta = -B sin(theta).

J_phi is pinned by charge: the node values times the node dual volumes sum
to q w v_phi for any move, and they equal v_phi times the cloud-in-cell node
charge of a particle standing at the mid-point of the move (an independent
routine of the oracle, the one Gauss's law is checked with)."""
import math

import numpy as np
import pytest

R_MIN, R_MAX = 1.0, 8.0


def _cfg(n, geom="uniform", nt=None):
    return dict(nr=n, nt=nt or n, r_min=R_MIN, r_max=R_MAX, r_lc=3.0, geom=geom, b_star=1.0,
                capacity=16, n_breaks=0)


# closed forms per component (distinct in r and theta, so a swapped or
# misplaced component cannot pass)
FORMS = {
    "E_r": lambda r, t: np.cos(t) / r,
    "E_th": lambda r, t: np.sin(t) * np.sqrt(r),
    "E_ph": lambda r, t: np.sin(t) * np.cos(t) * r,
    "B_r": lambda r, t: np.cos(2 * t) * (1.0 + 0.1 * r),
    "B_th": lambda r, t: -np.sin(t) / r ** 2,
    "B_ph": lambda r, t: np.sin(t) ** 2 * np.log(r + 1.0),
}
# staggering of each component: (half in r, half in theta)
STAG = {"E_r": (1, 0), "E_th": (0, 1), "E_ph": (0, 0), "B_r": (0, 1), "B_th": (1, 0), "B_ph": (1, 1)}


def _load_forms(o):
    d = math.log(R_MAX / R_MIN) / o.nr
    dth = math.pi / o.nt
    for name, f in FORMS.items():
        shp = o.shape(name)
        hr, ht = STAG[name]
        r = R_MIN * np.exp((np.arange(shp[0]) + 0.5 * hr) * d)[:, None]
        t = ((np.arange(shp[1]) + 0.5 * ht) * dth)[None, :]
        o.set(name, f(r, t) * np.ones(shp))


def _points():
    rng = np.random.default_rng(7)
    return rng.uniform(1.6, 6.0, 40), rng.uniform(0.35, math.pi - 0.35, 40)


OFFSETS = ((0.37, 0.61), (0.83, 0.12), (0.5, 0.5), (0.08, 0.94))


def _locate(o, r, t, off):
    """The cell holding the physical point (r, t), and a fixed offset inside it,
    so that the leading interpolation error scales as h^2 between grids."""
    d, dth = math.log(R_MAX / R_MIN) / o.nr, math.pi / o.nt
    i, j = int(math.floor(math.log(r / R_MIN) / d)), int(math.floor(t / dth))
    xo, yo = off
    return i, j, xo, yo, R_MIN * math.exp((i + xo) * d), (j + yo) * dth


def _gather_errors(oracle_mod, n):
    o = oracle_mod.Oracle(_cfg(n))
    _load_forms(o)
    rs, ts = _points()
    err = {k: 0.0 for k in FORMS}
    for r0, t0 in zip(rs, ts):
        for off in OFFSETS:
            i, j, xo, yo, r, t = _locate(o, r0, t0, off)
            e, b = o.gather(i, j, xo, yo)
            got = dict(zip(("E_r", "E_th", "E_ph"), e)) | dict(zip(("B_r", "B_th", "B_ph"), b))
            for k, f in FORMS.items():
                err[k] = max(err[k], abs(got[k] - f(r, t)))
    return err


def test_gather_converges_at_second_order_on_the_staggered_mesh(oracle_mod):
    errs = [_gather_errors(oracle_mod, n) for n in (24, 48, 96)]
    for k in FORMS:
        e = [x[k] for x in errs]
        rates = [math.log2(e[m] / e[m + 1]) for m in range(2)]
        assert all(q > 1.8 for q in rates), (k, e, rates)
        assert e[-1] < 2e-3, (k, e)


def test_gather_of_the_uniform_field(oracle_mod):
    """B_z = 1 built from Psi = r^2 sin^2(theta)/2 by exact face fluxes; E_z = 0.3
    given at the E locations.  Gathered in the local basis: (cos, -sin) x field,
    second order."""
    errs = []
    for n in (24, 48, 96):
        o = oracle_mod.Oracle(_cfg(n))
        d, dth = math.log(R_MAX / R_MIN) / n, math.pi / n
        r_h = R_MIN * np.exp((np.arange(n) + 0.5) * d)[:, None]
        t_n = (np.arange(n + 1) * dth)[None, :]
        t_h = ((np.arange(n) + 0.5) * dth)[None, :]
        o.set("E_r", 0.3 * np.cos(t_n) * np.ones_like(r_h))
        o.set("E_th", -0.3 * np.sin(t_h) * np.ones((n + 1, n)))
        o.set("E_ph", np.zeros((n + 1, n + 1)))
        rs, ts = _points()
        worst = 0.0
        for r0, t0 in zip(rs, ts):
            for off in OFFSETS:
                i, j, xo, yo, r, t = _locate(o, r0, t0, off)
                e, b = o.gather(i, j, xo, yo)
                ref_b = np.array([math.cos(t), -math.sin(t), 0.0])
                ref_e = 0.3 * ref_b
                worst = max(worst, np.abs(b - ref_b).max(), np.abs(e - ref_e).max())
        errs.append(worst)
    rates = [math.log2(errs[m] / errs[m + 1]) for m in range(2)]
    assert all(q > 1.8 for q in rates), (errs, rates)
    assert errs[-1] < 1e-3


def _node_volumes(o):
    """Exact volumes of the node dual cells (half-node bounds, clipped at
    r_min, r_max and the axis)."""
    nr, nt = o.nr, o.nt
    d, dth = math.log(R_MAX / R_MIN) / nr, math.pi / nt
    rh = R_MIN * np.exp((np.arange(nr) + 0.5) * d)
    rlo = np.concatenate([[R_MIN], rh])
    rhi = np.concatenate([rh, [R_MAX]])
    th = (np.arange(nt) + 0.5) * dth
    tlo = np.concatenate([[0.0], th])
    thi = np.concatenate([th, [math.pi]])
    return (2 * math.pi / 3) * (rhi ** 3 - rlo ** 3)[:, None] * (np.cos(tlo) - np.cos(thi))[None, :]


def _moves(seed, n, nr, nt):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        i0, j0 = int(rng.integers(2, nr - 3)), int(rng.integers(2, nt - 3))
        x0, y0 = rng.random(), rng.random()
        x1, y1 = x0 + rng.uniform(-0.45, 0.45), y0 + rng.uniform(-0.45, 0.45)
        yield i0, j0, x0, y0, x1, y1, rng.choice([-1.0, 1.0]) * rng.uniform(0.2, 2.0), rng.uniform(-0.9, 0.9)


def test_jphi_deposit_carries_q_w_vphi(oracle_mod):
    o = oracle_mod.Oracle(_cfg(20, nt=18))
    vol = _node_volumes(o)
    zero = {k: np.zeros(o.shape(k)) for k in ("J_r", "J_th", "J_ph")}
    for mv in _moves(3, 60, o.nr, o.nt):
        i0, j0, x0, y0, x1, y1, qw, v = mv
        for k, z in zero.items():
            o.set(k, z)
        o.deposit(qw, i0, j0, x0, y0, x1, y1, v)
        tot = float((o.get("J_ph") * vol).sum())
        assert abs(tot - qw * v) <= 1e-13 * abs(qw * v), (mv, tot)


def test_jphi_deposit_is_vphi_times_the_midpoint_charge(oracle_mod):
    o = oracle_mod.Oracle(_cfg(20, nt=18))
    vol = _node_volumes(o)
    nt = o.nt
    for mv in _moves(5, 60, o.nr, nt):
        i0, j0, x0, y0, x1, y1, qw, v = mv
        for k in ("J_r", "J_th", "J_ph"):
            o.set(k, np.zeros(o.shape(k)))
        o.deposit(qw, i0, j0, x0, y0, x1, y1, v)
        # a particle of charge qw standing at the mid-point of the move
        xm, ym = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        di, dj = math.floor(xm), math.floor(ym)
        o.set_particles(0, dict(cell=[(i0 + di) * nt + j0 + dj], xo=[xm - di], yo=[ym - dj],
                                ur=[0.0], ut=[0.0], up=[0.0], w=[abs(qw)]))
        o.set_particles(1, dict(cell=[], xo=[], yo=[], ur=[], ut=[], up=[], w=[]))
        q = o.node_charge() * (1.0 if qw < 0 else -1.0)  # species 0 has charge -1
        jv = o.get("J_ph") * vol
        assert np.abs(jv - v * q).max() <= 1e-13 * abs(qw * v), mv
        # nothing beyond the 2 x 2 nodes around the mid-point
        assert np.count_nonzero(jv) <= 4
