"""Shared helpers of the parity tests (CUDA path against the FP64 oracle)."""
import math

import numpy as np

FIELDS6 = ("E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph")


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def smooth(shape, seed, amp=1.0):
    """Smooth seeded test field: a few low-order modes over the array."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, shape[0])[:, None]
    y = np.linspace(0.0, 1.0, shape[1])[None, :]
    a = np.zeros(shape)
    for k in range(1, 4):
        A, p1, p2 = rng.normal(), rng.random(), rng.random()
        a += A * np.sin(2 * math.pi * (k * x + p1)) * np.sin(math.pi * (k * y + p2))
    return amp * a / 3.0


def shared_initial_state(sim, ref, seed, e_amp=0.05, bphi_amp=0.05):
    """Give both codes identical FP32-representable fields: the oracle's
    initial B_r, B_th rounded to the GPU precision, plus smooth E and B_phi
    scaled like 1/r^2 so that every force-free branch is exercised."""
    nr = ref.nr
    d = math.log(ref.cfg["r_max"] / ref.cfg["r_min"]) / nr
    real = sim.real
    for name in ("B_r", "B_th"):
        v = ref.get(name).astype(real)
        ref.set(name, v.astype(np.float64))
        sim.set(name, v)
    for k, name in enumerate(("E_r", "E_th", "E_ph", "B_ph")):
        shp = ref.shape(name)
        r = np.exp(np.arange(shp[0]) * d * (nr / max(1, shp[0] - 1)))[:, None]
        amp = bphi_amp if name == "B_ph" else e_amp
        v = (smooth(shp, seed + k, amp) / r ** 2).astype(real)
        if name == "E_ph":
            v[:, 0] = 0
            v[:, -1] = 0
            v[0, :] = 0
            v[-1, :] = 0
        if name == "E_th":
            v[-1, :] = 0
        ref.set(name, v.astype(np.float64))
        sim.set(name, v)


def particle_mismatches(g, o, nt, tol_face=1e-5):
    """Compare index-aligned particle arrays.  Returns (n_bad_cells,
    n_face_ties, max offset error in cells over agreeing cells).  A cell
    mismatch is tolerated only if the oracle's position lies within tol_face
    of a cell face (the FP32 and FP64 floors may differ there)."""
    assert len(g["cell"]) == len(o["cell"]), (len(g["cell"]), len(o["cell"]))
    gc, oc = g["cell"], o["cell"]
    same = gc == oc
    bad = 0
    ties = 0
    for k in np.flatnonzero(~same):
        if oc[k] < 0 or gc[k] < 0:
            # a removal decided differently: allowed only at a face / boundary tie
            xo, yo = o["xo"][k], o["yo"][k]
            near = min(xo, 1 - xo, yo, 1 - yo) < tol_face if oc[k] >= 0 else True
            if near:
                ties += 1
            else:
                bad += 1
            continue
        i0, j0 = divmod(int(oc[k]), nt)
        i1, j1 = divmod(int(gc[k]), nt)
        xi_o, eta_o = i0 + o["xo"][k], j0 + o["yo"][k]
        xi_g, eta_g = i1 + g["xo"][k], j1 + g["yo"][k]
        if abs(xi_o - xi_g) < 2 * tol_face and abs(eta_o - eta_g) < 2 * tol_face:
            ties += 1
        else:
            bad += 1
    live = same & (oc >= 0)
    err = 0.0
    if live.any():
        err = max(np.max(np.abs(g["xo"][live] - o["xo"][live])), np.max(np.abs(g["yo"][live] - o["yo"][live])))
    return bad, ties, float(err)


def michel_fields(cfg, split=False, real=np.float64):
    """Michel's monopole (Eqs. 32-35) on the staggered mesh from its closed
    form: B_r = Psi*/r^2 (exact face average), B_ph = E_th =
    -(Psi*/R_LC) sin(theta)/r at the points of each component, E_r = E_ph =
    B_th = 0.  split=True reverses B and E in the southern hemisphere (the
    split monopole, with its current sheet on the equator).  The southern
    columns are mirrors of the northern ones (nt even), so that the two
    hemispheres are exact negatives of each other when split."""
    nr, nt = cfg["nr"], cfg["nt"]
    assert nt % 2 == 0
    d = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    pst = cfg["b_star"] * cfg["r_min"] ** 2
    rn = cfg["r_min"] * np.exp(np.arange(nr + 1) * d)
    rh = cfg["r_min"] * np.exp((np.arange(nr) + 0.5) * d)
    h = nt // 2
    th = (np.arange(h) + 0.5) * math.pi / nt          # northern half columns
    sgn = -1.0 if split else 1.0

    def mirror(north, odd):
        south = north[:, ::-1] * (sgn if odd else 1.0)
        return np.concatenate([north, south], axis=1)

    br = mirror(np.repeat((pst / rn ** 2)[:, None], h, axis=1), True)
    bp = mirror(-(pst / cfg["r_lc"]) * np.sin(th)[None, :] / rh[:, None], True)
    et = mirror(-(pst / cfg["r_lc"]) * np.sin(th)[None, :] / rn[:, None], True)
    out = {"B_r": br, "B_ph": bp, "E_th": et,
           "E_r": np.zeros((nr, nt + 1)), "E_ph": np.zeros((nr + 1, nt + 1)), "B_th": np.zeros((nr, nt + 1))}
    return {k: v.astype(real) for k, v in out.items()}
