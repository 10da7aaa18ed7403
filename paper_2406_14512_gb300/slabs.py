"""Radial-slab decomposition of one run of the hybrid step across ranks.

The grid of Sect. 4 (r log-spaced, theta uniform on [0, pi]) is cut into
radial slabs.  Rank k owns the node rows [a_k, a_{k+1}) and the half rows
i + 1/2 with i in the same range (the last rank also owns node row nr), over
the whole theta range, so that the flux function of Eq. 27 -- a prefix along
theta -- never crosses a rank.  Each rank computes on its slab widened by
`halo` rows on either side (its local range) and, besides its own work, one
step needs three exchanges with its neighbours:

  1. after the push: the two ranks of a face swap the current their own
     particles deposited in the rows both compute, and each adds the other's
     (the J-halo sum; a particle moves less than a cell per step, so only rows
     next to a face receive any), which makes J complete in every row either
     rank updates -- a halo row's E feeds the first owned row's B within the
     same step;
  2. after the field update: its owned rows of E and B within `halo` of a
     face overwrite the neighbour's copies, so that every rank starts the
     next step with exact halo rows (the dependency depth of one step is
     five rows: collocation, Faraday, Ampere, renormalisation, return to the
     edges);
  3. after the injection: particles whose cell left the owned rows move to
     the rank that owns them.

Slab faces are placed by particle count (the current sheet beyond R_LC makes
the load uneven in r).  A slab's computation is an engine (see SlabEngine);
the exchanges go over torch.distributed with host tensors, so the same code
runs with the gloo backend on CPU ranks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# field components by row type: node rows (i) or half rows (i + 1/2)
NODE_ROWS = ("E_th", "E_ph", "B_r")
HALF_ROWS = ("E_r", "B_th", "B_ph")
J_NODE_ROWS = ("J_th", "J_ph")
J_HALF_ROWS = ("J_r",)
ST_NODE, ST_PUSH, ST_FARADAY1, ST_AMPERE, ST_CORRECT, ST_FARADAY2, ST_INJECT = 1, 4, 8, 16, 2, 32, 64
FIELD_STAGES = ST_FARADAY1 | ST_AMPERE | ST_CORRECT | ST_FARADAY2
DEPENDENCY_ROWS = 5  # rows one step reaches across (see the module docstring)


class SlabEngine:
    """What a slab's computation provides (duck-typed; documentation only).

    lo, hi       local node rows lo .. hi (global indices), hi - lo cells
    nt           cells in theta
    n_species    particle species
    stages(mask) run these stages of one step once, in the step's order,
                 without counting a step
    count_step() the step is complete: advance the step counter (the
                 injection generator's key)
    get(name)    a local array: node-row fields have hi - lo + 1 rows, half-row
                 fields hi - lo rows, theta fastest
    set(name, a) replace a local array
    particles(s) dict of SoA arrays of species s with GLOBAL cell indices
                 (removed particles have cell < 0)
    set_particles(s, d)  replace species s (global cell indices)
    """


@dataclass(frozen=True)
class SlabPlan:
    """Row ownership of every rank: faces[k] .. faces[k+1] - 1 are rank k's
    node rows (faces[-1] == nr; the last rank also owns node row nr)."""
    nr: int
    faces: tuple
    halo: int

    @property
    def world(self) -> int:
        return len(self.faces) - 1

    def owned(self, k: int) -> tuple:
        """Owned node rows [a, b) (the last rank: [a, nr] inclusive, as b = nr + 1)."""
        a, b = self.faces[k], self.faces[k + 1]
        return a, (b + 1 if k == self.world - 1 else b)

    def owned_half(self, k: int) -> tuple:
        return self.faces[k], self.faces[k + 1]

    def local(self, k: int) -> tuple:
        """Local node rows lo .. hi of rank k (its owned rows widened by the halo)."""
        return max(0, self.faces[k] - self.halo), min(self.nr, self.faces[k + 1] + self.halo)

    def owner(self, row: np.ndarray) -> np.ndarray:
        """Rank owning each node row."""
        k = np.searchsorted(np.asarray(self.faces[1:-1]), row, side="right")
        return k.astype(np.int64)


def partition_rows(row_counts: np.ndarray, world: int, halo: int, min_rows: int | None = None) -> SlabPlan:
    """Slab faces that split the particles as evenly as the rows allow.

    row_counts[i] = particles in cell row i (nr values).  Every slab keeps at
    least `min_rows` rows (default: the halo plus the dependency depth, so that
    a neighbour's halo never reaches past a slab)."""
    nr = len(row_counts)
    if min_rows is None:
        min_rows = halo + DEPENDENCY_ROWS
    if world < 1 or world * min_rows > nr:
        raise ValueError(f"cannot cut {nr} rows into {world} slabs of at least {min_rows} rows")
    if halo < DEPENDENCY_ROWS:
        raise ValueError(f"halo {halo} is below the {DEPENDENCY_ROWS} rows one step depends on")
    cum = np.concatenate([[0], np.cumsum(np.asarray(row_counts, np.float64))])
    total = cum[-1]
    faces = [0]
    for k in range(1, world):
        target = total * k / world
        f = int(np.searchsorted(cum, target, side="left"))
        lo_ok = faces[-1] + min_rows
        hi_ok = nr - (world - k) * min_rows
        faces.append(min(max(f, lo_ok), hi_ok))
    faces.append(nr)
    return SlabPlan(nr=nr, faces=tuple(int(f) for f in faces), halo=int(halo))


def row_counts(cells: list, nr: int, nt: int) -> np.ndarray:
    """Particles per cell row from global cell indices (removed ones skipped)."""
    out = np.zeros(nr, np.int64)
    for c in cells:
        c = np.asarray(c)
        live = c[c >= 0]
        out += np.bincount(live // nt, minlength=nr)[:nr]
    return out


class SlabRun:
    """Steps one rank's slab of a decomposed run and does its exchanges.

    engine : the rank's SlabEngine, built on plan.local(rank)
    plan   : the SlabPlan shared by all ranks
    dist   : torch.distributed (initialised; any backend that moves CPU tensors)
    """

    def __init__(self, engine, plan: SlabPlan, rank: int, dist):
        self.e, self.plan, self.rank, self.dist = engine, plan, rank, dist
        lo, hi = plan.local(rank)
        if (engine.lo, engine.hi) != (lo, hi):
            raise ValueError(f"engine rows {engine.lo}..{engine.hi} are not the plan's {lo}..{hi}")
        self.neighbours = [k for k in (rank - 1, rank + 1) if 0 <= k < plan.world]

    # -- row bookkeeping ---------------------------------------------------
    def _overlap(self, owner: int, viewer: int, half: bool) -> tuple:
        """Global rows [a, b) that `owner` owns and that lie in `viewer`'s
        local range (node rows lo .. hi, half rows lo .. hi - 1)."""
        a, b = self.plan.owned_half(owner) if half else self.plan.owned(owner)
        lo, hi = self.plan.local(viewer)
        a, b = max(a, lo), min(b, hi if half else hi + 1)
        return a, max(a, b)

    def _send_recv(self, k: int, payload: np.ndarray, n_recv: int) -> np.ndarray:
        """Exchange one float64 buffer with neighbour k (lower rank sends first)."""
        import torch
        send = torch.from_numpy(np.ascontiguousarray(payload, np.float64))
        recv = torch.empty(n_recv, dtype=torch.float64)
        if self.rank < k:
            self.dist.send(send, dst=k)
            self.dist.recv(recv, src=k)
        else:
            self.dist.recv(recv, src=k)
            self.dist.send(send, dst=k)
        return recv.numpy()

    def _common(self, k: int, half: bool) -> tuple:
        """Global rows [a, b) in both this rank's and neighbour k's local range."""
        lo0, hi0 = self.plan.local(self.rank)
        lo1, hi1 = self.plan.local(k)
        a, b = max(lo0, lo1), min(hi0, hi1) + (0 if half else 1)
        return a, max(a, b)

    def _exchange_rows(self, node_names, half_names, deposits: bool):
        """deposits = True (J-halo sum): the two ranks swap their own partial
        deposits over every row both compute and each adds the other's, so that
        J is complete wherever either rank evaluates the field update.
        deposits = False (E, B halo): each rank sends its owned rows inside a
        neighbour's local range, which overwrite the neighbour's copy."""
        e, me = self.e, self.rank
        items = [(n, False) for n in node_names] + [(n, True) for n in half_names]
        arrs = {n: e.get(n) for n, _ in items}
        own = {n: a.copy() for n, a in arrs.items()} if deposits else arrs
        for k in self.neighbours:
            send, recv_rows = [], []
            for name, half in items:
                if deposits:
                    sa, sb = ra, rb = self._common(k, half)
                else:
                    sa, sb = self._overlap(me, k, half)
                    ra, rb = self._overlap(k, me, half)
                send.append(own[name][sa - e.lo:sb - e.lo].ravel())
                recv_rows.append((name, ra, rb))
            n_recv = sum((rb - ra) * arrs[n].shape[1] for n, ra, rb in recv_rows)
            got = self._send_recv(k, np.concatenate(send), n_recv)
            off = 0
            for name, ra, rb in recv_rows:
                arr = arrs[name]
                n = (rb - ra) * arr.shape[1]
                block = got[off:off + n].reshape(rb - ra, arr.shape[1])
                if deposits:
                    arr[ra - e.lo:rb - e.lo] += block
                else:
                    arr[ra - e.lo:rb - e.lo] = block
                off += n
        for name, _ in items:
            e.set(name, arrs[name])

    def exchange_current(self):
        """J-halo sum: my deposits in a neighbour's rows go to the neighbour."""
        self._exchange_rows(J_NODE_ROWS, J_HALF_ROWS, deposits=True)

    def exchange_fields(self):
        """E and B halo rows: my owned rows overwrite the neighbours' copies."""
        self._exchange_rows(NODE_ROWS, HALF_ROWS, deposits=False)

    def migrate(self):
        """Particles whose cell row left this rank's rows go to their owner;
        removed particles are dropped."""
        e, nt = self.e, self.e.nt
        a, b = self.plan.owned(self.rank)
        keys = ("cell", "xo", "yo", "ur", "ut", "up", "w")
        for s in range(e.n_species):
            p = e.particles(s)
            cell = np.asarray(p["cell"])
            live = cell >= 0
            row = np.where(live, cell // nt, -1)
            stay = live & (row >= a) & (row < b)
            kept = {k: np.asarray(p[k])[stay] for k in keys}
            for k in self.neighbours:
                ka, kb = self.plan.owned(k)
                go = live & (row >= ka) & (row < kb)
                out = np.stack([np.asarray(p[q], np.float64)[go] for q in keys]) if go.any() else np.zeros((7, 0))
                n_out = np.array([out.shape[1]], np.float64)
                n_in = int(self._send_recv(k, n_out, 1)[0])
                got = self._send_recv(k, out.ravel(), 7 * n_in).reshape(7, n_in)
                for i, q in enumerate(keys):
                    dt = np.int32 if q == "cell" else kept[q].dtype
                    kept[q] = np.concatenate([kept[q], got[i].astype(dt)])
            lost = live & ~stay
            for k in self.neighbours:
                ka, kb = self.plan.owned(k)
                lost &= ~((row >= ka) & (row < kb))
            if lost.any():
                raise RuntimeError("a particle moved past a neighbouring slab in one step")
            e.set_particles(s, kept)

    def step(self, n: int = 1):
        """n whole steps of the decomposed run."""
        for _ in range(n):
            self.e.stages(ST_NODE | ST_PUSH)
            self.exchange_current()
            self.e.stages(FIELD_STAGES)
            self.exchange_fields()
            self.e.stages(ST_INJECT)
            self.e.count_step()
            self.migrate()


def slab_config(cfg: dict, lo: int, hi: int) -> dict:
    """The configuration of a slab on node rows lo .. hi of the run `cfg`:
    the same log grid cut at r_lo and r_hi, the same magnetic moment (flux
    unit) and time step, injection only on the slab that holds the star.  An
    absorber start beyond the slab's r_max leaves the slab without one."""
    d = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
    r_lo, r_hi = cfg["r_min"] * math.exp(lo * d), cfg["r_min"] * math.exp(hi * d)
    c = dict(cfg, nr=hi - lo, r_min=r_lo, r_max=r_hi, inject=bool(cfg.get("inject")) and lo == 0)
    mono = cfg.get("geom") in ("monopole", "michel")
    c["b_star"] = cfg.get("b_star", 1.0) * (cfg["r_min"] / r_lo) ** (2 if mono else 3)
    c["r_abs"] = cfg.get("r_abs", 3.0 * cfg["r_lc"])
    c["shell_r"] = cfg.get("shell_r", 2.0 * cfg["r_min"])
    c["courant"] = cfg.get("courant", 0.5) * _min_cell_limit(cfg) / _min_cell_limit(c)
    return c


def _min_cell_limit(c: dict) -> float:
    """The 2D light-crossing limit of the smallest cell of a log grid, which
    the Courant rule scales (the innermost cell)."""
    d, dth = math.log(c["r_max"] / c["r_min"]) / c["nr"], math.pi / c["nt"]
    dr = c["r_min"] * (math.exp(d) - 1.0)
    return 1.0 / math.sqrt(1.0 / dr ** 2 + 1.0 / (c["r_min"] * dth) ** 2)


class LibrarySlab:
    """A slab computed by the CUDA library: one instance (hff.Sim) on the
    slab's local rows, stepped in stage groups with hff_step_stages (the
    first two groups do not count a step; the injection group does).

    fields: global E and B arrays (node- and half-row shaped, as hff_fields
    returns them) that initialise the slab's rows."""

    HALF = {"E_r", "B_th", "B_ph", "J_r"}

    def __init__(self, cfg: dict, lo: int, hi: int, fields: dict, device: str = "cuda:0"):
        from . import hff
        self.hff = hff
        self.cfg = slab_config(cfg, lo, hi)
        self.sim = hff.Sim(self.cfg, device=device)
        self.lo, self.hi, self.nt, self.n_species = lo, hi, cfg["nt"], len(cfg.get("q", [-1.0, 1.0]))
        for name, a in fields.items():
            self.sim.set(name, a[lo:hi if name in self.HALF else hi + 1])

    def stages(self, mask: int) -> None:
        st = self.hff.ST
        if not mask & st["inject"]:
            mask |= st["nocount"]
        self.sim.step_stages(1, mask)

    def count_step(self) -> None:
        pass  # the injection group counted it

    def get(self, name: str):
        return self.sim.get(name).astype(np.float64)

    def set(self, name: str, a) -> None:
        self.sim.set(name, a)

    def particles(self, s: int) -> dict:
        p = self.sim.particles(s)
        c = p["cell"]
        p["cell"] = np.where(c >= 0, c + self.lo * self.nt, -1).astype(np.int32)
        return p

    def set_particles(self, s: int, p: dict) -> None:
        q = {k: np.asarray(v) for k, v in p.items()}
        q["cell"] = np.where(q["cell"] >= 0, q["cell"] - self.lo * self.nt, -1).astype(np.int32)
        self.sim.load(s, q)

    def close(self) -> None:
        self.sim.close()
