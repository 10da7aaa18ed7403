"""ctypes wrapper of the plain FP64 CPU oracle (``hff_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers, besides this package's
own stability analysis of the field return (``field_return_analysis``, run by
hand and by the tests).  The product path never imports this package.  Configuration arrives as a plain dict (the workload
description of ``paper_2406_14512_gb300.workloads``); nothing here is shared
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hff_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FIELD_NAMES = ["E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph", "J_r", "J_th", "J_ph",
               "psi", "jperp_r", "jperp_th", "jperp_ph", "dE_r", "dE_th", "dE_ph",
               "B0_r", "B0_th", "B0_ph"]
GEOM = {"dipole": 0, "monopole": 1, "synth": 2, "uniform": 3, "michel": 4}
ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64,
          sort=128, all=255)


class _Cfg(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nt", C.c_int32),
        ("r_min", C.c_double), ("r_max", C.c_double), ("r_lc", C.c_double),
        ("b_star", C.c_double), ("geom", C.c_int32), ("courant", C.c_double),
        ("r_abs", C.c_double), ("absorb_strength", C.c_double),
        ("n_breaks", C.c_int32), ("psi_break", C.c_double * 4), ("f_break", C.c_double * 4),
        ("n_species", C.c_int32), ("q", C.c_double * 4), ("m", C.c_double * 4),
        ("inject", C.c_int32), ("kappa_inj", C.c_double), ("w_inj", C.c_double),
        ("gamma_rad", C.c_double), ("b_ref", C.c_double), ("rr_scale", C.c_double),
        ("shell_r", C.c_double), ("synth_psi_open", C.c_double),
        ("seed", C.c_uint64), ("capacity", C.c_int64),
        ("tile_r", C.c_int32), ("tile_t", C.c_int32), ("sort_every", C.c_int32),
        ("gamma_th", C.c_double), ("gamma_s", C.c_double), ("inject_species", C.c_int32 * 2),
        ("ff_delta_only", C.c_int32), ("ff_filter", C.c_double),
    ]


class Diag(C.Structure):
    _fields_ = [
        ("psi_open", C.c_double), ("eps", C.c_double), ("l_in", C.c_double),
        ("l_out", C.c_double), ("gauss_max", C.c_double), ("gauss_rms", C.c_double),
        ("rho_max", C.c_double), ("u_e", C.c_double), ("u_b", C.c_double),
        ("kinetic", C.c_double * 4), ("count", C.c_double * 4),
        ("injected", C.c_double), ("killed", C.c_double), ("radiated", C.c_double),
        ("nonfinite", C.c_double), ("created", C.c_double), ("clamps", C.c_double),
        ("nonfinite_fields", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, -O2, no -march)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(os.path.dirname(_SRC), "hff_oracle.h")))
        if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
            os.makedirs(os.path.dirname(_OUT), exist_ok=True)
            tmp = _OUT + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp,
                                   _SRC, "-lm"])
            os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, d, i32, i64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
        pd = C.POINTER(C.c_double)
        L.or_create.restype = vp
        L.or_create.argtypes = [C.POINTER(_Cfg)]
        L.or_destroy.argtypes = [vp]
        L.or_config_dt.restype = d
        L.or_config_dt.argtypes = [C.POINTER(_Cfg)]
        L.or_dt.restype = d
        L.or_dt.argtypes = [vp]
        L.or_psi_unit.restype = d
        L.or_psi_unit.argtypes = [vp]
        L.or_step_index.restype = i64
        L.or_step_index.argtypes = [vp]
        L.or_set_step_index.argtypes = [vp, i64]
        L.or_field_size.restype = i64
        L.or_field_size.argtypes = [vp, C.c_int]
        L.or_get_field.argtypes = [vp, C.c_int, vp]
        L.or_set_field.argtypes = [vp, C.c_int, vp]
        L.or_count.restype = i64
        L.or_count.argtypes = [vp, C.c_int]
        L.or_set_particles.argtypes = [vp, C.c_int, i64] + [vp] * 7
        L.or_get_particles.argtypes = [vp, C.c_int] + [vp] * 7
        L.or_surface_count.restype = i32
        L.or_surface_count.argtypes = [vp, C.c_int]
        L.or_set_surface_count.argtypes = [vp, C.c_int, i32]
        L.or_inject_target.restype = i32
        L.or_inject_target.argtypes = [vp, C.c_int]
        L.or_set_rr_scale.argtypes = [vp, d]
        L.or_step.argtypes = [vp, i32, i32]
        L.or_sort_now.argtypes = [vp]
        L.or_diagnostics.argtypes = [vp, C.POINTER(Diag), vp]
        L.or_node_charge.argtypes = [vp, vp]
        L.or_species_maps.argtypes = [vp, C.c_int, vp, vp]
        L.or_spectrum.argtypes = [vp, C.c_int, C.c_int, d, d, vp]
        L.or_push_local.argtypes = [d, d, d, pd, pd, pd, pd, pd]
        L.or_move_local.argtypes = [d, d, d, pd, pd, pd, pd, pd]
        L.or_blend.restype = d
        L.or_blend.argtypes = [vp, d]
        L.or_gather.argtypes = [vp, i32, i32, d, d, pd, pd]
        L.or_deposit.argtypes = [vp, d, i32, i32, d, d, d, d, d]
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32)]
        _lib = L
    return _lib


def _cfg_struct(cfg: dict) -> _Cfg:
    c = _Cfg()
    c.nr, c.nt = int(cfg["nr"]), int(cfg["nt"])
    c.r_min, c.r_max, c.r_lc = cfg["r_min"], cfg["r_max"], cfg["r_lc"]
    c.b_star = cfg.get("b_star", 1.0)
    c.geom = GEOM[cfg.get("geom", "dipole")]
    c.courant = cfg.get("courant", 0.5)
    c.r_abs = cfg.get("r_abs", 3.0 * cfg["r_lc"])
    c.absorb_strength = cfg.get("absorb_strength", 0.1)
    pb, fb = list(cfg.get("psi_break", [])), list(cfg.get("f_break", []))
    c.n_breaks = len(pb)
    for k in range(len(pb)):
        c.psi_break[k], c.f_break[k] = pb[k], fb[k]
    q, m = list(cfg.get("q", [-1.0, 1.0])), list(cfg.get("m", [1.0, 1.0]))
    c.n_species = len(q)
    for k in range(len(q)):
        c.q[k], c.m[k] = q[k], m[k]
    c.inject = 1 if cfg.get("inject", False) else 0
    c.kappa_inj = cfg.get("kappa_inj", 10.0)
    c.w_inj = cfg.get("w_inj", 1.0)
    c.gamma_rad = cfg.get("gamma_rad", 0.0)
    c.b_ref = cfg.get("b_ref", 1.0)
    c.rr_scale = cfg.get("rr_scale", 1.0)
    c.shell_r = cfg.get("shell_r", 2.0 * cfg["r_min"])
    c.synth_psi_open = cfg.get("synth_psi_open", 1.25)
    c.seed = int(cfg.get("seed", 1234))
    c.capacity = int(cfg.get("capacity", 0))
    c.tile_r, c.tile_t = int(cfg.get("tile_r", 16)), int(cfg.get("tile_t", 16))
    c.sort_every = int(cfg.get("sort_every", 0))
    c.gamma_th = float(cfg.get("gamma_th", 0.0))
    c.gamma_s = float(cfg.get("gamma_s", 0.0))
    isp = list(cfg.get("inject_species", [0, 1]))
    c.inject_species[0], c.inject_species[1] = int(isp[0]), int(isp[1])
    c.ff_delta_only = int(cfg.get("ff_delta_only", 0))
    c.ff_filter = float(cfg.get("ff_filter", 0.0))
    return c


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One FP64 CPU instance of the scheme."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = _cfg_struct(cfg)
        self.L = lib()
        self.h = self.L.or_create(C.byref(self._c))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.nr, self.nt = self._c.nr, self._c.nt
        self.n_species = self._c.n_species

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.or_destroy(h)
            self.h = None

    @property
    def dt(self) -> float:
        return self.L.or_dt(self.h)

    @property
    def psi_unit(self) -> float:
        return self.L.or_psi_unit(self.h)

    @property
    def step_index(self) -> int:
        return self.L.or_step_index(self.h)

    @step_index.setter
    def step_index(self, v: int) -> None:
        self.L.or_set_step_index(self.h, int(v))

    def shape(self, name: str):
        nr, nt = self.nr, self.nt
        k = FIELD_NAMES.index(name)
        return {0: (nr, nt + 1), 6: (nr, nt + 1), 1: (nr + 1, nt), 7: (nr + 1, nt),
                3: (nr + 1, nt), 16: (nr + 1, nt), 4: (nr, nt + 1), 17: (nr, nt + 1),
                5: (nr, nt), 18: (nr, nt)}.get(k, (nr + 1, nt + 1))

    def get(self, name: str) -> np.ndarray:
        out = np.empty(self.shape(name), dtype=np.float64)
        assert self.L.or_get_field(self.h, FIELD_NAMES.index(name), _ptr(out)) == 0
        return out

    def set(self, name: str, arr) -> None:
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape(name), (a.shape, self.shape(name))
        assert self.L.or_set_field(self.h, FIELD_NAMES.index(name), _ptr(a)) == 0

    def fields(self) -> dict:
        return {n: self.get(n) for n in FIELD_NAMES[:6]}

    def set_particles(self, species: int, p: dict) -> None:
        n = len(p["cell"])
        cell = np.ascontiguousarray(p["cell"], dtype=np.int32)
        arrs = [np.ascontiguousarray(p[k], dtype=np.float64) for k in ("xo", "yo", "ur", "ut", "up", "w")]
        rc = self.L.or_set_particles(self.h, species, n, _ptr(cell), *[_ptr(a) for a in arrs])
        if rc != 0:
            raise ValueError("oracle: particle load rejected")

    def count(self, species: int) -> int:
        return self.L.or_count(self.h, species)

    def particles(self, species: int) -> dict:
        n = self.count(species)
        out = {"cell": np.empty(n, np.int32)}
        for k in ("xo", "yo", "ur", "ut", "up", "w"):
            out[k] = np.empty(n, np.float64)
        self.L.or_get_particles(self.h, species, _ptr(out["cell"]),
                                *[_ptr(out[k]) for k in ("xo", "yo", "ur", "ut", "up", "w")])
        return out

    def step(self, n: int = 1, stages: int = 255) -> None:
        self.L.or_step(self.h, n, stages)

    def sort_now(self) -> None:
        self.L.or_sort_now(self.h)

    def set_rr_scale(self, v: float) -> None:
        self.L.or_set_rr_scale(self.h, v)

    def diagnostics(self):
        d = Diag()
        prof = np.empty(self.nr, np.float64)
        self.L.or_diagnostics(self.h, C.byref(d), _ptr(prof))
        return d, prof

    def node_charge(self) -> np.ndarray:
        q = np.empty((self.nr + 1, self.nt + 1), np.float64)
        self.L.or_node_charge(self.h, _ptr(q))
        return q

    def species_maps(self, species: int):
        """(number density, kinetic energy density) per cell, nr x nt."""
        d = np.empty((self.nr, self.nt), np.float64)
        e = np.empty((self.nr, self.nt), np.float64)
        self.L.or_species_maps(self.h, species, _ptr(d), _ptr(e))
        return d, e

    def spectrum(self, species: int, nbins: int, lg_min: float, lg_max: float) -> np.ndarray:
        out = np.empty(nbins, np.float64)
        self.L.or_spectrum(self.h, species, nbins, lg_min, lg_max, _ptr(out))
        return out

    def blend(self, psi: float) -> float:
        return self.L.or_blend(self.h, psi)

    def gather(self, i: int, j: int, xo: float, yo: float):
        """(E, B) in the local spherical basis at offset (xo, yo) of cell (i, j)."""
        e, b = (C.c_double * 3)(), (C.c_double * 3)()
        self.L.or_gather(self.h, i, j, xo, yo, e, b)
        return np.array(e[:]), np.array(b[:])

    def deposit(self, qw: float, i0: int, j0: int, x0: float, y0: float, x1: float, y1: float,
                vphi: float) -> None:
        """One charge-conserving deposit into J_r, J_th, J_ph (added)."""
        self.L.or_deposit(self.h, qw, i0, j0, x0, y0, x1, y1, vphi)

    def surface_counts(self) -> np.ndarray:
        return np.array([self.L.or_surface_count(self.h, j) for j in range(self.nt)], np.int32)

    def set_surface_counts(self, counts) -> None:
        """Surface counts as a push elsewhere left them (the injection's input)."""
        for j, v in enumerate(counts):
            self.L.or_set_surface_count(self.h, j, int(v))

    def inject_targets(self) -> np.ndarray:
        return np.array([self.L.or_inject_target(self.h, j) for j in range(self.nt)], np.int32)


def config_dt(cfg: dict) -> float:
    c = _cfg_struct(cfg)
    return lib().or_config_dt(C.byref(c))


def push_local(qm, krr, dt, u, e, b):
    L = lib()
    A = lambda v: (C.c_double * 3)(*[float(x) for x in v])
    out = (C.c_double * 3)()
    rad = C.c_double()
    L.or_push_local(qm, krr, dt, A(u), A(e), A(b), out, C.byref(rad))
    return np.array(out[:]), rad.value


def move_local(r, th, dt, u):
    L = lib()
    uu = (C.c_double * 3)(*[float(x) for x in u])
    dr, dth, dph = C.c_double(), C.c_double(), C.c_double()
    uo = (C.c_double * 3)()
    L.or_move_local(r, th, dt, uu, C.byref(dr), C.byref(dth), C.byref(dph), uo)
    return dr.value, dth.value, dph.value, np.array(uo[:])


def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.or_philox4x32_10(c, k, o)
    return list(o)
