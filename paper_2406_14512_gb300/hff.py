"""ctypes binding of ``libhff.so`` (C ABI in ``include/hff.h``).

Argument marshalling only: every step of the hybrid force-free / PIC update
runs in the CUDA kernels of the library.  PyTorch supplies the device memory
(one uint8 tensor per instance or ensemble, sized by ``hff_plan``) and the
CUDA stream.  The functions keep the C names; :class:`Sim` owns one instance,
:class:`Ensemble` several independent ones stepped by one graph launch per
step (``ens[k]`` is instance k).  Both give fields (``get``/``set``),
particles (``load``, ``particles``, ``particle_views``), FP64 diagnostics,
per-species density / energy maps and spectra, and checkpoints
(``checkpoint``/``restore``, ``save``/``resume``).  There is no CPU fallback:
if the library or a GPU is missing, the calls raise.

    sim = Sim(workloads.config("c3"))
    ps = workloads.particles(sim.cfg)
    sim.load(0, ps[0]); sim.load(1, ps[1])
    sim.step(100)
    diag, L_of_r = sim.diagnostics()
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhff.so")

HFF_OK, HFF_ERR_ARG, HFF_ERR_CAPACITY, HFF_ERR_CUDA, HFF_ERR_TIMEOUT, HFF_ERR_NONFINITE = 0, -1, -2, -3, -4, -5
GEOM = {"dipole": 0, "monopole": 1, "synth": 2, "uniform": 3, "michel": 4}
FP32, FP64 = 0, 1
# hff_config.field_pass: the field update chosen by grid size, as one fused
# pass, or split in four kernels
FIELDS_AUTO, FIELDS_FUSED, FIELDS_SPLIT = 0, 1, 2
FIELD_PASS_DEFAULT = FIELDS_AUTO
HOST, DEVICE = 0, 1
ST = dict(node=1, correct=2, push=4, faraday1=8, ampere=16, faraday2=32, inject=64, sort=128, all=255, nocount=256)
SCALAR_RR_SCALE = 0
INFO_RING = 8  # tickets that stay collectable (HFF_INFO_RING)
FIELDS = ["E_r", "E_th", "E_ph", "B_r", "B_th", "B_ph", "J_r", "J_th", "J_ph", "psi",
          "jperp_r", "jperp_th", "jperp_ph", "dE_r", "dE_th", "dE_ph",
          "f_r", "f_th", "f_node", "ff_cell"]


class HffError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hff error {code}: {msg}")
        self.code = code


class hff_config(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nt", C.c_int32),
        ("r_min", C.c_double), ("r_max", C.c_double), ("r_lc", C.c_double), ("b_star", C.c_double),
        ("geom", C.c_int32), ("courant", C.c_double), ("r_abs", C.c_double),
        ("absorb_strength", C.c_double), ("n_breaks", C.c_int32),
        ("psi_break", C.c_double * 4), ("f_break", C.c_double * 4),
        ("n_species", C.c_int32), ("q", C.c_double * 4), ("m", C.c_double * 4),
        ("inject", C.c_int32), ("kappa_inj", C.c_double), ("w_inj", C.c_double),
        ("gamma_rad", C.c_double), ("b_ref", C.c_double), ("rr_scale", C.c_double),
        ("shell_r", C.c_double), ("synth_psi_open", C.c_double), ("seed", C.c_uint64),
        ("capacity", C.c_int64), ("tile_r", C.c_int32), ("tile_t", C.c_int32),
        ("sort_every", C.c_int32), ("precision", C.c_int32),
        ("gamma_th", C.c_double), ("gamma_s", C.c_double), ("inject_species", C.c_int32 * 2),
        ("ff_delta_only", C.c_int32), ("ff_filter", C.c_double), ("field_pass", C.c_int32),
    ]


class hff_info(C.Structure):
    _fields_ = [("dt", C.c_double), ("psi_unit", C.c_double), ("step", C.c_int64),
                ("count", C.c_int64 * 4), ("tile_r", C.c_int32), ("tile_t", C.c_int32),
                ("sort_every", C.c_int32), ("precision", C.c_int32),
                ("kernels_per_step", C.c_int64), ("kernels_launched", C.c_int64),
                ("pushed_tiled", C.c_int64), ("pushed_tail", C.c_int64),
                ("readback_bytes", C.c_int64), ("n_inst", C.c_int64), ("field_pass", C.c_int32)]


class hff_particle_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("cell", C.c_void_p), ("xo", C.c_void_p), ("yo", C.c_void_p),
                ("ur", C.c_void_p), ("ut", C.c_void_p), ("up", C.c_void_p), ("w", C.c_void_p)]


class hff_diag(C.Structure):
    _fields_ = [("psi_open", C.c_double), ("eps", C.c_double), ("l_in", C.c_double),
                ("l_out", C.c_double), ("gauss_max", C.c_double), ("gauss_rms", C.c_double),
                ("rho_max", C.c_double), ("u_e", C.c_double), ("u_b", C.c_double),
                ("kinetic", C.c_double * 4), ("count", C.c_double * 4), ("injected", C.c_double),
                ("killed", C.c_double), ("radiated", C.c_double), ("nonfinite", C.c_double),
                ("created", C.c_double), ("clamps", C.c_double), ("nonfinite_fields", C.c_double)]


_lib = None

# exported symbols (checked against include/hff.h by the tests)
SYMBOLS = ["hff_plan", "hff_init", "hff_load_particles", "hff_set_field", "hff_fields", "hff_step",
           "hff_step_timed", "hff_step_stages", "hff_set_scalar", "hff_particles", "hff_diagnostics", "hff_get_info",
           "hff_info_enqueue", "hff_info_collect", "hff_status", "hff_destroy", "hff_last_error", "hff_tile_order_noalloc",
           "hff_noalloc_last_error", "hff_species_maps", "hff_spectrum", "hff_checkpoint_size",
           "hff_checkpoint_save", "hff_checkpoint_load"]
NOALLOC_MAX_PARTICLES = 262144


def load(path: str = LIB_PATH):
    """Load libhff.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HffError(HFF_ERR_ARG, f"{path} is missing: build the CUDA library first")
    L = C.CDLL(path)
    vp, i32, i64, sz, d = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_double
    sig = {
        "hff_plan": ([C.POINTER(hff_config), C.c_int, C.POINTER(sz)], C.c_int),
        "hff_init": ([C.POINTER(hff_config), C.c_int, vp, sz, vp, C.POINTER(vp)], C.c_int),
        "hff_load_particles": ([vp, C.c_int, C.c_int, i64] + [vp] * 7 + [C.c_int], C.c_int),
        "hff_set_field": ([vp, C.c_int, C.c_int, vp, sz, C.c_int], C.c_int),
        "hff_fields": ([vp, C.c_int, C.c_int, vp, sz, C.c_int], C.c_int),
        "hff_step": ([vp, i32], C.c_int),
        "hff_step_timed": ([vp, i32, vp, vp], C.c_int),
        "hff_step_stages": ([vp, i32, i32], C.c_int),
        "hff_set_scalar": ([vp, C.c_int, d], C.c_int),
        "hff_particles": ([vp, C.c_int, C.c_int, C.POINTER(hff_particle_view)], C.c_int),
        "hff_diagnostics": ([vp, C.c_int, C.POINTER(hff_diag), vp], C.c_int),
        "hff_get_info": ([vp, C.POINTER(hff_info)], C.c_int),
        "hff_info_enqueue": ([vp, C.POINTER(i64)], C.c_int),
        "hff_info_collect": ([vp, i64, C.POINTER(hff_info)], C.c_int),
        "hff_status": ([vp], C.c_int),
        "hff_destroy": ([vp], C.c_int),
        "hff_last_error": ([], C.c_char_p),
        "hff_tile_order_noalloc": ([vp, i64, i32, i32, i32, i32, vp, C.POINTER(i64), vp], C.c_int),
        "hff_noalloc_last_error": ([], C.c_char_p),
        "hff_species_maps": ([vp, C.c_int, C.c_int, vp, vp], C.c_int),
        "hff_spectrum": ([vp, C.c_int, C.c_int, C.c_int, d, d, vp], C.c_int),
        "hff_checkpoint_size": ([vp, C.c_int, C.POINTER(sz)], C.c_int),
        "hff_checkpoint_save": ([vp, C.c_int, vp, sz], C.c_int),
        "hff_checkpoint_load": ([vp, C.c_int, vp, sz], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes, f.restype = args, res
    _lib = L
    return L


def _check(rc: int):
    if rc != HFF_OK:
        raise HffError(rc, load().hff_last_error().decode())


def config_struct(cfg: dict) -> hff_config:
    """Workload dict (see workloads.config) -> hff_config."""
    c = hff_config()
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
    c.tile_r, c.tile_t = int(cfg.get("tile_r", 16)), int(cfg.get("tile_t", 32))
    c.sort_every = int(cfg.get("sort_every", 0))
    if c.tile_r == 0 and c.tile_t == 0 and c.sort_every == -1:
        # a shape left to the autotuner and not resolved (Sim resolves it):
        # the library gets the tuner's fallback shape
        from .autotune import DEFAULT_SHAPE
        c.tile_r, c.tile_t, c.sort_every = DEFAULT_SHAPE
    c.precision = FP64 if cfg.get("precision", "fp32") == "fp64" else FP32
    c.gamma_th = float(cfg.get("gamma_th", 0.0))
    c.gamma_s = float(cfg.get("gamma_s", 0.0))
    isp = list(cfg.get("inject_species", [0, 1]))
    c.inject_species[0], c.inject_species[1] = int(isp[0]), int(isp[1])
    c.ff_delta_only = int(cfg.get("ff_delta_only", 0))
    c.ff_filter = float(cfg.get("ff_filter", 0.0))
    c.field_pass = int(cfg.get("field_pass", FIELD_PASS_DEFAULT))
    return c


# ---------------------------------------------------------- C-named wrappers
def _configs(cfg):
    """One hff_config or a sequence of them -> (pointer, count)."""
    if isinstance(cfg, hff_config):
        return C.byref(cfg), 1
    arr = (hff_config * len(cfg))(*cfg)
    return arr, len(cfg)


def hff_plan(cfg, n_inst: int | None = None) -> int:
    """cfg: one hff_config, or a list of them for an ensemble."""
    ptr, n = _configs(cfg)
    b = C.c_size_t()
    _check(load().hff_plan(ptr, n if n_inst is None else n_inst, C.byref(b)))
    return b.value


def hff_init(cfg, dev_ptr: int, nbytes: int, stream: int, n_inst: int | None = None):
    ptr, n = _configs(cfg)
    h = C.c_void_p()
    _check(load().hff_init(ptr, n if n_inst is None else n_inst, C.c_void_p(dev_ptr), nbytes,
                           C.c_void_p(stream), C.byref(h)))
    return h


def hff_load_particles(h, inst, species, n, ptrs, where):
    _check(load().hff_load_particles(h, inst, species, n, *[C.c_void_p(p) for p in ptrs], where))


def hff_set_field(h, inst, which, src_ptr, nbytes, where):
    _check(load().hff_set_field(h, inst, which, C.c_void_p(src_ptr), nbytes, where))


def hff_fields(h, inst, which, dst_ptr, nbytes, where):
    _check(load().hff_fields(h, inst, which, C.c_void_p(dst_ptr), nbytes, where))


def hff_step(h, nsteps: int):
    _check(load().hff_step(h, nsteps))


def hff_step_timed(h, nsteps: int, ev_begin, ev_end):
    """ev_begin / ev_end: sequences of nsteps cudaEvent_t handles (ints)."""
    arr = C.c_void_p * max(1, nsteps)
    b = arr(*[C.c_void_p(e) for e in ev_begin])
    e = arr(*[C.c_void_p(x) for x in ev_end])
    _check(load().hff_step_timed(h, nsteps, C.cast(b, C.c_void_p), C.cast(e, C.c_void_p)))


def hff_step_stages(h, nsteps: int, stages: int):
    _check(load().hff_step_stages(h, nsteps, stages))


def hff_set_scalar(h, which: int, value: float):
    _check(load().hff_set_scalar(h, which, value))


def hff_particles(h, inst, species) -> hff_particle_view:
    v = hff_particle_view()
    _check(load().hff_particles(h, inst, species, C.byref(v)))
    return v


def hff_diagnostics(h, inst, nr: int):
    d = hff_diag()
    prof = np.empty(nr, np.float64)
    _check(load().hff_diagnostics(h, inst, C.byref(d), prof.ctypes.data_as(C.c_void_p)))
    return d, prof


def hff_get_info(h) -> hff_info:
    i = hff_info()
    _check(load().hff_get_info(h, C.byref(i)))
    return i


def hff_info_enqueue(h) -> int:
    t = C.c_int64()
    _check(load().hff_info_enqueue(h, C.byref(t)))
    return t.value


def hff_info_collect(h, ticket: int) -> hff_info:
    i = hff_info()
    _check(load().hff_info_collect(h, ticket, C.byref(i)))
    return i


def hff_status(h) -> int:
    return load().hff_status(h)


def hff_destroy(h):
    _check(load().hff_destroy(h))


def hff_last_error() -> str:
    return load().hff_last_error().decode()


def hff_species_maps(h, inst, species, nr, nt):
    d = np.empty((nr, nt), np.float64)
    e = np.empty((nr, nt), np.float64)
    _check(load().hff_species_maps(h, inst, species, d.ctypes.data_as(C.c_void_p), e.ctypes.data_as(C.c_void_p)))
    return d, e


def hff_spectrum(h, inst, species, nbins, lg_min, lg_max):
    out = np.empty(nbins, np.float64)
    _check(load().hff_spectrum(h, inst, species, nbins, lg_min, lg_max, out.ctypes.data_as(C.c_void_p)))
    return out


def hff_checkpoint_save(h, inst) -> np.ndarray:
    """The checkpoint blob of instance inst as a uint8 array."""
    n = C.c_size_t()
    _check(load().hff_checkpoint_size(h, inst, C.byref(n)))
    buf = np.empty(n.value, np.uint8)
    _check(load().hff_checkpoint_save(h, inst, buf.ctypes.data_as(C.c_void_p), n.value))
    return buf


def hff_checkpoint_load(h, inst, blob) -> None:
    b = np.ascontiguousarray(blob, np.uint8)
    _check(load().hff_checkpoint_load(h, inst, b.ctypes.data_as(C.c_void_p), b.nbytes))


def hff_tile_order_noalloc(cell_ptr: int, n: int, nr: int, nt: int, tile_r: int, tile_t: int,
                           order_ptr: int, stream: int) -> int:
    """Stable tile order of n device cell indices into order_ptr (device,
    n uint32) without allocating device memory; returns the live count.
    For callers that may not allocate: the scratch is a fixed device array
    inside the library (at most NOALLOC_MAX_PARTICLES particles per call)."""
    live = C.c_int64()
    rc = load().hff_tile_order_noalloc(C.c_void_p(cell_ptr), n, nr, nt, tile_r, tile_t,
                                       C.c_void_p(order_ptr), C.byref(live), C.c_void_p(stream))
    if rc != HFF_OK:
        raise HffError(rc, load().hff_noalloc_last_error().decode())
    return live.value


# ------------------------------------------------------------- convenience
class _InstanceOps:
    """Per-instance calls (fields, particles, diagnostics) of instance
    ``self.inst`` behind handle ``self.h`` in buffer ``self.mem``."""

    def _setup(self, c: hff_config):
        self.nr, self.nt = c.nr, c.nt
        self.real = np.float64 if c.precision == FP64 else np.float32
        self.tdtype = self.torch.float64 if c.precision == FP64 else self.torch.float32

    def shape(self, name: str):
        nr, nt = self.nr, self.nt
        return {"E_r": (nr, nt + 1), "J_r": (nr, nt + 1), "E_th": (nr + 1, nt), "J_th": (nr + 1, nt),
                "B_r": (nr + 1, nt), "B_th": (nr, nt + 1), "B_ph": (nr, nt), "f_r": (nr, nt + 1),
                "f_th": (nr + 1, nt), "ff_cell": (nr, nt)}.get(name, (nr + 1, nt + 1))

    def get(self, name: str) -> np.ndarray:
        """A field, J, Psi (FP64), a node array, or the blend weights f_r, f_th,
        f_node and the force-free cell flags ff_cell (uint8) of the current B."""
        dt = np.float64 if name == "psi" else (np.uint8 if name == "ff_cell" else self.real)
        out = np.empty(self.shape(name), dt)
        hff_fields(self.h, self.inst, FIELDS.index(name), out.ctypes.data, out.nbytes, HOST)
        return out

    def set(self, name: str, arr) -> None:
        a = np.ascontiguousarray(arr, dtype=self.real)
        assert a.shape == self.shape(name)
        hff_set_field(self.h, self.inst, FIELDS.index(name), a.ctypes.data, a.nbytes, HOST)

    def load(self, species: int, p: dict) -> None:
        n = len(p["cell"])
        arrs = [np.ascontiguousarray(p["cell"], np.int32)] + [
            np.ascontiguousarray(p[k], self.real) for k in ("xo", "yo", "ur", "ut", "up", "w")]
        hff_load_particles(self.h, self.inst, species, n, [a.ctypes.data for a in arrs], HOST)

    def load_device(self, species: int, t: dict) -> None:
        n = int(t["cell"].numel())
        hff_load_particles(self.h, self.inst, species, n,
                           [t[k].data_ptr() for k in ("cell", "xo", "yo", "ur", "ut", "up", "w")], DEVICE)

    def particle_views(self, species: int) -> dict:
        """Torch views (on the device, inside the instance buffer) of one
        species' particle arrays; valid until the next step."""
        torch = self.torch
        v = hff_particles(self.h, self.inst, species)
        n, base = int(v.n), self.mem.data_ptr()
        out = {}
        for k, dt, sz in [("cell", torch.int32, 4)] + [(k, self.tdtype, np.dtype(self.real).itemsize)
                                                         for k in ("xo", "yo", "ur", "ut", "up", "w")]:
            off = getattr(v, k) - base
            out[k] = self.mem[off:off + n * sz].view(dt)
        return out

    def particles(self, species: int) -> dict:
        """Host copies of one species' particle arrays (slots in use)."""
        return {k: t.cpu().numpy() for k, t in self.particle_views(species).items()}

    def diagnostics(self):
        return hff_diagnostics(self.h, self.inst, self.nr)

    def species_maps(self, species: int):
        """(number density, kinetic energy density) per cell, FP64, nr x nt."""
        return hff_species_maps(self.h, self.inst, species, self.nr, self.nt)

    def spectrum(self, species: int, nbins: int, lg_min: float, lg_max: float) -> np.ndarray:
        return hff_spectrum(self.h, self.inst, species, nbins, lg_min, lg_max)

    def checkpoint(self) -> np.ndarray:
        """Checkpoint blob (host bytes) of this instance."""
        return hff_checkpoint_save(self.h, self.inst)

    def restore(self, blob) -> None:
        hff_checkpoint_load(self.h, self.inst, blob)

    def save(self, path: str) -> None:
        self.checkpoint().tofile(path)

    def resume(self, path: str) -> None:
        self.restore(np.fromfile(path, np.uint8))


class _Stepping:
    """Whole-handle calls (an instance or a whole ensemble)."""

    def step(self, n: int = 1) -> None:
        hff_step(self.h, n)

    def step_timed(self, ev_begin, ev_end) -> None:
        """One step per event pair (torch.cuda.Event with timing); the events
        bracket the tiled push kernel of an instance, or the whole step of an
        ensemble.  Torch creates its CUDA events lazily, so any event not yet
        created is recorded once here first."""
        for e in list(ev_begin) + list(ev_end):
            if not e.cuda_event:
                e.record(self.stream)
        hff_step_timed(self.h, len(ev_begin), [e.cuda_event for e in ev_begin],
                       [e.cuda_event for e in ev_end])

    def step_stages(self, n: int, stages: int) -> None:
        hff_step_stages(self.h, n, stages)

    def set_rr_scale(self, v: float) -> None:
        hff_set_scalar(self.h, SCALAR_RR_SCALE, v)

    def info(self) -> hff_info:
        return hff_get_info(self.h)

    def info_enqueue(self) -> int:
        """Queue a read-back of the counters; returns a ticket for info_collect."""
        return hff_info_enqueue(self.h)

    def info_collect(self, ticket: int) -> hff_info:
        """The counters as they were when the ticket was queued."""
        return hff_info_collect(self.h, ticket)

    def status(self) -> int:
        return hff_status(self.h)

    def close(self):
        if getattr(self, "h", None):
            hff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_and_stream(device, stream):
    import torch
    if not torch.cuda.is_available():
        raise HffError(HFF_ERR_CUDA, "no CUDA device: the hybrid step runs only on the GPU")
    dev = torch.device(device)
    return torch, dev, (stream if stream is not None else torch.cuda.current_stream(dev))


class Sim(_InstanceOps, _Stepping):
    """One instance in a torch-owned device buffer on the current stream.

    A configuration with tile_r = tile_t = 0 and sort_every = -1 gets its
    launch shape from the autotuner (autotune.resolve): measured on
    `particles` (the species list the caller will load) and cached, or the
    cached / default shape when no particles are given."""

    def __init__(self, cfg: dict, device: str = "cuda:0", stream=None, particles=None):
        self.torch, self.dev, self.stream = _device_and_stream(device, stream)
        from . import autotune
        if autotune.wants_tuning(cfg):
            with self.torch.cuda.device(self.dev):
                cfg = autotune.resolve(cfg, particles)
        self.cfg = dict(cfg)
        self.c = config_struct(cfg)
        self.inst = 0
        self.nbytes = hff_plan(self.c)
        self.mem = self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.dev)
        self.h = hff_init(self.c, self.mem.data_ptr(), self.nbytes, self.stream.cuda_stream)
        self._setup(self.c)


class Member(_InstanceOps):
    """Instance `inst` of an :class:`Ensemble` (fields, particles, diagnostics)."""

    def __init__(self, ens: "Ensemble", inst: int):
        self.ens, self.inst, self.torch, self.mem = ens, inst, ens.torch, ens.mem
        self.cfg = ens.cfgs[inst]
        self._setup(ens.cs[inst])

    @property
    def h(self):
        return self.ens.h


class Ensemble(_Stepping):
    """Independent instances in one buffer, stepped together by one graph
    launch per step; ``ens[k]`` gives instance k."""

    def __init__(self, cfgs: list, device: str = "cuda:0", stream=None):
        self.torch, self.dev, self.stream = _device_and_stream(device, stream)
        self.cfgs = [dict(c) for c in cfgs]
        self.cs = [config_struct(c) for c in cfgs]
        self.nbytes = hff_plan(self.cs)
        self.mem = self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.dev)
        self.h = hff_init(self.cs, self.mem.data_ptr(), self.nbytes, self.stream.cuda_stream)
        self.members = [Member(self, k) for k in range(len(cfgs))]

    def __len__(self):
        return len(self.members)

    def __getitem__(self, k: int) -> Member:
        return self.members[k]
