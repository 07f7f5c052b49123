"""ctypes binding of libpic (include/pic.h): the same entry points, argument
marshalling only.  Every step of the PIC cycle runs in the CUDA library; there
is no CPU path here, and loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import workloads as W

MAX_SPECIES = 8
PIC_OK = 0
PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA, PIC_ERR_TIMEOUT, PIC_ERR_STATE, PIC_ERR_CAPACITY = -1, -2, -3, -4, -5, -6
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_OOM", -3: "PIC_ERR_CUDA", -4: "PIC_ERR_TIMEOUT", -5: "PIC_ERR_STATE",
          -6: "PIC_ERR_CAPACITY"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic.so")

EXPORTED = ["pic_init", "pic_destroy", "pic_load_particles", "pic_load_species", "pic_save_particles",
            "pic_restore_particles", "pic_set_step", "pic_clear_particles", "pic_step", "pic_sync",
            "pic_moments", "pic_fields", "pic_set_fields", "pic_particle_count", "pic_get_particles",
            "pic_diagnostics", "pic_set_timing", "pic_timings", "pic_sort_keys_noalloc", "pic_last_error",
            "pic_estimate_bytes", "pic_server_create", "pic_server_destroy", "pic_server_submit",
            "pic_server_status", "pic_server_result", "pic_server_release", "pic_server_cancel", "pic_server_wait_all", "pic_selftest_wait",
            "pic_probe_fp64_rate", "pic_ionize", "pic_collide",
            "pic_server_now", "pic_batch_create", "pic_batch_destroy", "pic_batch_step",
            "pic_prefetch_species", "pic_load_prefetched"]
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4
SUBMIT_KEEP_GRIDS = 1
NOALLOC_MAX_KEYS = 1048576


class PicConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
                ("bc_x", ctypes.c_int32), ("field_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("deposit", ctypes.c_int32), ("n_species", ctypes.c_int32),
                ("tile_nx", ctypes.c_int32), ("tile_ny", ctypes.c_int32),
                ("q", ctypes.c_double * MAX_SPECIES), ("m", ctypes.c_double * MAX_SPECIES),
                ("laser_a0", ctypes.c_double), ("laser_omega", ctypes.c_double),
                ("laser_tau", ctypes.c_double), ("laser_t0", ctypes.c_double),
                ("laser_pol", ctypes.c_int32), ("cn_max_iter", ctypes.c_int32),
                ("cn_tol", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("capacity", ctypes.c_int64 * MAX_SPECIES), ("shape", ctypes.c_int32), ("cn_precond", ctypes.c_int32)]


class PicServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_slots", ctypes.c_int32), ("steps_per_round", ctypes.c_int32),
                ("batch_min_runs", ctypes.c_int32)]


class PicSpeciesData(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("ux", ctypes.c_void_p),
                ("uy", ctypes.c_void_p), ("uz", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class PicRequestStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("steps_done", ctypes.c_int64),
                ("steps_total", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_finish", ctypes.c_double), ("particle_steps", ctypes.c_double), ("device_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PicIonization(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int32), ("ion", ctypes.c_int32 * MAX_SPECIES),
                ("target", ctypes.c_int32 * MAX_SPECIES), ("electron", ctypes.c_int32 * MAX_SPECIES),
                ("ip_ev", ctypes.c_double * MAX_SPECIES), ("field_unit_au", ctypes.c_double),
                ("time_unit_au", ctypes.c_double), ("seed", ctypes.c_uint64)]


MAX_COLLISION_PAIRS = 16


class PicCollisions(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int32), ("a", ctypes.c_int32 * MAX_COLLISION_PAIRS),
                ("b", ctypes.c_int32 * MAX_COLLISION_PAIRS), ("ln_lambda", ctypes.c_double),
                ("kappa", ctypes.c_double), ("seed", ctypes.c_uint64)]


class PicDiag(ctypes.Structure):
    _fields_ = [("kinetic", ctypes.c_double), ("field", ctypes.c_double), ("total", ctypes.c_double),
                ("charge_grid", ctypes.c_double), ("charge_particles", ctypes.c_double),
                ("count", ctypes.c_int64), ("removed", ctypes.c_int64), ("step", ctypes.c_int64),
                ("cn_residual", ctypes.c_double), ("cn_iterations", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("cn_refinements", ctypes.c_int32), ("full_regroups", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PicError(RuntimeError):
    pass


_lib = None


def lib(path: Optional[str] = None):
    """Load libpic.so (built by paper_1308_2590_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise PicError(f"libpic.so not built ({p}); run `python -m paper_1308_2590_gb300.build`")
    L = ctypes.CDLL(p)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    L.pic_init.argtypes = [ctypes.POINTER(PicConfig), ctypes.POINTER(vp)]
    L.pic_destroy.argtypes = [vp]
    L.pic_load_particles.argtypes = [vp, i32, i64, dp, dp, dp, dp, dp, dp]
    L.pic_load_species.argtypes = [vp, i32, ctypes.POINTER(PicSpeciesData)]
    L.pic_prefetch_species.argtypes = [vp, i32, ctypes.POINTER(PicSpeciesData)]
    L.pic_load_prefetched.argtypes = [vp]
    L.pic_ionize.argtypes = [vp, ctypes.POINTER(PicIonization), ctypes.POINTER(ctypes.c_int64)]
    L.pic_collide.argtypes = [vp, ctypes.POINTER(PicCollisions), ctypes.POINTER(ctypes.c_int64)]
    L.pic_save_particles.argtypes = [vp, i32, vp, dp, dp, dp, dp, dp, dp]
    L.pic_restore_particles.argtypes = [vp, i32, i64, vp, dp, dp, dp, dp, dp, dp]
    L.pic_set_step.argtypes = [vp, i64]
    L.pic_clear_particles.argtypes = [vp]
    L.pic_step.argtypes = [vp, i32]
    L.pic_sync.argtypes = [vp]
    L.pic_moments.argtypes = [vp, dp, dp, dp]
    L.pic_fields.argtypes = [vp, dp, dp]
    L.pic_set_fields.argtypes = [vp, dp, dp]
    L.pic_particle_count.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64)]
    L.pic_get_particles.argtypes = [vp, i32, dp, dp, dp, dp, dp, dp, dp]
    L.pic_diagnostics.argtypes = [vp, ctypes.POINTER(PicDiag)]
    L.pic_set_timing.argtypes = [vp, i32]
    L.pic_timings.argtypes = [vp, dp, dp, i32]
    L.pic_sort_keys_noalloc.argtypes = [dp, i64, ctypes.c_uint32, dp, vp]
    L.pic_estimate_bytes.argtypes = [ctypes.POINTER(PicConfig), dp, ctypes.POINTER(ctypes.c_uint64)]
    L.pic_server_create.argtypes = [ctypes.POINTER(PicServerConfig), ctypes.POINTER(vp)]
    L.pic_server_destroy.argtypes = [vp]
    L.pic_server_submit.argtypes = [vp, ctypes.POINTER(PicConfig), i32, ctypes.POINTER(PicSpeciesData), i32,
                                    ctypes.POINTER(ctypes.c_int64)]
    L.pic_server_status.argtypes = [vp, i64, ctypes.POINTER(PicRequestStatus)]
    L.pic_server_result.argtypes = [vp, i64, ctypes.POINTER(PicDiag), dp, dp, dp, dp, dp]
    L.pic_server_release.argtypes = [vp, i64]
    L.pic_server_cancel.argtypes = [vp, i64]
    L.pic_selftest_wait.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.pic_probe_fp64_rate.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.pic_server_wait_all.argtypes = [vp, ctypes.c_double]
    L.pic_server_now.argtypes = [vp]
    L.pic_batch_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
    L.pic_batch_destroy.argtypes = [vp]
    L.pic_batch_step.argtypes = [vp, ctypes.POINTER(vp), i32, i32]
    L.pic_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("pic_last_error", "pic_server_now"):
            getattr(L, name).restype = ctypes.c_int
    L.pic_server_now.restype = ctypes.c_double
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != PIC_OK:
        msg = lib().pic_last_error().decode(errors="replace")
        raise PicError(f"{what} -> {ERRORS.get(rc, rc)}: {msg}")


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def pic_sort_keys_noalloc(keys_dev_ptr: int, n: int, max_key: int, perm_dev_ptr: int,
                          stream: Optional[int] = None) -> None:
    """Allocation-free stable sort of n uint32 keys (device pointers) into a permutation."""
    _check(lib().pic_sort_keys_noalloc(keys_dev_ptr, int(n), int(max_key), perm_dev_ptr, stream),
           "pic_sort_keys_noalloc")


def make_config(cfg: W.RunConfig, stream: Optional[int] = None, capacity: Optional[list] = None) -> PicConfig:
    c = PicConfig()
    c.nx, c.ny = cfg.nx, cfg.ny
    c.dx, c.dy, c.dt = cfg.dx, cfg.dy, cfg.dt
    c.bc_x, c.field_mode, c.precision, c.deposit = cfg.bc_x, cfg.field_mode, cfg.precision, cfg.deposit
    c.n_species = len(cfg.species)
    c.tile_nx, c.tile_ny = cfg.tile_nx, cfg.tile_ny
    for k, s in enumerate(cfg.species):
        c.q[k], c.m[k] = s.q, s.m
    c.laser_a0, c.laser_omega, c.laser_tau, c.laser_t0 = cfg.laser.a0, cfg.laser.omega, cfg.laser.tau, cfg.laser.t0
    c.laser_pol = cfg.laser.pol
    c.cn_max_iter = cfg.cn_max_iter
    c.shape = int(getattr(cfg, "shape", 1))
    c.cn_precond = int(getattr(cfg, "cn_precond", 0))
    c.cn_tol = cfg.cn_tol
    c.cuda_stream = stream
    if capacity:
        for k, n in enumerate(capacity):
            c.capacity[k] = int(n)
    return c


class Pic:
    """One PIC run on the GPU behind the C ABI."""

    def __init__(self, cfg: W.RunConfig, stream: Optional[int] = None, capacity: Optional[list] = None):
        self.cfg = cfg
        self.nsp = len(cfg.species)
        self.nxn = cfg.nx if cfg.bc_x == W.BC_PERIODIC else cfg.nx + 1
        self._c = make_config(cfg, stream, capacity)
        h = ctypes.c_void_p()
        _check(lib().pic_init(ctypes.byref(self._c), ctypes.byref(h)), "pic_init")
        self.h = h

    def close(self):
        if self.h:
            lib().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def pic_load_particles(self, s: int, x, y, ux, uy, uz, w):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, ux, uy, uz, w)]
        _check(lib().pic_load_particles(self.h, s, arrs[0].size, *[_ptr(a) for a in arrs]), "pic_load_particles")

    def load(self, s: int, P: dict):
        self.pic_load_particles(s, P["x"], P["y"], P["ux"], P["uy"], P["uz"], P["w"])

    def pic_load_species(self, parts):
        """parts[s] (dict of x, y, ux, uy, uz, w) into species s, all or nothing."""
        arrays = []
        sd = (PicSpeciesData * max(1, len(parts)))()
        for s, P in enumerate(parts):
            a = [np.ascontiguousarray(P[k], dtype=np.float64) for k in ("x", "y", "ux", "uy", "uz", "w")]
            arrays.append(a)
            sd[s].n = a[0].size
            sd[s].x, sd[s].y, sd[s].ux, sd[s].uy, sd[s].uz, sd[s].w = [_ptr(v) for v in a]
        _check(lib().pic_load_species(self.h, len(parts), sd), "pic_load_species")

    def pic_prefetch_species(self, parts):
        """Start copying parts[s] (dict of x, y, ux, uy, uz, w; FP64 C-contiguous arrays, page-locked for
        an asynchronous copy) to the device for a later pic_load_prefetched; the arrays are kept
        referenced (and must stay unchanged) until that load."""
        arrays = []
        sd = (PicSpeciesData * max(1, len(parts)))()
        for s, P in enumerate(parts):
            a = [P[k] for k in ("x", "y", "ux", "uy", "uz", "w")]
            for v in a:
                if v.dtype != np.float64 or not v.flags["C_CONTIGUOUS"] or v.size != a[0].size:
                    raise ValueError("prefetched arrays must be C-contiguous float64 arrays of one length")
            arrays.append(a)
            sd[s].n = a[0].size
            sd[s].x, sd[s].y, sd[s].ux, sd[s].uy, sd[s].uz, sd[s].w = [_ptr(v) for v in a]
        _check(lib().pic_prefetch_species(self.h, len(parts), sd), "pic_prefetch_species")
        self._prefetched = getattr(self, "_prefetched", []) + [arrays]

    def pic_load_prefetched(self):
        try:
            _check(lib().pic_load_prefetched(self.h), "pic_load_prefetched")
        finally:
            if getattr(self, "_prefetched", None):
                self._prefetched.pop(0)

    def pic_clear_particles(self):
        _check(lib().pic_clear_particles(self.h), "pic_clear_particles")

    def pic_step(self, n: int = 1):
        _check(lib().pic_step(self.h, int(n)), "pic_step")

    def pic_sync(self):
        _check(lib().pic_sync(self.h), "pic_sync")

    def pic_moments(self, out: Optional[np.ndarray] = None):
        """The 13 area-normalised moment planes [rho, S (9), dj (3)] as one (13, ny, nxn) FP64 array,
        written in place into `out` when given (e.g. page-locked memory)."""
        ny, nxn = self.cfg.ny, self.nxn
        M = np.empty((13, ny, nxn)) if out is None else out
        if M.shape != (13, ny, nxn) or M.dtype != np.float64 or not M.flags["C_CONTIGUOUS"]:
            raise ValueError(f"moments buffer must be a C-contiguous float64 array of shape {(13, ny, nxn)}")
        base, plane = M.ctypes.data, ny * nxn * 8
        _check(lib().pic_moments(self.h, ctypes.c_void_p(base), ctypes.c_void_p(base + plane),
                                 ctypes.c_void_p(base + 10 * plane)), "pic_moments")
        return M

    def pic_fields(self):
        ny, nx, nxn = self.cfg.ny, self.cfg.nx, self.nxn
        E = np.empty((3, ny, nxn)); H = np.empty((3, ny, nx))
        _check(lib().pic_fields(self.h, _ptr(E), _ptr(H)), "pic_fields")
        return E, H

    def pic_set_fields(self, E=None, H=None):
        E = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
        H = None if H is None else np.ascontiguousarray(H, dtype=np.float64)
        _check(lib().pic_set_fields(self.h, _ptr(E), _ptr(H)), "pic_set_fields")

    def pic_particle_count(self, s: int) -> int:
        n = ctypes.c_int64()
        _check(lib().pic_particle_count(self.h, s, ctypes.byref(n)), "pic_particle_count")
        return n.value

    def pic_save_particles(self, s: int) -> dict:
        """Checkpoint form: cell, ox, oy, ux, uy, uz, w exactly as stored."""
        n = self.pic_particle_count(s)
        out = {k: np.empty(n) for k in ("ox", "oy", "ux", "uy", "uz", "w")}
        out["cell"] = np.empty(n, np.int32)
        _check(lib().pic_save_particles(self.h, s, out["cell"].ctypes.data_as(ctypes.c_void_p),
                                        *[_ptr(out[k]) for k in ("ox", "oy", "ux", "uy", "uz", "w")]),
               "pic_save_particles")
        return out

    def pic_restore_particles(self, s: int, P: dict):
        cell = np.ascontiguousarray(P["cell"], dtype=np.int32)
        arrs = [np.ascontiguousarray(P[k], dtype=np.float64) for k in ("ox", "oy", "ux", "uy", "uz", "w")]
        _check(lib().pic_restore_particles(self.h, s, cell.size, cell.ctypes.data_as(ctypes.c_void_p),
                                           *[_ptr(a) for a in arrs]), "pic_restore_particles")

    def pic_ionize(self, chains, seed: int, field_unit_au: float, time_unit_au: float) -> int:
        """One field-ionisation pass; chains = [(ion, target, electron, ip_ev), ...]; returns the transitions."""
        p = PicIonization()
        p.n_chains = len(chains)
        for c, (a, t, e, ip) in enumerate(chains):
            p.ion[c], p.target[c], p.electron[c], p.ip_ev[c] = int(a), int(t), int(e), float(ip)
        p.field_unit_au, p.time_unit_au, p.seed = float(field_unit_au), float(time_unit_au), int(seed)
        n = ctypes.c_int64()
        _check(lib().pic_ionize(self.h, ctypes.byref(p), ctypes.byref(n)), "pic_ionize")
        return n.value

    def pic_collide(self, pairs, seed: int, ln_lambda: float, kappa: float) -> int:
        """One binary-collision pass; pairs = [(species_a, species_b), ...]; returns the pairs processed."""
        p = PicCollisions()
        p.n_pairs = len(pairs)
        for k, (a, b) in enumerate(pairs):
            p.a[k], p.b[k] = int(a), int(b)
        p.ln_lambda, p.kappa, p.seed = float(ln_lambda), float(kappa), int(seed)
        n = ctypes.c_int64()
        _check(lib().pic_collide(self.h, ctypes.byref(p), ctypes.byref(n)), "pic_collide")
        return n.value

    def pic_set_step(self, step: int):
        _check(lib().pic_set_step(self.h, int(step)), "pic_set_step")

    def pic_get_particles(self, s: int) -> dict:
        n = self.pic_particle_count(s)
        out = {k: np.empty(n) for k in ("x", "y", "ux", "uy", "uz", "w")}
        cell = np.empty(n, np.int32)
        _check(lib().pic_get_particles(self.h, s, *[_ptr(out[k]) for k in ("x", "y", "ux", "uy", "uz", "w")],
                                       _ptr(cell)), "pic_get_particles")
        out["cell"] = cell
        return out

    def pic_diagnostics(self) -> dict:
        d = PicDiag()
        _check(lib().pic_diagnostics(self.h, ctypes.byref(d)), "pic_diagnostics")
        return d.as_dict()

    def pic_set_timing(self, on: bool):
        _check(lib().pic_set_timing(self.h, int(bool(on))), "pic_set_timing")

    def pic_timings(self, reset: bool = False):
        ms = np.zeros(4); la = np.zeros(5, np.int64)
        _check(lib().pic_timings(self.h, _ptr(ms), _ptr(la), int(bool(reset))), "pic_timings")
        return ms, la


def estimate_bytes(cfg: W.RunConfig, n_per_species) -> int:
    """Device bytes a run of this configuration holds with these particle counts."""
    c = make_config(cfg)
    n = (ctypes.c_int64 * MAX_SPECIES)(*[int(v) for v in n_per_species])
    out = ctypes.c_uint64()
    _check(lib().pic_estimate_bytes(ctypes.byref(c), ctypes.cast(n, ctypes.c_void_p), ctypes.byref(out)),
           "pic_estimate_bytes")
    return out.value


def selftest_wait(stream=None):
    """Run the bounded-wait self-test; returns (status code, seconds)."""
    sec = ctypes.c_double()
    rc = lib().pic_selftest_wait(stream, ctypes.byref(sec))
    return rc, sec.value


def probe_fp64_rate(stream=None, repeats: int = 5) -> float:
    """Measured FP64 FMA rate of this GPU in TFLOP/s (best of `repeats` timed launches)."""
    tf = ctypes.c_double()
    _check(lib().pic_probe_fp64_rate(stream, int(repeats), ctypes.byref(tf)), "pic_probe_fp64_rate")
    return tf.value


class Server:
    """Continuous-batching server over the C ABI (the GPU loop runs in the library's worker thread)."""

    def __init__(self, mem_budget: int = 0, max_slots: int = 0, steps_per_round: int = 0, batch_min_runs: int = 0):
        c = PicServerConfig(int(mem_budget), int(max_slots), int(steps_per_round), int(batch_min_runs))
        h = ctypes.c_void_p()
        _check(lib().pic_server_create(ctypes.byref(c), ctypes.byref(h)), "pic_server_create")
        self.h = h
        self._cfgs = {}

    def close(self):
        if self.h:
            lib().pic_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, cfg: W.RunConfig, parts, nsteps: int, keep_grids: bool = False) -> int:
        c = make_config(cfg)
        arrays = []
        sd = (PicSpeciesData * len(cfg.species))()
        for s, P in enumerate(parts):
            a = [np.ascontiguousarray(P[k], dtype=np.float64) for k in ("x", "y", "ux", "uy", "uz", "w")]
            arrays.append(a)
            sd[s].n = a[0].size
            sd[s].x, sd[s].y, sd[s].ux, sd[s].uy, sd[s].uz, sd[s].w = [_ptr(v) for v in a]
        rid = ctypes.c_int64()
        _check(lib().pic_server_submit(self.h, ctypes.byref(c), int(nsteps), sd,
                                       SUBMIT_KEEP_GRIDS if keep_grids else 0, ctypes.byref(rid)), "pic_server_submit")
        self._cfgs[rid.value] = cfg
        return rid.value

    def status(self, rid: int) -> dict:
        st = PicRequestStatus()
        _check(lib().pic_server_status(self.h, int(rid), ctypes.byref(st)), "pic_server_status")
        return st.as_dict()

    def result(self, rid: int, grids: bool = False):
        d = PicDiag()
        if not grids:
            _check(lib().pic_server_result(self.h, int(rid), ctypes.byref(d), None, None, None, None, None),
                   "pic_server_result")
            return d.as_dict(), None
        cfg = self._cfgs[rid]
        nxn = cfg.nx if cfg.bc_x == W.BC_PERIODIC else cfg.nx + 1
        n = cfg.ny * nxn
        rho = np.empty(n); S9 = np.empty(9 * n); dj3 = np.empty(3 * n)
        E = np.empty((3, cfg.ny, nxn)); H = np.empty((3, cfg.ny, cfg.nx))
        _check(lib().pic_server_result(self.h, int(rid), ctypes.byref(d), _ptr(rho), _ptr(S9), _ptr(dj3), _ptr(E),
                                       _ptr(H)), "pic_server_result")
        M = np.empty((13, cfg.ny, nxn))
        M[0] = rho.reshape(cfg.ny, nxn); M[1:10] = S9.reshape(9, cfg.ny, nxn); M[10:13] = dj3.reshape(3, cfg.ny, nxn)
        return d.as_dict(), (M, E, H)

    def release(self, rid: int):
        _check(lib().pic_server_release(self.h, int(rid)), "pic_server_release")
        self._cfgs.pop(rid, None)

    def cancel(self, rid: int):
        _check(lib().pic_server_cancel(self.h, int(rid)), "pic_server_cancel")

    def wait_all(self, timeout_s: float = 600.0):
        _check(lib().pic_server_wait_all(self.h, float(timeout_s)), "pic_server_wait_all")

    def now(self) -> float:
        return lib().pic_server_now(self.h)


class Batch:
    """Batched stepping of several Pic runs: one push and one regroup launch per step for all of them."""

    def __init__(self, max_runs: int, stream: Optional[int] = None):
        h = ctypes.c_void_p()
        _check(lib().pic_batch_create(int(max_runs), stream, ctypes.byref(h)), "pic_batch_create")
        self.h = h

    def close(self):
        if self.h:
            lib().pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, runs, nsteps: int = 1):
        arr = (ctypes.c_void_p * len(runs))(*[r.h for r in runs])
        _check(lib().pic_batch_step(self.h, arr, len(runs), int(nsteps)), "pic_batch_step")
