"""ctypes binding of libp3maze.so (include/p3maze.h).

Argument marshalling only: every step of the electrostatics path runs in the
CUDA library.  Importing this module fails loudly if the library has not been
built (python -m paper_2606_31379_b300.build).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libp3maze.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_2606_31379_b300.build`")
lib = C.CDLL(_LIB_PATH)

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_NONFINITE = 0, -1, -2, -3, -4, -5
FP64, MIXED = 0, 1
METHOD_MAZE, METHOD_P3M, METHOD_PMAZE = 0, 1, 2
SR_NONE, SR_BMH, SR_LJ = 0, 1, 2
SR_TRUNCATE, SR_SHIFT_FORCE = 0, 1
MAX_TYPES = 4
MESH = {"q": 0, "qs": 1, "phi": 2, "y": 3, "sigma": 4}
FORCE = {"total": 0, "sr": 1, "lr": 2, "bond": 3}


class SRTable(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_types", C.c_int32),
                ("p", (C.c_double * (MAX_TYPES * MAX_TYPES)) * 5)]


class Topology(C.Structure):
    _fields_ = [("n_molecules", C.c_int32), ("triples", C.POINTER(C.c_int32)),
                ("kb", C.c_double), ("r0", C.c_double), ("ka", C.c_double), ("theta0", C.c_double)]


class Params(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("n_particles", C.c_int32),
                ("charges", C.POINTER(C.c_double)), ("masses", C.POINTER(C.c_double)),
                ("types", C.POINTER(C.c_int32)), ("alpha", C.c_double), ("r_cut", C.c_double),
                ("mesh", C.c_int32), ("order", C.c_int32), ("tol", C.c_double), ("dt", C.c_double),
                ("predictor", C.c_int32), ("precision", C.c_int32), ("max_mg_iters", C.c_int32),
                ("pre_sweeps", C.c_int32), ("post_sweeps", C.c_int32), ("coulomb_k", C.c_double),
                ("sr", C.POINTER(SRTable)), ("topology", C.POINTER(Topology)), ("method", C.c_int32),
                ("coarse_max", C.c_int32), ("lr_force", C.c_int32), ("sr_shift", C.c_int32)]


class Energies(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("v_sr", "v_lr", "v_self", "v_excl", "v_vdw", "v_bond", "kinetic", "total", "w_sr")]


class Stats(C.Structure):
    _fields_ = [("last_iters", C.c_int32), ("last_residual", C.c_double), ("steps", C.c_int64),
                ("total_iters", C.c_int64), ("init_iters", C.c_int32), ("smooth_steps", C.c_int32),
                ("smooth_coeff", C.c_double), ("mg_levels", C.c_int32), ("coarse_n", C.c_int32),
                ("cells_per_axis", C.c_int32), ("sigma", C.c_double), ("device_bytes", C.c_int64)]


NSTAGES = 9
STAGES = ("integrate", "cells", "spread", "smooth", "predict", "solve", "update", "pair", "gather")


class Timing(C.Structure):
    _fields_ = [("ms", C.c_double * NSTAGES), ("launches", C.c_int64 * NSTAGES),
                ("timed_steps", C.c_int64), ("total_launches", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("predictor", C.c_int32), ("pre_sweeps", C.c_int32), ("post_sweeps", C.c_int32),
                ("diffusion_zc", C.c_int32), ("diffusion_fuse", C.c_int32),
                ("pair_fork", C.c_int32), ("coarse_max", C.c_int32),
                ("pair_blocks", C.c_int32), ("cluster_ctas", C.c_int32), ("sweep_fuse", C.c_int32),
                ("ms_per_step", C.c_double), ("initial_ms_per_step", C.c_double),
                ("trials", C.c_int32), ("steps", C.c_int32)]


TUNING_TIMING = ("ms_per_step", "initial_ms_per_step", "trials", "steps")


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_ctx = C.c_void_p
_sig = {
    "p3maze_init": (C.c_int, [C.POINTER(Params), _dp, _dp, C.c_void_p, C.POINTER(_ctx)]),
    "p3maze_step": (C.c_int, [_ctx, C.c_int32]),
    "p3maze_step_async": (C.c_int, [_ctx, C.c_int32]),
    "p3maze_wait": (C.c_int, [_ctx]),
    "p3maze_set_rollback": (C.c_int, [_ctx, C.c_int32]),
    "p3maze_set_solver": (C.c_int, [_ctx, C.c_double, C.c_int32]),
    "p3maze_step_host": (C.c_int, [_ctx, _dp, _dp, C.c_int32, _dp, _dp]),
    "p3maze_set_tuning": (C.c_int, [_ctx, C.c_void_p]),
    "p3maze_init_device": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_ctx)]),
    "p3maze_state_bytes": (C.c_int, [_ctx, C.POINTER(C.c_size_t)]),
    "p3maze_save_state": (C.c_int, [_ctx, C.c_void_p, C.c_size_t]),
    "p3maze_load_state": (C.c_int, [_ctx, C.c_void_p, C.c_size_t]),
    "p3maze_get_tuning": (C.c_int, [_ctx, C.c_void_p]),
    "p3maze_reinit": (C.c_int, [_ctx]),
    "p3maze_equilibrate": (C.c_int, [_ctx, C.c_int32, C.c_double]),
    "p3maze_destroy": (None, [_ctx]),
    "p3maze_device_bytes": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_size_t)]),
    "p3maze_energy": (C.c_int, [_ctx, C.POINTER(Energies)]),
    "p3maze_get_stats": (C.c_int, [_ctx, C.POINTER(Stats)]),
    "p3maze_get_positions": (C.c_int, [_ctx, _dp]),
    "p3maze_get_velocities": (C.c_int, [_ctx, _dp]),
    "p3maze_get_forces": (C.c_int, [_ctx, C.c_int32, _dp]),
    "p3maze_set_state": (C.c_int, [_ctx, _dp, _dp]),
    "p3maze_get_mesh": (C.c_int, [_ctx, C.c_int32, _dp]),
    "p3maze_get_cells": (C.c_int, [_ctx, _ip, _ip, _ip]),
    "p3maze_set_timing": (C.c_int, [_ctx, C.c_int32]),
    "p3maze_get_timing": (C.c_int, [_ctx, C.POINTER(Timing)]),
    "p3maze_set_graphs": (C.c_int, [_ctx, C.c_int32]),
    "p3maze_autotune": (C.c_int, [_ctx, C.c_int32, C.POINTER(Tuning)]),
    "p3maze_smooth_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p]),
    "p3maze_last_error": (C.c_char_p, [_ctx]),
    "p3maze_batch_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "p3maze_batch_add": (C.c_int, [C.c_void_p, _ctx]),
    "p3maze_batch_remove": (C.c_int, [C.c_void_p, _ctx]),
    "p3maze_batch_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "p3maze_batch_wait": (C.c_int, [C.c_void_p]),
    "p3maze_batch_size": (C.c_int, [C.c_void_p]),
    "p3maze_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int32]),
    "p3maze_batch_set_fused_smoothing": (C.c_int, [C.c_void_p, C.c_int32]),
    "p3maze_batch_destroy": (None, [C.c_void_p]),
    "p3maze_batch_last_error": (C.c_char_p, [C.c_void_p]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class P3MaZeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"p3maze error {code}: {msg}")
        self.code = code


def smooth_noalloc(q_ptr: int, qs_ptr: int, mesh: int, steps: int, coeff: float, stream: int | None = None):
    """p3maze_smooth_noalloc on device pointers (no device allocation)."""
    rc = lib.p3maze_smooth_noalloc(C.c_void_p(q_ptr), C.c_void_p(qs_ptr), int(mesh), int(steps), float(coeff),
                                   C.c_void_p(stream or 0))
    if rc:
        raise P3MaZeError(rc, lib.p3maze_last_error(None).decode())


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


def sr_table_from(kind: str, table: dict) -> SRTable | None:
    """SRTable from a {'A','rho','sigma','C','D'} (BMH) or {'eps','sigma'} (LJ)
    dict of [n_types][n_types] arrays."""
    if kind in (None, "none") or not table:
        return None
    t = SRTable()
    keys = ("A", "rho", "sigma", "C", "D") if kind == "bmh" else ("eps", "sigma")
    nt = np.asarray(table[keys[0]]).shape[0]
    t.kind = SR_BMH if kind == "bmh" else SR_LJ
    t.n_types = nt
    for a, k in enumerate(keys):
        m = np.asarray(table[k], dtype=np.float64)
        for i in range(nt):
            for j in range(nt):
                t.p[a][i * nt + j] = float(m[i, j])
    return t


def build_params(pos, charges, masses, box: float, *, alpha: float, r_cut: float, mesh: int,
                 tol: float, dt: float, vel=None, types=None, sr_kind: str = "none",
                 sr_table: dict | None = None, triples=None, bonded: dict | None = None,
                 order: int = 4, predictor: int = 3, precision: str = "fp64",
                 max_mg_iters: int = 0, pre_sweeps: int = 0, post_sweeps: int = 0,
                 coulomb_k: float = 0.0, method: str = "maze", coarse_max: int = 0, lr_force: str = "fd",
                 sr_shift: str = "none"):
    """p3maze_params for these arguments, plus the arrays it points into
    (keep them alive while the struct is used)."""
    n = int(np.asarray(charges).shape[0])
    pos = _f64(pos, (n, 3))
    vel = None if vel is None else _f64(vel, (n, 3))
    q = _f64(charges)
    m = _f64(masses)
    p = Params()
    p.box[0] = p.box[1] = p.box[2] = float(box)
    p.n_particles = n
    p.charges = _ptr(q)
    p.masses = _ptr(m)
    keep = {"pos": pos, "vel": vel, "q": q, "m": m}
    if types is not None:
        t = np.ascontiguousarray(types, dtype=np.int32)
        keep["types"] = t
        p.types = _ptr(t, C.c_int32)
    p.alpha, p.r_cut, p.mesh, p.order = float(alpha), float(r_cut), int(mesh), int(order)
    p.tol, p.dt, p.predictor = float(tol), float(dt), int(predictor)
    p.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    p.max_mg_iters, p.pre_sweeps, p.post_sweeps = int(max_mg_iters), int(pre_sweeps), int(post_sweeps)
    p.coulomb_k = float(coulomb_k)
    p.method = {"maze": METHOD_MAZE, "p3m": METHOD_P3M, "pmaze": METHOD_PMAZE}[method]
    p.coarse_max = int(coarse_max)
    p.lr_force = {"fd": 0, "analytic": 1}[lr_force]
    p.sr_shift = {"none": SR_TRUNCATE, "force": SR_SHIFT_FORCE}[sr_shift]
    tab = sr_table_from(sr_kind, sr_table or {})
    if tab is not None:
        keep["sr"] = tab
        p.sr = C.pointer(tab)
    if triples is not None and len(triples):
        tri = np.ascontiguousarray(triples, dtype=np.int32).reshape(-1, 3)
        topo = Topology()
        topo.n_molecules = tri.shape[0]
        topo.triples = _ptr(tri, C.c_int32)
        topo.kb, topo.r0 = float(bonded["kb"]), float(bonded["r0"])
        topo.ka, topo.theta0 = float(bonded["ka"]), float(bonded["theta0"])
        keep["tri"], keep["topo"] = tri, topo
        p.topology = C.pointer(topo)
    return p, keep


def system_kwargs(system) -> dict:
    """Context/build_params keyword arguments of a synth.System."""
    kw = dict(vel=system.vel, types=system.types, sr_kind=system.sr_kind, sr_table=system.sr_table)
    if system.angles is not None and len(system.angles):
        kw["triples"] = system.angles          # (h1, o, h2)
        kw["bonded"] = system.bonded
    return kw


def device_bytes(system, **kw) -> int:
    """Device memory p3maze_init would allocate for this system and setting
    (host-only; p3maze_device_bytes)."""
    p, keep = build_params(system.pos, system.charge, system.mass, system.box, **system_kwargs(system), **kw)
    out = C.c_size_t()
    rc = lib.p3maze_device_bytes(C.byref(p), C.byref(out))
    if rc:
        raise P3MaZeError(rc, lib.p3maze_last_error(None).decode())
    return int(out.value)


class Context:
    """One periodic system resident on the current CUDA device.

    Parameters follow p3maze_params; `stream` is a raw cudaStream_t handle
    (e.g. torch.cuda.Stream().cuda_stream) or None for the default stream."""

    def __init__(self, pos, charges, masses, box: float, *, stream: int | None = None,
                 device_pos: int | None = None, device_vel: int | None = None, **kw):
        """pos: host [n][3] positions (A).  With device_pos/device_vel (device
        addresses of caller-owned [n][3] float64 arrays, e.g. a tensor's
        data_ptr()) the context borrows them as its positions and velocities
        (p3maze_init_device); pos then only gives the shape."""
        self._h = _ctx()
        p, keep = build_params(pos, charges, masses, box, **kw)
        self.n = int(p.n_particles)
        self.mesh_n = int(p.mesh)
        self.box = float(box)
        vel = keep["vel"]
        if device_pos is not None:
            rc = lib.p3maze_init_device(C.byref(p), C.c_void_p(int(device_pos)), C.c_void_p(int(device_vel)),
                                        C.c_void_p(stream or 0), C.byref(self._h))
        else:
            rc = lib.p3maze_init(C.byref(p), _ptr(keep["pos"]), None if vel is None else _ptr(vel),
                                 C.c_void_p(stream or 0), C.byref(self._h))
        if rc:
            raise P3MaZeError(rc, lib.p3maze_last_error(None).decode())
        self.precision = kw.get("precision", "fp64")

    @classmethod
    def from_system(cls, system, **kw) -> "Context":
        """Build from a synth.System (positions, charges, tables, topology)."""
        return cls(system.pos, system.charge, system.mass, system.box, **system_kwargs(system), **kw)

    # ------------------------------------------------------------------ calls
    def _check(self, rc: int):
        if rc:
            raise P3MaZeError(rc, lib.p3maze_last_error(self._h).decode())

    @property
    def handle(self) -> int:
        return self._h.value

    def step(self, n: int = 1):
        self._check(lib.p3maze_step(self._h, int(n)))

    def step_async(self, n: int = 1):
        """Queue n steps without waiting (graph steps); see wait()."""
        self._check(lib.p3maze_step_async(self._h, int(n)))

    def step_host(self, pos_in=None, vel_in=None, n: int = 1, pos_out=None, vel_out=None):
        """Copy pos_in/vel_in in (None keeps the device state), advance n
        steps, copy positions/velocities out into pos_out/vel_out (float64
        C-contiguous [n][3] arrays, filled in place), one host wait."""
        def arg_in(a):
            return None if a is None else _f64(a, (self.n, 3))

        def arg_out(a):
            if a is None:
                return None
            if a.dtype != np.float64 or a.shape != (self.n, 3) or not a.flags.c_contiguous:
                raise ValueError("output arrays must be float64, C-contiguous, shape (n, 3)")
            return a

        pi, vi, po, vo = arg_in(pos_in), arg_in(vel_in), arg_out(pos_out), arg_out(vel_out)
        ptr = lambda a: None if a is None else _ptr(a)
        self._check(lib.p3maze_step_host(self._h, ptr(pi), ptr(vi), int(n), ptr(po), ptr(vo)))

    def wait(self):
        """Wait for queued steps; raises on a recorded solver failure."""
        self._check(lib.p3maze_wait(self._h))

    def set_rollback(self, enable: bool = True):
        """Keep a device copy of the state so that steps ending in a solver
        failure are undone before the error is raised."""
        self._check(lib.p3maze_set_rollback(self._h, 1 if enable else 0))

    def set_solver(self, tol: float, max_mg_iters: int):
        """Constraint tolerance and V-cycle limit of later solves."""
        self._check(lib.p3maze_set_solver(self._h, float(tol), int(max_mg_iters)))

    def equilibrate(self, nsteps: int, temperature: float):
        """nsteps MD steps with velocity rescaling to temperature (K) after each."""
        self._check(lib.p3maze_equilibrate(self._h, int(nsteps), float(temperature)))

    def reinit(self):
        self._check(lib.p3maze_reinit(self._h))

    def energy(self) -> dict:
        e = Energies()
        self._check(lib.p3maze_energy(self._h, C.byref(e)))
        return {k: getattr(e, k) for k, _ in Energies._fields_}

    def stats(self) -> dict:
        s = Stats()
        self._check(lib.p3maze_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def _out(self, out):
        if out is None:
            return np.empty((self.n, 3))
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != 3 * self.n:
            raise ValueError("out must be a C-contiguous float64 array of n*3 elements")
        return out

    def positions(self, out: np.ndarray | None = None) -> np.ndarray:
        out = self._out(out)
        self._check(lib.p3maze_get_positions(self._h, _ptr(out)))
        return out

    def velocities(self, out: np.ndarray | None = None) -> np.ndarray:
        out = self._out(out)
        self._check(lib.p3maze_get_velocities(self._h, _ptr(out)))
        return out

    def forces(self, which: str = "total", out: np.ndarray | None = None) -> np.ndarray:
        out = self._out(out)
        self._check(lib.p3maze_get_forces(self._h, FORCE[which], _ptr(out)))
        return out

    def set_state(self, pos, vel):
        pos = _f64(pos, (self.n, 3))
        vel = _f64(vel, (self.n, 3))
        self._check(lib.p3maze_set_state(self._h, _ptr(pos), _ptr(vel)))

    def mesh(self, which: str) -> np.ndarray:
        """Mesh array indexed [ix, iy, iz] (the library stores x fastest)."""
        n = self.mesh_n
        out = np.empty(n ** 3)
        self._check(lib.p3maze_get_mesh(self._h, MESH[which], _ptr(out)))
        return out.reshape(n, n, n).transpose(2, 1, 0)

    def cells(self):
        st = self.stats()
        nc = st["cells_per_axis"]
        cell = np.empty(self.n, np.int32)
        start = np.empty(nc ** 3 + 1, np.int32)
        order = np.empty(self.n, np.int32)
        self._check(lib.p3maze_get_cells(self._h, _ptr(cell, C.c_int32), _ptr(start, C.c_int32),
                                         _ptr(order, C.c_int32)))
        return nc, cell, start, order

    def set_timing(self, enable: bool = True):
        """Enable per-stage CUDA-event timing and reset the counters."""
        self._check(lib.p3maze_set_timing(self._h, 1 if enable else 0))

    def autotune(self, steps_per_trial: int = 8) -> dict:
        """Time candidate solver settings on real MD steps and keep the fastest."""
        t = Tuning()
        self._check(lib.p3maze_autotune(self._h, int(steps_per_trial), C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def save_state(self) -> np.ndarray:
        """Checkpoint of the full stepping state (p3maze_save_state), as bytes."""
        nb = C.c_size_t()
        self._check(lib.p3maze_state_bytes(self._h, C.byref(nb)))
        buf = np.empty(nb.value, np.uint8)
        self._check(lib.p3maze_save_state(self._h, buf.ctypes.data_as(C.c_void_p), nb.value))
        return buf

    def load_state(self, buf) -> None:
        """Resume from save_state() of a context with the same parameters."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(lib.p3maze_load_state(self._h, b.ctypes.data_as(C.c_void_p), b.nbytes))

    def tuning(self) -> dict:
        """The solver setting in use (the setting keys of autotune())."""
        t = Tuning()
        self._check(lib.p3maze_get_tuning(self._h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_ if k not in TUNING_TIMING}

    def set_tuning(self, **setting):
        """Apply solver settings (keys as tuning(); missing keys are kept)."""
        t = Tuning()
        self._check(lib.p3maze_get_tuning(self._h, C.byref(t)))
        for k, v in setting.items():
            if k not in dict(Tuning._fields_) or k in TUNING_TIMING:
                raise KeyError(k)
            setattr(t, k, int(v))
        self._check(lib.p3maze_set_tuning(self._h, C.byref(t)))

    def set_graphs(self, enable: bool = True):
        """Replay steady-state steps as CUDA graphs (default) or launch eagerly."""
        self._check(lib.p3maze_set_graphs(self._h, 1 if enable else 0))

    def timing(self) -> dict:
        t = Timing()
        self._check(lib.p3maze_get_timing(self._h, C.byref(t)))
        return {"ms": {k: t.ms[i] for i, k in enumerate(STAGES)},
                "launches": {k: t.launches[i] for i, k in enumerate(STAGES)},
                "timed_steps": t.timed_steps, "total_launches": t.total_launches}

    def close(self):
        if self._h and self._h.value:
            lib.p3maze_destroy(self._h)
            self._h = _ctx()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Several contexts advanced together: one CUDA graph launch per batch
    step holds one MD step of every member (p3maze_batch_*)."""

    SHARED_GRAPH, PER_MEMBER = 0, 1

    def __init__(self, stream: int | None = None, mode: str = "shared", fused_smoothing: bool | None = None):
        self._h = C.c_void_p()
        rc = lib.p3maze_batch_create(C.c_void_p(stream or 0), C.byref(self._h))
        if rc:
            raise P3MaZeError(rc, lib.p3maze_last_error(None).decode())
        self.members: list[Context] = []
        if mode != "shared":
            self._check(lib.p3maze_batch_set_mode(self._h, {"per_member": self.PER_MEMBER}[mode]))
        if fused_smoothing is not None:
            self.set_fused_smoothing(fused_smoothing)

    def set_fused_smoothing(self, enable: bool | None):
        """Smooth the members whose smoothing is a cluster launch together
        (one launch per cluster size), each inside its own step, or (None)
        as the mode prefers: together per member, apart in the shared graph."""
        self._check(lib.p3maze_batch_set_fused_smoothing(self._h, -1 if enable is None else 1 if enable else 0))

    def _check(self, rc: int):
        if rc:
            raise P3MaZeError(rc, lib.p3maze_batch_last_error(self._h).decode())

    def add(self, ctx: Context):
        self._check(lib.p3maze_batch_add(self._h, ctx._h))
        self.members.append(ctx)

    def remove(self, ctx: Context):
        self._check(lib.p3maze_batch_remove(self._h, ctx._h))
        self.members.remove(ctx)

    def step(self, n: int = 1):
        self._check(lib.p3maze_batch_step(self._h, int(n)))

    def wait(self):
        self._check(lib.p3maze_batch_wait(self._h))

    def __len__(self):
        return int(lib.p3maze_batch_size(self._h))

    def close(self):
        if self._h and self._h.value:
            lib.p3maze_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
