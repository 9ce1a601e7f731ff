"""Continuous-batching server for independent P3MaZe systems on one GPU.

Requests -- "advance this system by N MD steps" -- arrive over time.  The
server admits them as batch slots and device memory free up (the memory a
system needs comes from p3maze_device_bytes), prepares each admitted system
on an admission thread (its seeded configuration, its context, the initial
constraint solve and its first steps) while the resident systems keep
stepping, keeps every admitted system's particles, meshes and multigrid
hierarchy resident, advances all resident systems together (one batch step
per iteration: each member replays its captured step graph on its own
stream, so their kernels overlap on the device), and retires each system
when its steps are done.  Requests that arrive while others are running
join at a step boundary once prepared.

The GPU work sits behind a small backend interface so that the admission and
bookkeeping logic can be exercised on the CPU with a fake backend.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth as S

NACL_DENSITY = 0.031899      # ions per A^3 (molten NaCl at the 32768-ion box size)
WATER_DENSITY = 0.033427     # molecules per A^3 (1.0 g/cm^3)
MESH_SPACING = 0.8           # A, target mesh spacing of served systems


@dataclass
class Request:
    rid: int
    kind: str                # "nacl" or "water"
    n_atoms: int
    seed: int
    steps: int
    arrival: float           # seconds after the start of the run
    admitted: float | None = None
    finished: float | None = None
    status: str = "queued"   # queued, starting, running, done, failed, rejected
    step_latencies: list = field(default_factory=list)
    result: dict = field(default_factory=dict)
    admit_host_s: float = 0.0  # host time of the preparation (system, context, first steps)


def allowed_mesh(target: float, lo: int = 16, hi: int = 128) -> int:
    """Smallest N >= target (clamped to [lo, hi]) that is a multiple of 4 (the
    vectorised FP32 diffusion kernel) and a valid multigrid mesh: halving
    while even and above 16 must end at 64 or below (the exact coarse solve)."""
    want = max(lo, int(math.ceil(target)))
    n = want + (-want) % 4
    while n <= hi:
        m = n
        while m > 16 and m % 2 == 0:
            m //= 2
        if m <= 64:
            return n
        n += 4
    return hi


def request_system(req: Request):
    """Seeded synthetic system of a request and its solver parameters."""
    if req.kind == "nacl":
        n = max(2, req.n_atoms - req.n_atoms % 2)
        box = (n / NACL_DENSITY) ** (1.0 / 3.0)
        system = S.nacl_melt(n, box, seed=req.seed)
        dt = 1.0
    else:
        nmol = max(1, req.n_atoms // 3)
        box = (nmol / WATER_DENSITY) ** (1.0 / 3.0)
        system = S.spcfw_water(nmol, box, seed=req.seed)
        dt = 0.5
    mesh = allowed_mesh(box / MESH_SPACING)
    params = dict(alpha=S.EWALD_ALPHA, r_cut=min(S.R_CUT, box), mesh=mesh, tol=S.TOL, dt=dt)
    return system, params


def poisson_requests(n: int, rate: float, seed: int, lo: int = 216, hi: int = 32768, steps: int = 200):
    """n requests with Poisson arrivals (rate per second), kinds 50/50 and
    atom counts log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        kind = "nacl" if rng.random() < 0.5 else "water"
        atoms = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append(Request(rid=i, kind=kind, n_atoms=atoms, seed=1000 + i, steps=steps, arrival=t))
    return out


# ----------------------------------------------------------------- backends
class GpuBackend:
    """Resident contexts in a per-member batch on the current CUDA device.

    Admission work runs on a host thread of its own: the request's seeded
    system is generated, its context created (device allocation, the initial
    constraint solve) and advanced by its first steps (the ones that fill the
    multiplier history and test convergence on the host), all on the
    admission stream, while the stepping thread keeps advancing the batch.
    A prepared context joins the batch at the next step boundary.  One
    admission thread: contexts are created one at a time (a context is used
    by one thread at a time -- the admission thread until it hands it over).
    """

    WARMUP_STEPS = 3                        # fills the predictor history of any order

    def __init__(self, precision: str = "mixed", stream: int | None = None, admit_stream: int | None = None,
                 smoothing: str = "default"):
        """smoothing: "default" smooths meshes of at most 64^3 in cluster
        launches, fused across the batch's members (between separately
        launched member graphs this beats each member's own smoothing);
        "per_step" forces one diffusion kernel launch per two steps (the
        25-point kernel), for comparison."""
        import queue
        import threading

        from . import p3maze as P

        self.P = P
        self.precision = precision
        self.stream = stream
        self.admit_stream = admit_stream
        self.batch = P.Batch(stream=stream, mode="per_member")
        self.clock = time.perf_counter
        self.steps = {}                     # host-side step count per member
        self.smoothing = smoothing
        self._todo = queue.Queue()
        self._ready = queue.Queue()
        self._worker = threading.Thread(target=self._admit_loop, name="p3maze-admission", daemon=True)
        self._worker.start()

    def estimate(self, req: Request) -> int:
        system, prm = request_system(req)
        return self.P.device_bytes(system, precision=self.precision, **prm)

    def _admit_loop(self):
        while True:
            req = self._todo.get()
            if req is None:
                return
            t0 = time.perf_counter()
            try:
                system, prm = request_system(req)
                ctx = self.P.Context.from_system(system, precision=self.precision, stream=self.admit_stream, **prm)
                if ctx.tuning()["diffusion_fuse"] >= 5:  # spectral default: meshes of at most 64^3, or 128^3
                    if self.smoothing == "per_step":
                        ctx.set_tuning(diffusion_fuse=2 if prm["mesh"] % 4 == 0 else 1, diffusion_zc=2)
                    else:
                        # the cluster launch, fused across the batch's members
                        try:
                            ctx.set_tuning(diffusion_fuse=5)
                        except self.P.P3MaZeError:
                            pass                # no such clusters (or a 128^3 mesh): keep the default
                ctx.step(self.WARMUP_STEPS)
                self._ready.put((req, ctx, time.perf_counter() - t0, None))
            except Exception as e:          # reported to the stepping thread
                self._ready.put((req, None, time.perf_counter() - t0, e))

    def submit(self, req: Request):
        """Queue a request's preparation on the admission thread."""
        self._todo.put(req)

    def poll(self, block: bool = False) -> list:
        """Prepared requests: (request, handle or None, admission host seconds,
        error or None).  block: wait for at least one."""
        import queue

        out = []
        try:
            out.append(self._ready.get(block=block))
            while True:
                out.append(self._ready.get_nowait())
        except queue.Empty:
            pass
        return out

    def attach(self, ctx):
        """Join a prepared context to the batch (its history is full, so no
        steps run here)."""
        self.batch.add(ctx)
        self.steps[ctx] = ctx.stats()["steps"]

    def steps_done(self, handle) -> int:
        return self.steps[handle]

    def step(self) -> list:
        """One batch step of all members; returns the members that failed."""
        self.batch.step(1)
        for ctx in self.batch.members:
            self.steps[ctx] += 1
        try:
            self.batch.wait()
            return []
        except self.P.P3MaZeError:
            failed = []
            for ctx in list(self.batch.members):
                # a failure is recorded per member on the device
                try:
                    ctx.wait()
                except self.P.P3MaZeError:
                    failed.append(ctx)
            return failed

    def result(self, handle) -> dict:
        e = handle.energy()
        return {"energy": e["total"], "positions": handle.positions(), "steps": handle.stats()["steps"]}

    def close(self, handle):
        if handle in self.batch.members:
            self.batch.remove(handle)
        self.steps.pop(handle, None)
        handle.close()

    def sleep_until(self, t_abs: float):
        dt = t_abs - self.clock()
        if dt > 0:
            time.sleep(dt)

    def shutdown(self):
        self._todo.put(None)
        self._worker.join()
        for req, ctx, _, _ in self.poll():
            if ctx is not None:
                ctx.close()
        self.batch.close()


# ----------------------------------------------------------------- server
class Server:
    """Continuous batching: the stepping loop reserves a slot and the
    request's device memory, hands the request to the backend's admission
    worker, keeps stepping the resident systems, and attaches each prepared
    system at the next step boundary."""

    def __init__(self, backend, budget_bytes: int, max_slots: int, margin: float = 1.05,
                 margin_bytes: int = 4 << 20):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.margin = margin
        self.margin_bytes = margin_bytes
        self.used = 0
        self.peak_used = 0
        self.peak_slots = 0                 # slots taken: resident systems and systems being prepared
        self.peak_resident = 0              # systems stepping together on the device

    def _need(self, req: Request) -> int:
        return int(self.backend.estimate(req) * self.margin) + self.margin_bytes

    def run(self, requests: list[Request]) -> dict:
        be = self.backend
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        starting: dict[int, int] = {}       # rid -> bytes reserved, preparation in flight
        active: dict[int, tuple] = {}       # rid -> (request, handle, bytes)
        t0 = be.clock()
        need = {}

        def attach(ready):
            for req, handle, host_s, err in ready:
                nbytes = starting.pop(req.rid)
                req.admit_host_s = host_s
                if err is not None or handle is None:
                    req.status = "failed"
                    req.finished = be.clock() - t0
                    self.used -= nbytes
                    continue
                be.attach(handle)
                req.admitted = be.clock() - t0
                req.status = "running"
                active[req.rid] = (req, handle, nbytes)

        while pending or queue or active or starting:
            now = be.clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            attach(be.poll())
            # admission: FIFO, later arrivals may pass a head that does not fit
            for req in list(queue):
                if len(active) + len(starting) >= self.max_slots:
                    break
                if req.rid not in need:
                    need[req.rid] = self._need(req)
                if need[req.rid] > self.budget:
                    req.status = "rejected"
                    queue.remove(req)
                    continue
                if self.used + need[req.rid] > self.budget:
                    continue
                queue.remove(req)
                req.status = "starting"
                starting[req.rid] = need[req.rid]
                self.used += need[req.rid]
                be.submit(req)
            self.peak_used = max(self.peak_used, self.used)
            self.peak_slots = max(self.peak_slots, len(active) + len(starting))
            if not active:
                if starting:
                    attach(be.poll(block=True))
                    continue
                if pending:
                    be.sleep_until(t0 + pending[0].arrival)
                    continue
                if queue:
                    continue
                break
            self.peak_resident = max(self.peak_resident, len(active))
            t_step = be.clock()
            failed = be.step()
            lat = be.clock() - t_step
            done = []
            for rid, (req, handle, nbytes) in active.items():
                if handle in failed:
                    req.status = "failed"
                    done.append(rid)
                    continue
                req.step_latencies.append(lat)
                if be.steps_done(handle) >= req.steps:   # steps since the system's start
                    req.result = be.result(handle)
                    req.status = "done"
                    done.append(rid)
            for rid in done:
                req, handle, nbytes = active.pop(rid)
                req.finished = be.clock() - t0
                be.close(handle)
                self.used -= nbytes
        return self.metrics(requests, be.clock() - t0)

    def metrics(self, requests: list[Request], makespan: float) -> dict:
        done = [r for r in requests if r.status == "done"]
        steps = sum(len(r.step_latencies) for r in done)
        atom_steps = sum(len(r.step_latencies) * r.n_atoms for r in done)
        lat = np.concatenate([np.asarray(r.step_latencies) for r in done]) if done else np.zeros(1)
        rl = np.asarray([r.finished - r.arrival for r in done]) if done else np.zeros(1)
        qw = np.asarray([r.admitted - r.arrival for r in done]) if done else np.zeros(1)
        ah = np.asarray([getattr(r, "admit_host_s", 0.0) for r in done]) if done else np.zeros(1)
        return {
            "requests": len(requests), "done": len(done),
            "failed": sum(r.status == "failed" for r in requests),
            "rejected": sum(r.status == "rejected" for r in requests),
            "makespan_s": makespan,
            "steps_per_s": steps / makespan if makespan > 0 else 0.0,
            "atom_steps_per_s": atom_steps / makespan if makespan > 0 else 0.0,
            "step_latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
            "step_latency_ms_p99": 1e3 * float(np.percentile(lat, 99)),
            "request_latency_s_p50": float(np.percentile(rl, 50)),
            "request_latency_s_p99": float(np.percentile(rl, 99)),
            "queue_wait_s_p50": float(np.percentile(qw, 50)),
            "queue_wait_s_p99": float(np.percentile(qw, 99)),
            "admission_host_s_p50": float(np.percentile(ah, 50)),
            "admission_host_s_p99": float(np.percentile(ah, 99)),
            "peak_bytes": self.peak_used, "peak_slots": self.peak_slots, "peak_resident": self.peak_resident,
        }
