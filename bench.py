#!/usr/bin/env python
"""Benchmark of one P3MaZe molecular-dynamics step on a B300.

Workload (seeded, synthetic): molten NaCl, 32768 ions (16384 Na+, 16384 Cl-)
in a cubic box L = 100.9 A, uniform random positions with minimum pair
distance 2 A, Maxwell-Boltzmann velocities at 1200 K, Tosi-Fumi
Born-Mayer-Huggins short-range term, Ewald alpha 0.30 1/A, r_cut 9 A, 128^3
mesh, cubic B-spline assignment, constraint tolerance 1e-6, dt 1 fs.

One step = one velocity-Verlet MD step through the whole path: kick/drift,
cell list, charge assignment, 25 diffusion smoothing steps, Mass-Zero
prediction and multigrid correction solve to tol, field update, erfc +
Born-Mayer pair forces, force interpolation, kick.  Inputs are resident on
the device when the timed region starts.  The timed steps run back to back,
as in an MD run; each step reads and writes about 160 MB of mesh state, more
than the 126 MB L2.  The same number of steps with the L2 overwritten
(256 MiB) before each, outside the step's events, is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "nacl_32k"
METRIC = "ns/day, molten NaCl 32768 ions, 128^3 mesh (full MD step with Mass-Zero long-range solve)"
DATA = "synthetic: seeded molten-NaCl configuration (uniform random, d_min 2 A, 1200 K Maxwell-Boltzmann)"


def ns_per_day(sec_per_step: float, dt_fs: float) -> float:
    return 86400.0 / sec_per_step * dt_fs * 1e-6


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest x over all ranks (the slowest replica sets the whole job's
    time).  torch.distributed must be initialised when world > 1; the tensor
    lives on ``device`` (a CUDA device for NCCL, the CPU for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ns_per_day(ms_per_step_max: float, world: int, dt_fs: float) -> float:
    """Whole-job throughput of ``world`` independent replicas, each of which
    advances its own system by one step in at most ms_per_step_max."""
    return world * ns_per_day(ms_per_step_max * 1e-3, dt_fs)


def workload_config(prm):
    """The workload both arms run (identical in the GPU and the oracle line;
    how each arm computes it is under "settings" and "dtype")."""
    return {
        "workload": "molten NaCl, 32768 ions, L=100.9 A, 128^3 mesh, alpha 0.30/A, r_cut 9 A, "
                    "order-4 B-spline, tol 1e-6, dt 1 fs, NVE",
        "n_particles": 32768, "mesh": prm["mesh"], "tol": prm["tol"], "dt_fs": prm["dt"],
        "l2": "inputs larger than L2: the timed GPU steps run back to back, as in an MD run, and each step "
              "reads and writes about 160 MB of mesh state (phi and psi at two times, two multiplier-history "
              "buffers and the residual as 64-bit fixed point, five FP32 meshes at 128^3), more than the "
              "126 MB L2; the same steps with a 256 MiB L2 overwrite before each are ms_per_step_l2_flushed",
        "parallelism": "replicas (one independent system per GPU, no collective)",
        "parameters": "Fumi-Tosi BMH table written from memory, not verified against the 1964 source "
                      "(parity does not depend on it: both arms read the same table)",
    }


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and throttle reasons sampled during the timed region: an NVML
    thread polling every ~2 ms (nvidia-smi -lms 200 as a fallback)."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, gpu_index: str | None):
        self.gpu = gpu_index
        self.samples = []
        self._stop = False
        self._thread = None
        self.proc = None
        self.path = None
        self.handle = None
        self.nvml_error = None
        self.lib = None

    def _nvml_handle(self):
        """Open NVML through ctypes (read-only queries) and return the handle
        of this process's CUDA device, matched by UUID."""
        import ctypes

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        self.lib = lib
        h = ctypes.c_void_p()
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            if lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0:
                return h
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        first = vis.split(",")[0].strip() if vis else ""
        if first.startswith("GPU-"):
            rc = lib.nvmlDeviceGetHandleByUUID(first.encode(), ctypes.byref(h))
        else:
            idx = int(first) if first.isdigit() else int(self.gpu or 0)
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"NVML device handle lookup failed ({rc})")
        return h

    def _poll(self):
        import ctypes

        lib = self.lib
        try:
            get_reasons = lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            get_reasons = lib.nvmlDeviceGetCurrentClocksThrottleReasons
        sm, smax, reasons = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        NVML_CLOCK_SM = 1
        while not self._stop:
            ok = (lib.nvmlDeviceGetClockInfo(self.handle, NVML_CLOCK_SM, ctypes.byref(sm)) == 0 and
                  lib.nvmlDeviceGetMaxClockInfo(self.handle, NVML_CLOCK_SM, ctypes.byref(smax)) == 0 and
                  get_reasons(self.handle, ctypes.byref(reasons)) == 0)
            if ok:
                self.samples.append((sm.value, smax.value, reasons.value))
            time.sleep(0.002)

    def __enter__(self):
        import threading
        try:
            self.handle = self._nvml_handle()
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
            t0 = time.time()
            while not self.samples and time.time() - t0 < 1.0:
                time.sleep(0.001)
            self.samples.clear()            # keep only samples taken inside the region
        except Exception as exc:
            self.handle = None
            self.nvml_error = f"{type(exc).__name__}: {exc}"
            try:
                fd, self.path = tempfile.mkstemp(suffix=".csv")
                os.close(fd)
                fields = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                          "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                          "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
                cmd = ["nvidia-smi", f"--query-gpu={fields}", "--format=csv,noheader,nounits", "-lms", "200"]
                if self.gpu is not None:
                    cmd += ["-i", self.gpu]
                self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            except Exception:
                self.proc = None
        return self

    def __exit__(self, *a):
        self._stop = True
        if self._thread is not None:
            self._thread.join(timeout=1.0)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if self.samples:
            sm = [s[0] for s in self.samples]
            reasons = sorted({k for s in self.samples for k, bit in self.REASONS.items() if s[2] & bit})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(s[1] for s in self.samples),
                    "samples": len(sm), "source": "nvml", "reasons": reasons}
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "nvml_error": self.nvml_error}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "source": "nvidia-smi", "nvml_error": self.nvml_error, "reasons": sorted(reasons)}


# ----------------------------------------------------------------- roofline
def smoothing_launches(K: int, fuse: int) -> int:
    """Diffusion launches per MD step: one per step, or two steps per launch
    (a single step first when K is odd), or fuse = 3, 4 steps per launch;
    all steps in one cluster launch (5) or three transform launches (6)."""
    if fuse == 2:
        return K // 2 + K % 2
    if fuse == 5:
        return 1
    if fuse == 6:
        return 3
    if fuse > 2:
        return -(-K // fuse)
    return K


def fft_smoothing_flops(n: int) -> float:
    """Algorithmic FP32 operations of one spectral smoothing by FFT on an n^3
    mesh: six passes of n^2 / 2 complex radix-2 FFTs of length n (5 n log2 n
    each, the textbook count), the split of each into two Hartley lines
    (3 per output point), and the scaling (1 per point)."""
    lg = math.log2(n)
    return 6.0 * (2.5 * n ** 3 * lg + 3.0 * n ** 3) + n ** 3


def fp32_peak_tflops(sm_mhz: float, sms: int = 148) -> float:
    """FP32 peak from unit counts: 128 FP32 lanes per SM (four sub-partitions
    of 32), one FMA (2 operations) per lane per clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# kernel of each mesh stage (mixed precision / FP64)
STAGE_KERNEL = {"spread": ("k_spread_tile", "k_spread_tile"),
                "predict": ("k_predict_resid_fix", "k_predict"),
                "update": ("k_update_fix", "k_update"),
                "gather": ("k_gather_mp", "k_gather")}


def algorithmic_bytes(stage: str, b: int, P: int, npart: int, K: int, fuse: int = 1,
                      order: int = 3) -> tuple[float, int]:
    """Compulsory bytes of one launch of the stage's main kernel and the
    launches per step.  b = bytes of a bulk mesh value, P = mesh points.
    A smoothing launch (one diffusion step, or several fused) reads the mesh
    once and writes it once."""
    if stage == "smooth":
        return 2.0 * P * b, smoothing_launches(K, fuse)
    if stage == "spread":        # write q once, read 32 B per particle
        return P * b + 32.0 * npart, 1
    if stage == "predict":       # read Psi^k, Psi^{k-1}, q^s and `order` multiplier histories (8 B each);
        # write the residual and the guess y0 (8 B each), in mixed mode also the FP32 residual copy
        return P * (8 + 8 + b + 8 * order + 16 + (4 if b == 4 else 0)), 1
    if stage == "update":        # read phi^k, phi^{k-1}, y; write phi^{k+1}
        return P * 32.0, 1
    if stage == "gather":        # read phi once, 32 B per particle in, 3 x 24 B out
        return P * 8.0 + 104.0 * npart, 1
    return float("nan"), 1


def kernel_source_sha(kernel: str) -> str | None:
    """sha256 prefix of a kernel's own source text (from its name at the
    start of a line to the end of its body) in the package's CUDA headers."""
    import hashlib
    import re

    for f in ("mesh.cuh", "particles.cuh"):
        with open(os.path.join(ROOT, "paper_2606_31379_b300", "csrc", f)) as fh:
            src = fh.read()
        m = re.search(r"^" + re.escape(kernel) + r"\(", src, re.M)
        if m:
            return hashlib.sha256(src[m.start():src.index("\n}\n", m.start()) + 3].encode()).hexdigest()[:16]
    return None


def recorded_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per launch from the committed ncu record, if it was taken on
    the kernel's current source (profiles/roofline_traffic.json)."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)[f"{kernel}|{workload}|{precision}"]
        ok = kernel_source_sha(kernel) == rec["kernel_source_sha256_16"]
        return float(rec["dram_bytes_per_launch"]) if ok else None
    except Exception:
        return None


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "source": "fallback"}


# ----------------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


def oracle_md_steps(system, prm, steps: int, budget_s: float, warmup: int = 0) -> dict:
    """Whole MD steps of the oracle's plain FP64 Mass-Zero stepper
    (oracle.maze_md_step) on one host core, unextrapolated: kick and drift,
    assignment, smoothing, the Verlet-predicted field and its multigrid
    correction to tol (red-black Gauss-Seidel 2+2, exact coarse level at
    <= 64^3), field update, interpolation, short-range forces through the
    oracle's cell list, kick.  The start (exact field and forces at the
    initial positions) is set up untimed.  Steps are timed until `steps` are
    done or `budget_s` of timed work is spent (at least one); the steps
    actually timed are reported."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:          # numpy's FFT and array ops run on one thread anyway
        import contextlib

        def threadpool_limits(_n):
            return contextlib.nullcontext()
    import copy

    from oracle import p3maze_oracle as O

    sysm = copy.deepcopy(system)
    n, dt = prm["mesh"], prm["dt"]
    args = (prm["alpha"], prm["r_cut"], n, dt, prm["tol"])
    with threadpool_limits(1):
        t0 = time.perf_counter()
        state = O.maze_initial_state(sysm, prm["alpha"], prm["r_cut"], n)
        setup_s = time.perf_counter() - t0
        for _ in range(warmup):
            O.maze_md_step(sysm, state, *args)
        sec, sr, iters = [], [], []
        while len(sec) < max(1, steps):
            tim = {}
            t = time.perf_counter()
            iters.append(O.maze_md_step(sysm, state, *args, timings=tim))
            sec.append(time.perf_counter() - t)
            sr.append(tim["sr"])
            if sum(sec) >= budget_s:
                break
    mean = sum(sec) / len(sec)
    mesh = mean - sum(sr) / len(sr)
    sigma = O.sigma_of_alpha(prm["alpha"])
    K, _ = O.smoothing_schedule(sigma, system.box / n)
    desc = (f"{len(sec)} whole MD step(s) of the FP64 oracle's Mass-Zero stepper on {system.n} ions, {n}^3 "
            f"({K} smoothing steps, {sum(iters) / len(iters):g} multigrid V-cycles per step to tol "
            f"{prm['tol']:g}, cell-list short-range forces); 1 thread; untimed set-up {setup_s:.1f} s")
    return {"sec_per_step": mean, "mesh_sec_per_step": mesh, "sr_sec_per_step": sum(sr) / len(sr),
            "steps_timed": len(sec), "warmup_run": warmup, "vcycles_per_step": sum(iters) / len(iters),
            "setup_s": setup_s, "sample": desc}


def cpu_baseline(system, prm, budget_s: float = 15.0) -> dict:
    r = oracle_md_steps(system, prm, 1, budget_s)
    return {"value": ns_per_day(r["sec_per_step"], prm["dt"]), "unit": "ns/day", "cores": 1, "kind": "oracle",
            "sample": r["sample"], "sec_per_step": r["sec_per_step"],
            "mesh_sec_per_step": r["mesh_sec_per_step"], "sr_sec_per_step": r["sr_sec_per_step"],
            "cpu_model": cpu_model(), "cores_available": os.cpu_count()}


def run_reference(args) -> int:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2606_31379_b300 import synth as S
    system, prm = S.make_workload(WORKLOAD)
    # the oracle has no warm-up effects (no JIT, caches or clocks to settle):
    # at most one untimed step, and whole steps timed within a bounded budget
    r = oracle_md_steps(system, prm, args.steps, budget_s=args.reference_budget, warmup=min(args.warmup, 1))
    sec = r["sec_per_step"]
    value = ns_per_day(sec, prm["dt"])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": args.gpus,
        "steps": r["steps_timed"], "warmup": r["warmup_run"], "steps_requested": args.steps,
        "warmup_requested": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": DATA,
        "config": workload_config(prm),
        "settings": {"precision": "fp64 (CPU oracle)", "start": "seeded random configuration (no equilibration)"},
        "cpu_baseline": {"value": value, "unit": "ns/day", "cores": 1, "kind": "oracle", "sample": r["sample"],
                         "mesh_sec_per_step": r["mesh_sec_per_step"], "sr_sec_per_step": r["sr_sec_per_step"],
                         "cpu_model": cpu_model(), "cores_available": os.cpu_count()},
        "e2e": {"value": value, "unit": "ns/day", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- accuracy
def accuracy_vs_oracle(ctx, system, prm, n_sample: int = 64) -> dict:
    """Errors of a context's observables against the FP64 oracle at the
    context's own current positions: the mesh force of every particle and the
    total force of a seeded sample (relative RMS), and each energy term of
    Eqs. 5, 6 and 14 plus the non-Coulomb term (relative error)."""
    import copy

    from oracle import p3maze_oracle as O

    s = copy.copy(system)
    s.pos = ctx.positions()
    sample = np.random.default_rng(7).choice(s.n, n_sample, replace=False)
    mf = O.mesh_fields(s, prm["alpha"], prm["mesh"])
    F_lr = O.interpolate_lr_forces(s.pos, s.charge, s.box, prm["mesh"], mf["phi"])
    F_sr_s, _, _ = O.sr_forces(s, mf["sigma"], prm["r_cut"], subset=sample)
    _, ec, ev = O.sr_forces_cells(s, mf["sigma"], prm["r_cut"])
    ref = {"v_lr": 0.5 * O.COULOMB_K * float((mf["phi"] * mf["q"]).sum()), "v_sr": float(ec.sum()),
           "v_vdw": float(ev.sum()), "v_self": O.self_energy(s.charge, mf["sigma"])}

    def rel_rms(a, b):
        return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))

    e = ctx.energy()
    return {"force_lr_rel_rms": rel_rms(ctx.forces("lr"), F_lr),
            "force_rel_rms_sampled": rel_rms(ctx.forces()[sample], F_lr[sample] + F_sr_s),
            "energy_rel_err": {k: abs(e[k] - v) / abs(v) for k, v in ref.items()},
            "sample": f"{n_sample} particles (seeded) for the total force; mesh force and energies over all "
                      f"{s.n}; oracle field by the FFT solve, short-range energy through the oracle's cell list",
            "bars": {"note": "the parity tests' bars, 1e-5 (FP64) / 1e-4 (mixed) relative RMS on forces, hold "
                             "with the constraint solved to tol 1e-8..1e-9; here the field is solved to the "
                             "workload's tol (max|r| <= 1e-6), whose own error, set by tol and the solver "
                             "setting, dominates the mesh force"}}


# ----------------------------------------------------------------- GPU arm
def time_context(ctx, torch, stream, steps: int, flush=None):
    """K timed steps (CUDA events on ctx's stream); returns per-step ms.
    flush=None: the K steps back to back, one event pair around them (the
    per-step list is their mean K times); else the L2 is overwritten with
    `flush` before every step and each step is timed alone."""
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            ctx.step(steps)
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) / steps] * steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            ctx.step(1)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_ours(args) -> int:
    import torch
    import torch.distributed as dist
    from paper_2606_31379_b300 import p3maze as P
    from paper_2606_31379_b300 import synth as S

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    system, prm = S.make_workload(WORKLOAD)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # The seeded random start (d_min 2 A) is far from equilibrium and heats up
    # by hundreds of kelvin in the first hundreds of fs.  Equilibrate once at
    # 1200 K with velocity rescaling (untimed) and start every measured context
    # from that state, as the paper measures in the equilibrated regime.
    with P.Context.from_system(system, alpha=prm["alpha"], r_cut=prm["r_cut"], mesh=prm["mesh"],
                               tol=prm["tol"], dt=prm["dt"], precision="mixed", stream=stream.cuda_stream) as eq:
        eq.equilibrate(args.equilibrate, 1200.0)
        system.pos = eq.positions()
        system.vel = eq.velocities()

    def make(precision):
        return P.Context.from_system(system, alpha=prm["alpha"], r_cut=prm["r_cut"], mesh=prm["mesh"],
                                     tol=prm["tol"], dt=prm["dt"], precision=precision,
                                     stream=stream.cuda_stream)

    ctx = make(args.precision)
    if args.no_graphs:
        ctx.set_graphs(False)
    ctx.step(args.warmup)
    if args.tuning:
        ctx.set_tuning(**json.loads(args.tuning))
        tuning = dict(ctx.tuning(), source="--tuning")
    else:
        tuning = None if args.no_tune else ctx.autotune(40)
    # the warm-up steps again with the final setting: a setting change drops
    # the step graphs, and these steps record them (one per pointer phase of
    # the field and correction rings) outside the timed region
    ctx.step(max(args.warmup, 4))
    torch.cuda.synchronize()
    gpu_id = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if world == 1 else str(local)
    it0 = ctx.stats()["total_iters"]
    launches0 = ctx.timing()["total_launches"]
    barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    with ClockSampler(gpu_id) as clk:
        ms = time_context(ctx, torch, stream, args.steps)
    clocks = clk.summary()
    fuse_used = ctx.tuning()["diffusion_fuse"]
    pred_used = ctx.tuning()["predictor"]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    iters = (ctx.stats()["total_iters"] - it0) / args.steps
    launches = ctx.timing()["total_launches"] - launches0
    # the same number of steps with the L2 overwritten before each one
    ms_flushed = time_context(ctx, torch, stream, args.steps, flush)
    # stage breakdown: the same number of steps again with CUDA events around
    # each stage (recorded inside the step graph; not part of the headline)
    ctx.set_timing(True)
    ctx.step(2)
    ctx.set_timing(True)                    # reset the stage tallies
    ms_staged = time_context(ctx, torch, stream, args.steps)
    tm = ctx.timing()
    ctx.set_timing(False)
    # accuracy of the state the timed setting produced (before the
    # end-to-end and one-kernel measurements below change anything)
    accuracy = None if (args.no_accuracy or rank != 0) else accuracy_vs_oracle(ctx, system, prm)
    total_ms = max_over_ranks(sum(ms), world, device="cuda")
    ms_per_step = total_ms / args.steps
    value = job_ns_per_day(ms_per_step, world, prm["dt"])

    # end to end through the C ABI with pinned host buffers, every step: the
    # state (r, v) copied in from the host, one MD step, r and v copied back
    # out, one host wait (p3maze_step_host).  Stage timing is off here, as in
    # a production run.
    ctx.set_timing(False)
    pos_h = torch.empty((system.n, 3), dtype=torch.float64, pin_memory=True).numpy()
    vel_h = torch.empty((system.n, 3), dtype=torch.float64, pin_memory=True).numpy()
    ctx.positions(out=pos_h)
    ctx.velocities(out=vel_h)
    for _ in range(3):
        ctx.step_host(pos_h, vel_h, 1, pos_h, vel_h)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.step_host(pos_h, vel_h, 1, pos_h, vel_h)
    torch.cuda.synchronize()
    e2e_sec = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, device="cuda")
    e2e = {"value": job_ns_per_day(1e3 * e2e_sec, world, prm["dt"]), "unit": "ns/day",
           "h2d_bytes_per_step": int(pos_h.nbytes + vel_h.nbytes),
           "d2h_bytes_per_step": int(pos_h.nbytes + vel_h.nbytes), "steps": e2e_steps}
    K_smooth = ctx.stats()["smooth_steps"]
    # the one-step diffusion kernel alone, live in real MD steps: one launch
    # per diffusion step and nothing beside it (pair branch forked after
    # smoothing); CUDA events around the smoothing stage on the work stream
    ctx.set_tuning(diffusion_fuse=1, diffusion_zc=2, pair_fork=0)
    ctx.set_timing(True)
    ctx.step(2)
    ctx.set_timing(True)
    n_alone = max(5, args.steps // 2)
    time_context(ctx, torch, stream, n_alone, flush)
    alone_launch_us = 1e3 * ctx.timing()["ms"]["smooth"] / n_alone / K_smooth
    ctx.close()

    # beside the headline: the plain FP64 path, the multiplier predictors and
    # the real-space P3M baseline (Sec. 3.3) and PMaZe on the same workload
    variants = {}
    if not args.no_variants:
        # fp64: the plain FP64 path, autotuned like the headline.  The
        # predictor / P3M study keeps the default sweeps (2, 2) and its own
        # predictor so the solvers compare as in Fig. 8.
        studies = [("fp64", dict(precision="fp64")),
                   ("maze_y1", dict(precision=args.precision, predictor=1)),
                   ("maze_y2", dict(precision=args.precision, predictor=2)),
                   ("maze_y3", dict(precision=args.precision, predictor=3)),
                   ("p3m", dict(precision=args.precision, method="p3m")),
                   # PMaZe: the whole Coulomb problem on a mesh of twice the
                   # points per axis (the paper's NaCl comparison: 60^3 -> 120^3)
                   ("pmaze", dict(precision=args.precision, method="pmaze", mesh=2 * prm["mesh"], alpha=0.0))]
        for name, kw in studies:
            if name == "fp64" and args.precision == "fp64":
                continue
            ckw = dict(alpha=prm["alpha"], r_cut=prm["r_cut"], mesh=prm["mesh"], tol=prm["tol"], dt=prm["dt"])
            ckw.update(kw)
            cv = P.Context.from_system(system, stream=stream.cuda_stream, **ckw)
            cv.step(args.warmup)
            tv_tune = None if (args.no_tune or name != "fp64") else cv.autotune(8)
            if tv_tune is not None:
                cv.step(max(args.warmup, 4))  # the step graphs of the final setting, untimed
            it0 = cv.stats()["total_iters"]
            msv = time_context(cv, torch, stream, args.steps)
            itv = (cv.stats()["total_iters"] - it0) / args.steps
            cv.set_timing(True)
            cv.step(2)
            cv.set_timing(True)
            time_context(cv, torch, stream, args.steps)
            tv = cv.timing()
            msv_step = max_over_ranks(sum(msv), world, device="cuda") / args.steps
            if name == "fp64" and not args.no_accuracy and rank == 0:
                acc_v = accuracy_vs_oracle(cv, system, prm)
            else:
                acc_v = None
            variants[name] = {
                "value": job_ns_per_day(msv_step, world, prm["dt"]),
                "ms_per_step": msv_step,
                "mg_iters_per_step": itv,
                "stage_us": {k: 1e3 * v / args.steps for k, v in tv["ms"].items()},
                "settings": {k: v for k, v in kw.items()},
                "accuracy_vs_oracle": acc_v,
                "tuning": tv_tune,
            }
            cv.close()

    if rank != 0:
        return 0
    stage_us = {k: 1e3 * v / args.steps for k, v in tm["ms"].items()}
    lr_stages = ("spread", "smooth", "predict", "solve", "update", "gather")
    b = 4 if args.precision == "mixed" else 8
    P3 = prm["mesh"] ** 3
    # dominant mesh stage by time
    mesh_stages = ("smooth", "spread", "predict", "update", "gather")
    dom = max(mesh_stages, key=lambda k: stage_us[k])
    peaks = measured_peaks()
    fuse = fuse_used
    if dom == "smooth" and fuse == 6:
        # spectral smoothing by FFT: FP32 arithmetic on L2-resident planes,
        # bound by instruction issue and shared-memory/shuffle traffic, not
        # HBM: reported against the FP32 peak from unit counts and the clock
        # sampled during the timed steps
        sm_mhz = clocks.get("sm_mhz") or 2032.0
        flops = fft_smoothing_flops(prm["mesh"])
        launch_us = stage_us["smooth"] / 3.0
        achieved = flops / 3.0 / (launch_us * 1e-6) / 1e12
        peak = fp32_peak_tflops(sm_mhz)
        roofline = {"bound": "alu", "kernel": "k_fht_xy / k_fht_z (spectral smoothing by FFT, three launches)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": recorded_traffic("k_fht_xy", WORKLOAD, args.precision),
                    "peak_source": f"FP32 units: 148 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz",
                    "algorithmic_flops_per_launch": flops / 3.0, "launch_us": launch_us}
    else:
        bytes_per_launch, launches_per_step = algorithmic_bytes(dom, b, P3, system.n, K_smooth, fuse,
                                                                pred_used)
        launch_us = stage_us[dom] / launches_per_step
        achieved = bytes_per_launch / (launch_us * 1e-6) / 1e9
        if dom == "smooth":
            kernel = (f"k_diffuse_tq ({fuse} steps per launch)" if fuse in (3, 4) else
                      "k_diffuse_cluster" if fuse == 5 else "k_diffuse4x2" if fuse == 2 else
                      "k_diffuse4" if args.precision == "mixed" else "k_diffuse")
        else:
            kernel = STAGE_KERNEL[dom][0 if args.precision == "mixed" else 1]
        roofline = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": recorded_traffic(kernel, WORKLOAD, args.precision),
                    "peak_source": peaks["source"], "algorithmic_bytes_per_launch": bytes_per_launch,
                    "launch_us": launch_us}
    line = {
        "metric": METRIC, "value": value, "unit": "ns/day", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": DATA,
        "config": workload_config(prm),
        "settings": {"precision": args.precision, "graphs": not args.no_graphs, "tuning": tuning,
                     "start": f"seeded random configuration equilibrated {args.equilibrate} steps at 1200 K "
                              "(velocity rescaling), untimed"},
        "lr_step_us": sum(stage_us[k] for k in lr_stages),
        "stage_us": stage_us, "mg_iters_per_step": iters,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
        "ms_per_step_with_stage_events": sum(ms_staged) / args.steps,
        "ms_per_step_l2_flushed": max_over_ranks(sum(ms_flushed), world, device="cuda") / args.steps,
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "variants": variants,
        "accuracy_vs_oracle": accuracy,
        "roofline_alone": {
            "kernel": "k_diffuse4 (one diffusion step per launch, 2 planes per thread, nothing beside it)",
            "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
            "achieved": 2.0 * P3 * b / (alone_launch_us * 1e-6) / 1e9,
            "frac": 2.0 * P3 * b / (alone_launch_us * 1e-6) / 1e9 / peaks["hbm_gbs"],
            "launch_us": alone_launch_us, "algorithmic_bytes_per_launch": 2.0 * P3 * b,
            "traffic": recorded_traffic("k_diffuse4", WORKLOAD, args.precision),
            "note": "the two 8 MB FP32 meshes stay in L2 at 128^3; the HBM-bound sizes are in "
                    "bench.py --sweep (k_diffuse4_alone)"},
    }
    if not args.no_serve:
        line["served"] = served_run(stream.cuda_stream, n_req=256, steps=200, slots=16)
        # the same stream of requests with every member launching its own
        # diffusion kernels (no shared cluster smoothing), for comparison
        line["served_per_step_smoothing"] = served_run(stream.cuda_stream, n_req=256, steps=200, slots=16,
                                                       smoothing="per_step")
    if not args.no_serve:
        line["batch_small"] = batch_small_run(stream, peaks)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(system, prm)
    print(json.dumps(line))
    return 0


def small_batch_bytes(mesh: int, n_atoms: int, iters: float) -> float:
    """Algorithmic bytes of one mixed-precision MD step of a member: each
    mesh array read or written once per pass that needs it, FP32 meshes 4 B
    and fixed-point meshes 8 B per point, particles 4 B per coordinate.  Per
    mesh point: assignment output 4, smoothing in + out 8, prediction and
    residual 64, per V-cycle about 100 (sweeps 8 + 24, restriction and
    prolongation 8.5 each, residual update 44, coarser levels 1/7 more),
    field update 56, interpolation input 4.  Per particle: kick/drift 120,
    cell list 32, assignment 32, pair forces 32, interpolation 104."""
    P3 = float(mesh) ** 3
    return P3 * (4 + 8 + 64 + 100.0 * iters + 56 + 4) + n_atoms * (120 + 32 + 32 + 32 + 104)


def batch_small_run(stream, peaks, members: int = 32, steps: int = 60, warmup: int = 6) -> dict:
    """Many small systems (16^3-64^3 meshes) advanced as one batch: system-
    steps/s of eight batch configurations -- one graph for the whole batch or
    each member's own cached graphs, each with the smoothing of every member
    in one cluster launch per cluster size (cluster_fused), each member's
    smoothing in its own cluster launch (cluster_own), each member's own
    per-step diffusion launches (per_step), or each member's smoothing in the
    Hartley basis (spectral).  The same seeded members in every
    configuration."""
    import torch
    from paper_2606_31379_b300 import p3maze as P
    from paper_2606_31379_b300.serve import Request, request_system

    rng = np.random.default_rng(11)
    reqs = []
    for i in range(members):
        kind = "nacl" if i % 2 == 0 else "water"
        atoms = int(round(math.exp(rng.uniform(math.log(216), math.log(4096)))))
        reqs.append(Request(rid=i, kind=kind, n_atoms=atoms, seed=2000 + i, steps=steps, arrival=0.0))
    systems = [request_system(r) for r in reqs]
    out = {"config": {"members": members, "steps": steps, "warmup": warmup,
                      "sizes": "216-4096 atoms log-uniform, molten NaCl / SPC/Fw alternating, mesh ~0.8 A",
                      "meshes": sorted({p["mesh"] for _, p in systems}), "precision": "mixed"}}
    ref_F = None
    for mode in ("shared", "per_member"):
        for smoothing in ("cluster_fused", "cluster_own", "per_step", "spectral"):
            ctxs = []
            batch = P.Batch(stream=stream.cuda_stream, mode=mode, fused_smoothing=smoothing == "cluster_fused")
            try:
                n_atoms = 0
                for system, prm in systems:
                    c = P.Context.from_system(system, precision="mixed", **prm)
                    if prm["mesh"] <= 64:  # every member here; the default is the spectral mode
                        if smoothing == "per_step":
                            c.set_tuning(diffusion_fuse=2 if prm["mesh"] % 4 == 0 else 1, diffusion_zc=2)
                        elif smoothing.startswith("cluster"):
                            c.set_tuning(diffusion_fuse=5)
                    ctxs.append(c)
                    n_atoms += system.n
                for c in ctxs:
                    batch.add(c)
                with torch.cuda.stream(stream):
                    batch.step(warmup)
                    batch.wait()
                    it0 = [c.stats()["total_iters"] for c in ctxs]
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    batch.step(steps)
                    e1.record(stream)
                    batch.wait()
                    torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) * 1e-3
                iters = [(c.stats()["total_iters"] - i0) / steps for c, i0 in zip(ctxs, it0)]
                algo = sum(small_batch_bytes(p["mesh"], s.n, it) for (s, p), it in zip(systems, iters)) * steps
                F = np.concatenate([c.forces() for c in ctxs])
                rec = {"system_steps_per_s": members * steps / sec, "ms_per_batch_step": 1e3 * sec / steps,
                       "atom_steps_per_s": n_atoms * steps / sec,
                       "mg_iters_per_step": float(np.mean(iters)),
                       "algorithmic_GBps": algo / sec / 1e9,
                       "hbm_frac": algo / sec / 1e9 / peaks["hbm_gbs"]}
                if ref_F is None:
                    ref_F = F
                else:  # all four advance the same members the same number of steps
                    rec["force_rel_rms_vs_first"] = float(np.sqrt(np.mean((F - ref_F) ** 2) / np.mean(ref_F ** 2)))
                out[f"{mode}_{smoothing}"] = rec
            finally:
                batch.close()
                for c in ctxs:
                    c.close()
    # one context alone: the whole smoothing in one cluster launch or per-step launches
    alone = {}
    for atoms in (512, 1728, 4096):
        system, prm = request_system(Request(rid=0, kind="nacl", n_atoms=atoms, seed=77, steps=0, arrival=0.0))
        rec = {"mesh": prm["mesh"]}
        for smoothing in ("cluster", "per_step", "spectral"):
            with P.Context.from_system(system, precision="mixed", stream=stream.cuda_stream, **prm) as c:
                if smoothing == "per_step":
                    c.set_tuning(diffusion_fuse=2 if prm["mesh"] % 4 == 0 else 1, diffusion_zc=2)
                elif smoothing == "cluster":
                    c.set_tuning(diffusion_fuse=5)
                c.step(warmup)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                c.step(steps)
                e1.record(stream)
                torch.cuda.synchronize()
                c.set_timing(True)
                c.step(steps)
                rec[smoothing] = {"ms_per_step": e0.elapsed_time(e1) / steps,
                                  "smooth_us_per_step": 1e3 * c.timing()["ms"]["smooth"] / steps}
        alone[f"nacl_{atoms}"] = rec
    out["alone"] = alone
    out["note"] = ("hbm_frac: algorithmic bytes of every member's step (small_batch_bytes) over the batch "
                   "time, of measured HBM bandwidth; meshes this small stay in L2, so the steps are bound by "
                   "launch latency and the fraction measures how well the batch fills the GPU")
    return out


def served_run(stream, n_req: int, steps: int, slots: int, rate: float = 200.0, smoothing: str = "default") -> dict:
    """The served-batch workload: n_req requests with Poisson arrivals,
    molten NaCl or SPC/Fw (50/50), 216-32768 atoms log-uniform, mesh ~0.8 A,
    each advanced `steps` steps, admitted by device memory into `slots`
    slots.  smoothing="default": members of at most 64^3 are smoothed by one
    cluster launch per batch step; "per_step": every member launches its own
    diffusion kernels (the comparison)."""
    from paper_2606_31379_b300.serve import GpuBackend, Server, poisson_requests
    reqs = poisson_requests(n_req, rate=rate, seed=4, steps=steps)
    be = GpuBackend(precision="mixed", stream=stream, smoothing=smoothing)
    try:
        m = Server(be, budget_bytes=60 << 30, max_slots=slots).run(reqs)
    finally:
        be.shutdown()
    m["config"] = {"requests": n_req, "arrival_rate_per_s": rate, "steps_per_request": steps, "slots": slots,
                   "sizes": "216-32768 atoms log-uniform, molten NaCl / SPC/Fw 50:50, mesh ~0.8 A",
                   "precision": "mixed", "start": "seeded random configurations", "smoothing": smoothing}
    return m


SWEEP = [("nacl_4k", 4096, 50.45, 64), ("nacl_32k", 32768, 100.9, 128), ("nacl_262k", 262144, 201.8, 256),
         ("nacl_580k", 580000, 263.0, 320), ("nacl_1m", 1000000, 315.4, 384)]


def run_sweep(args) -> int:
    """Linear-scaling sweep of molten NaCl (and the SPC/Fw workload): one JSON
    line per size with per-stage time, V-cycles per step and the smoothing
    kernel's algorithmic bandwidth."""
    import torch
    from paper_2606_31379_b300 import p3maze as P
    from paper_2606_31379_b300 import synth as S

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peaks = measured_peaks()
    only = set(args.sweep_cases.split(",")) if args.sweep_cases else None
    cases = [(name, S.nacl_melt(n, box, seed=5 + i), mesh, 1.0)
             for i, (name, n, box, mesh) in enumerate(SWEEP)
             if (args.sweep_max is None or n <= args.sweep_max) and (only is None or name in only)]
    if not args.no_water and (only is None or "spcfw_30k" in only):
        cases.append(("spcfw_30k", S.spcfw_water(30000, 96.4, seed=3), 128, 0.5))
    for name, system, mesh, dt in cases:
        kw = dict(alpha=S.EWALD_ALPHA, r_cut=S.R_CUT, mesh=mesh, tol=S.TOL, dt=dt, precision=args.precision,
                  stream=stream.cuda_stream)
        with P.Context.from_system(system, **kw) as eq:
            eq.equilibrate(args.equilibrate, 1200.0 if system.sr_kind == "bmh" else 298.15)
            system.pos, system.vel = eq.positions(), eq.velocities()
        with P.Context.from_system(system, **kw) as ctx:
            if args.no_graphs:
                ctx.set_graphs(False)
            ctx.step(args.warmup)
            if args.tuning:
                ctx.set_tuning(**json.loads(args.tuning))
                tuning = dict(ctx.tuning(), source="--tuning")
            else:
                tuning = ctx.autotune(12)
            ctx.step(max(args.warmup, 4))  # record the step graphs of the final setting untimed
            ctx.set_timing(True)
            it0 = ctx.stats()["total_iters"]
            ms = time_context(ctx, torch, stream, args.steps, flush)
            tm = ctx.timing()
            st = ctx.stats()
            # the one-step diffusion kernel alone: one launch per step, 4
            # planes per thread, pair branch forked after smoothing so that
            # nothing runs beside it
            ctx.set_tuning(diffusion_fuse=1, diffusion_zc=4, pair_fork=0)
            ctx.set_timing(True)
            ctx.step(2)
            ctx.set_timing(True)
            time_context(ctx, torch, stream, max(3, args.steps // 2), flush)
            iso_us = 1e3 * ctx.timing()["ms"]["smooth"] / max(3, args.steps // 2)
        stage_us = {k: 1e3 * v / args.steps for k, v in tm["ms"].items()}
        b = 4 if args.precision == "mixed" else 8
        K = st["smooth_steps"]
        # algorithmic bytes: each smoothing launch reads and writes the mesh once
        nl = smoothing_launches(K, tuning.get("diffusion_fuse", 1))
        smooth_gbs = 2.0 * mesh ** 3 * b * nl / (stage_us["smooth"] * 1e-6) / 1e9
        ms_step = sum(ms) / args.steps
        print(json.dumps({
            "workload": name, "n_particles": system.n, "mesh": mesh, "ms_per_step": ms_step,
            "ns_per_day": ns_per_day(ms_step * 1e-3, dt), "mg_iters_per_step": (st["total_iters"] - it0) / args.steps,
            "stage_us": stage_us, "smooth_steps": K, "smooth_launches": nl,
            "smooth_us_per_launch": stage_us["smooth"] / nl, "smooth_algorithmic_gbs": smooth_gbs,
            "k_diffuse4_alone": {"us_per_launch": iso_us / K,
                                 "gbs": 2.0 * mesh ** 3 * b * K / (iso_us * 1e-6) / 1e9,
                                 "frac_of_hbm_peak": 2.0 * mesh ** 3 * b * K / (iso_us * 1e-6) / 1e9
                                 / peaks["hbm_gbs"]},
            "smooth_frac_of_hbm_peak": smooth_gbs / peaks["hbm_gbs"],
            "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": peaks["source"], "tuning": tuning,
            "device_bytes": st["device_bytes"], "precision": args.precision,
        }), flush=True)
    return 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-budget", type=float, default=120.0,
                    help="seconds of timed oracle work in --impl reference (whole steps, at least one)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle check of the timed states")
    ap.add_argument("--no-tune", action="store_true", help="skip the solver-setting autotuner")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-batch measurement")
    ap.add_argument("--tuning", type=str, default=None,
                    help='apply this solver setting instead of autotuning, e.g. \'{"diffusion_fuse": 2}\'')
    ap.add_argument("--sweep", action="store_true",
                    help="linear-scaling sweep (4096 to 1e6 ions) and SPC/Fw 90000 atoms, one line per size")
    ap.add_argument("--sweep-max", type=int, default=None)
    ap.add_argument("--sweep-cases", type=str, default=None, help="comma-separated subset of the sweep")
    ap.add_argument("--no-water", action="store_true")
    ap.add_argument("--equilibrate", type=int, default=400,
                    help="untimed velocity-rescaled steps at 1200 K before any measurement")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel eagerly (profiling: ncu does not list kernels of graph while nodes)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
