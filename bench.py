"""Benchmark of the GB300 HLBM time step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload hindered_settling|single_sphere|nonspherical|dense_batch]

A step is one full HLBM time step (momentum exchange, external force,
Newton-Euler update, particle work lists, EDM coupling, collision and
streaming) over the whole lattice.  The metric is MLUPS including the particle
coupling: cells x steps / seconds / 1e6, summed over all GPUs (N > 1 runs N
independent replicas, one per GPU: weak scaling, no data-path collective).

Default workload: hindered settling, 128^3 cells, walls at z = 0 / 127,
periodic x and y, 200 spheres r ~ U(4, 8), density ratio 2.5, tau 0.6,
g = 1e-5, FP32 storage of f - w.  Its 19 FP32 planes (159 MB) exceed the
126 MB L2, so the FP32 steps run back to back; the FP16 variant (80 MB) is
timed one step at a time with a 512 MB L2 flush between steps.

The JSON line adds: roofline (collision kernel, algorithmic bytes over its
CUDA-event time), step_roofline (the whole step's bytes with and without the
momentum exchange's per interior cell, against the step time, and the MLUPS
rooflines they give), coupling (interior cells per step, momentum-exchange
cell updates and particles per second), cpu_baseline (the FP64 oracle on
the host), e2e (the same
metric through the C-ABI with pinned host buffers copied every step), clocks,
gpu_launches, fp16 (the FP16-storage run and its error against FP32), and
nonspherical: the 256^3 box of 2000 ellipsoids and cuboids with FP32 and FP16
storage; batched_fp16: the large dense batch (512 x 512 x 1024 cells, 50 000 spheres)
with FP32 and with FP16 storage, its collision roofline and the FP16 error;
ensemble: 64 independent boxes of 64..96^3 advanced together, FP32 (its fp16
entry: the same with FP16 storage).
Opt-in legs: --capsules (the non-spherical box with 2000 capsules),
--grid-shapes (the same box with 2000 signed-distance grid particles),
--phi-matched, --settling-validation.

--impl reference times the FP64 CPU oracle (the reference arm of this
repository) on the same workload, rank 0 only.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = {"fp32": 2 * 19 * 4, "fp16": 2 * 19 * 2}


WORKLOADS = ("hindered_settling", "single_sphere", "nonspherical", "dense_batch", "fluid_256",
             "dense_batch_256", "nonspherical_phi", "dense_batch_phi", "capsules", "grid_shapes")


def make_workload(name):
    """The benchmark workloads; the two 256^3 ones are smaller stand-ins used
    for profiling (no particles; the 50 000-sphere density on 256^3)."""
    from paper_2312_14172_gb300 import workloads
    if name == "hindered_settling":
        return workloads.hindered_settling()
    if name == "single_sphere":
        return workloads.single_sphere()
    if name == "nonspherical":
        return workloads.nonspherical()
    if name == "dense_batch":
        return workloads.dense_batch()
    if name == "fluid_256":
        return workloads.dense_batch(n=(256, 256, 256), count=0)
    if name == "dense_batch_256":
        return workloads.dense_batch(n=(256, 256, 256), count=50000 * 256 ** 3 // (512 * 512 * 1024))
    if name == "nonspherical_phi":
        return workloads.nonspherical_phi_matched()
    if name == "dense_batch_phi":
        return workloads.dense_batch_phi_matched()
    if name == "capsules":
        return workloads.nonspherical(kinds=(workloads.CAPSULE,), name="capsules")
    if name == "grid_shapes":
        return workloads.grid_shapes()
    raise SystemExit(f"unknown workload {name}")


def l2_note(prec, cells):
    """How the timed steps meet L2: the library takes odd steps' bricks in
    reverse order when the populations are within twice the L2, so those
    steps start on populations the step before left there."""
    import torch
    pop = BYTES_PER_CELL[prec] // 2 * cells
    note = f"inputs larger than L2 ({pop / 1e6:.0f} MB of populations); no flush between steps"
    try:
        l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    except Exception:
        l2 = 0
    if l2 and pop <= 2 * l2:
        note += (f"; within twice the {l2 / 1e6:.0f} MB L2, so odd steps take the bricks in reverse order "
                 "and start on populations the previous step left in L2 (traffic: ncu, cold cache)")
    return note


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text):
    """C++ source without its comments and blank lines (a comment does not
    change the kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash(cells_x=2):
    """Hash of the code (comments left out) that defines the collision kernel
    with cells_x cells per thread (a committed ncu figure holds only for the
    same code)."""
    h = hashlib.sha256()
    main = "lbm_pair_kernels.cu" if cells_x == 2 else "lbm_kernels.cu"
    for f in (main, "lbm_common.cuh", "hlbm_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2312_14172_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload, precision, cells, cells_x):
    """DRAM bytes per collision launch from a committed ncu summary, if it was
    taken on the current kernel source with the same cells per thread; else
    None."""
    path = os.path.join(ROOT, "profiles", f"collide_stream_{workload}_{precision}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_source_hash") != kernel_source_hash(cells_x) or d.get("cells_per_thread", 1) != cells_x:
        return None
    per_cell = d.get("dram_bytes_per_cell")
    return None if per_cell is None else per_cell * cells


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml of the NVIDIA driver):
    SM clock, its maximum and the active clock-event reasons of one GPU."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, device):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device).uuid)
            uuid = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            uuid = None
        if uuid is None or self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.dev)) != 0:
            if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device), ctypes.byref(self.dev)) != 0:
                raise OSError("no NVML handle")
        get = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.get_reasons = get or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(v))
        self.max_mhz = float(v.value)

    def sample(self):
        v = self.ct.c_uint(0)
        r = self.ct.c_ulonglong(0)
        if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, self.ct.byref(v)) != 0:
            return None
        self.get_reasons(self.dev, self.ct.byref(r))
        return float(v.value), [nm for bit, nm in self.REASONS.items() if r.value & bit]


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed window:
    NVML queried in a thread as fast as it answers (tens of samples even in a
    window of a few milliseconds), else nvidia-smi every 10 ms (the nearest
    two samples when the window is shorter than that interval)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.window = None
        self.nvml = None
        self.rows = []
        self.thread = None
        self.halt = False

    def start(self):
        try:
            self.nvml = _Nvml(self.device)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            import threading

            def run():
                while not self.halt:
                    s = self.nvml.sample()
                    if s is not None:
                        self.rows.append((time.perf_counter(), s[0], self.nvml.max_mhz, s[1]))
                    time.sleep(0.0002)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def mark(self, t0, t1, wall0, wall1):
        """bounds of the timed region: time.perf_counter() values t0, t1
        (NVML samples) and time.time() values wall0, wall1 (nvidia-smi)"""
        self.window = (t0, t1, wall0, wall1)

    def _smi_rows(self):
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             [nm for nm, v in zip(names, parts[4:8]) if v.lower().startswith("active")]))
            except ValueError:
                continue
        return rows

    def stop(self):
        if self.thread is not None:
            self.halt = True
            self.thread.join(timeout=5)
            rows, source = list(self.rows), "nvml"
            window = (self.window[0], self.window[1]) if self.window else None
        elif self.proc is not None:
            rows, source = self._smi_rows(), "nvidia-smi"
            window = (self.window[2], self.window[3]) if self.window else None
        else:
            return None
        if not rows:
            return None
        sel = rows
        if window is not None:
            t0, t1 = window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            sel = inside if inside else sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:2]
        reasons = sorted({nm for r in sel for nm in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": sel[0][2], "reasons": reasons,
                "samples": len(sel), "source": source, "in_window": bool(window and any(
                    window[0] <= r[0] <= window[1] for r in rows))}


# D3Q19 velocities in the library's order (include/hlbm.h)
C19 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], float)


def _rel(got, ref, axis=None):
    """max |got - ref| / max |ref| (vectors by their length when axis is
    given) and the L2 relative error ||got - ref|| / ||ref||."""
    d, r = np.asarray(got, float) - ref, np.asarray(ref, float)
    if axis is not None:
        d, r = np.linalg.norm(d, axis=axis), np.linalg.norm(r, axis=axis)
    rmax, rl2 = float(np.abs(r).max()), float(np.sqrt((r * r).sum()))
    return {"max": float(np.abs(d).max()) / rmax if rmax > 0 else float(np.abs(d).max()),
            "l2": float(np.sqrt((d * d).sum())) / rl2 if rl2 > 0 else float(np.sqrt((d * d).sum()))}


def state_errors(ref, got, n, bc, X0, coupling=None):
    """Per-quantity error of a run `got` against a reference run `ref` after
    the same steps, each a dict with populations f [19, nz, ny, nx] (FP64
    values f_i) and the particle state of particle_state().  Returns for
    each quantity {"max", "l2"} (see _rel):
      rho    density, relative to rho itself;
      p      density deviation rho - 1 (the pressure fluctuation over c_s^2),
             relative to the reference's deviation;
      u      fluid velocity sum_i c_i f_i / rho, relative to the largest speed;
      u_out  the macroscopic velocity of the exact-difference forcing,
             u + B (u_p - u) / 2 (when coupling = (B, pid) gives the
             indicator field and its particle per cell; each run's own
             particle state gives u_p(x) = U + omega x (x - X));
      F, T   hydrodynamic force and torque per particle (vector lengths);
      X      displacement X - X0 (minimum image on periodic axes);
      U, omega  particle velocities.
    Pure numpy: the callers supply both runs."""
    L = np.asarray(n, float)
    per = np.array([not (bc >> j) & 1 for j in range(3)])
    out = {}
    moments = {}
    for key, run in (("ref", ref), ("got", got)):
        f = run["f"]
        rho = f.sum(0)
        moments[key] = (rho, np.einsum("ai,izyx->azyx", C19, f) / rho)
    (r_ref, u_ref), (r_got, u_got) = moments["ref"], moments["got"]
    out["rho"] = _rel(r_got, r_ref)
    out["p"] = _rel(r_got - 1.0, r_ref - 1.0)
    out["u"] = _rel(u_got, u_ref, axis=0)
    if coupling is not None:
        B, pid = coupling
        zz, yy, xx = np.nonzero(pid >= 0)
        sh = {}
        for key, run, u in (("ref", ref, u_ref), ("got", got, u_got)):
            st = run["state"]
            p = pid[zz, yy, xx]
            r = np.stack([xx, yy, zz], 1) - st["X"][p]
            r -= np.where(per, L * np.round(r / L), 0.0)
            up = st["U"][p] + np.cross(st["omega"][p], r)
            us = u.copy()
            b = B[zz, yy, xx][:, None]
            us[:, zz, yy, xx] = (u[:, zz, yy, xx].T + 0.5 * b * (up - u[:, zz, yy, xx].T)).T
            sh[key] = us
        out["u_out"] = _rel(sh["got"], sh["ref"], axis=0)
    sr, sg = ref["state"], got["state"]
    if len(sr["X"]):
        for key in ("F", "T", "U", "omega"):
            out[key] = _rel(sg[key], sr[key], axis=1)
        dr, dg = sr["X"] - X0, sg["X"] - X0
        dr -= np.where(per, L * np.round(dr / L), 0.0)
        dg -= np.where(per, L * np.round(dg / L), 0.0)
        out["X"] = _rel(dg, dr, axis=1)
    return out


def oracle_mlups(w, steps, warmup=0, omp=False, keep=False):
    """FP64 oracle on the workload (single thread, or its OpenMP build on all
    host cores): MLUPS and seconds (and the oracle itself when keep)."""
    from oracle import oracle
    oracle.build(omp=omp)
    o = oracle.from_workload(w, omp=omp)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = w["n"][0] * w["n"][1] * w["n"][2]
    if keep:
        return cells * steps / dt / 1e6, dt, o
    o.close()
    return cells * steps / dt / 1e6, dt


def error_vs_fp64(w, o, steps):
    """The full workload on the GPU with FP32 and with FP16 storage for the
    same steps as the timed oracle o took from the same initial state: the
    error of each quantity against that FP64 state (state_errors)."""
    from paper_2312_14172_gb300 import hlbm
    ref = {"f": o.populations(), "state": o.particle_state()}
    coupling = o.indicator_field()
    out = {"steps": steps, "mea_mode": "moments"}
    for prec in ("fp32", "fp16"):
        lat = hlbm.from_workload(w, precision=prec)
        lat.set_mea_mode("moments")
        lat.step(steps)
        got = {"f": lat.populations(), "state": lat.particle_state()}
        lat.close()
        out[prec] = state_errors(ref, got, w["n"], w["bc"], w["particles"]["X"], coupling=coupling)
    return out


def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def max_over_ranks(v):
    """The largest of one value over all ranks (the value itself on one rank):
    whole-job times are the slowest replica's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells, steps, ms, ws):
    """MLUPS of ws replicas of `cells` cells that took `ms` (max over ranks)."""
    return ws * cells * steps / (ms / 1e3) / 1e6


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    w = make_workload(args.workload)
    cells = w["n"][0] * w["n"][1] * w["n"][2]
    # bound the run: at most ~120 s of timed oracle work
    probe_mlups, probe_dt = oracle_mlups(w, 1)
    per_step = probe_dt
    steps = max(1, min(args.steps, int(120.0 / max(per_step, 1e-3))))
    warm = min(args.warmup, max(0, int(30.0 / max(per_step, 1e-3))))
    mlups, dt = oracle_mlups(w, steps, warmup=warm)
    sample = (f"{steps} timed step(s) after {warm} warm-up step(s) of the full "
              f"{w['n'][0]}x{w['n'][1]}x{w['n'][2]} workload ({len(w['particles']['shape'])} particles)")
    return {
        "impl": "reference", "metric": "MLUPS incl. particle coupling", "value": mlups, "unit": "MLUPS",
        "n_gpus": ws, "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "cells": cells,
                                        "particles": len(w["particles"]["shape"])},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_gpu(args, ws, rank, local):
    import torch
    from paper_2312_14172_gb300 import build, hlbm
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    torch.cuda.set_device(local)
    build.build()
    hlbm.load()
    dist = None
    if ws > 1:
        import torch.distributed as dist
    w = make_workload(args.workload)
    prec = args.precision or w["precision"]
    cells = w["n"][0] * w["n"][1] * w["n"][2]
    npart = len(w["particles"]["shape"])
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- main timed region: K graph-launched steps, inputs resident in HBM
    lat = hlbm.from_workload(w, precision=prec, stream=stream)
    tune = None
    if args.autotune:
        tune = lat.autotune(nsteps=5)
    if args.mea_mode:
        lat.set_mea_mode(args.mea_mode)
    if args.launch:
        lat.set_launch(*[int(v) for v in args.launch.split(",")])
    mea_mode = lat.get_mea_mode()
    lat.step(args.warmup)
    lat.sync()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    t_host0, t_wall0 = time.perf_counter(), time.time()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_host1, t_wall1 = time.perf_counter(), time.time()
    barrier()
    sampler.mark(t_host0, t_host1, t_wall0, t_wall1)
    clocks = sampler.stop()
    lat.sync()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms)
    value = whole_job_mlups(cells, args.steps, ms, ws)

    lat_launch = lat.get_launch()
    # ---- per-kernel CUDA-event times on the same stream (roofline)
    kt = lat.kernel_times(nsteps=max(5, min(args.steps, 50)))
    peak, peak_kind = measured_peaks()
    k1_ms = kt["collide_stream"]
    algo_bytes = BYTES_PER_CELL[prec] * cells
    achieved = algo_bytes / (k1_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.workload, prec, cells, lat_launch[2])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "kernel": "collide_pair_kernel" if lat_launch[2] == 2 else "collide_stream_kernel",
                "algorithmic_bytes": algo_bytes,
                "kernel_ms": k1_ms, "kernel_ms_mea": kt["mea"], "kernel_ms_update": kt["update"]}

    coupling, step_roofline = coupling_and_step_roofline(lat, cells, npart, args.steps, ms, ws, prec, peak)

    # ---- end to end through the C-ABI with pinned host buffers
    st0 = lat.particle_state()
    pin = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy() for k, v in st0.items()}
    for k in pin:
        pin[k][...] = st0[k]
    e2e_steps = max(3, min(args.steps, 200))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_particle_state(pin["X"], pin["U"], pin["omega"], pin["quat"])
        lat.step(1)
        lat.particle_state(out=pin)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    barrier()
    # the same loop for a caller that moves the particles itself every step
    # (positions written back changed): every step then takes the
    # bounding-box momentum exchange
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pin["X"][:, 0] += 1e-9
        lat.set_particle_state(pin["X"], pin["U"], pin["omega"], pin["quat"])
        lat.step(1)
        lat.particle_state(out=pin)
    torch.cuda.synchronize()
    t_moved = max_over_ranks(time.perf_counter() - t0)
    barrier()
    e2e = {"value": whole_job_mlups(cells, e2e_steps, t_e2e * 1e3, ws), "unit": "MLUPS",
           "h2d_bytes_per_step": npart * 13 * 8, "d2h_bytes_per_step": npart * 19 * 8 + 4,
           "steps": e2e_steps,
           "note": "per step: hlbm_set_particle_state (X, U, omega, q) + hlbm_step(1) + "
                   "hlbm_particle_state (X, U, omega, q, F, T), pinned host arrays; the state written back "
                   "is the one just read, so the step keeps the momentum exchange from the recorded moments",
           "moved": {"value": whole_job_mlups(cells, e2e_steps, t_moved * 1e3, ws), "unit": "MLUPS",
                     "note": "the same loop with every position written back changed (by 1e-9 cells): "
                             "each step takes the bounding-box momentum exchange; the figure for a caller "
                             "that moves its particles itself"}}
    # state after the runs, for the FP16 comparison
    fp32_state = lat.particle_state()
    fp32_steps = lat.steps_done
    f32 = lat.populations() if cells <= 4_000_000 else None
    lat.close()

    # ---- FP16 storage on the same workload, L2 flushed between steps
    fp16 = None
    if args.fp16 and prec == "fp32":
        lat16 = hlbm.from_workload(w, precision="fp16", stream=stream)
        if args.autotune:
            lat16.autotune(nsteps=5)
        if args.mea_mode:
            lat16.set_mea_mode(args.mea_mode)
        if args.launch:
            lat16.set_launch(*[int(v) for v in args.launch.split(",")])
        lat16.step(args.warmup)
        lat16.sync()
        flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            lat16.step(1)
            b.record(stream)
        torch.cuda.synchronize()
        lat16.sync()
        ms16 = sum(a.elapsed_time(b) for a, b in evs)
        ms16 = max_over_ranks(ms16)
        kt16 = lat16.kernel_times(nsteps=max(5, min(args.steps, 50)))
        cx16 = lat16.get_launch()[2]
        ach16 = BYTES_PER_CELL["fp16"] * cells / (kt16["collide_stream"] / 1e3) / 1e9
        # error against FP32 after the same number of steps
        rest = fp32_steps - lat16.steps_done
        if rest > 0:
            lat16.step(rest)
        s16 = lat16.particle_state()
        err = {}
        X0 = w["particles"]["X"]
        for key in ("X", "U", "F", "T"):
            a32 = fp32_state[key] - (X0 if key == "X" else 0)
            a16 = s16[key] - (X0 if key == "X" else 0)
            scale = float(np.abs(a32).max()) or 1.0
            err[key] = float(np.abs(a16 - a32).max() / scale)
        if f32 is not None:
            f16 = lat16.populations()
            c = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                          [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                          [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], float)
            r32, r16 = f32.sum(0), f16.sum(0)
            u32 = np.einsum("ai,izyx->azyx", c, f32) / r32
            u16 = np.einsum("ai,izyx->azyx", c, f16) / r16
            err["rho"] = float(np.abs(r16 - r32).max())
            err["u"] = float(np.abs(u16 - u32).max() / max(np.abs(u32).max(), 1e-30))
        lat16.close()
        fp16 = {"value": whole_job_mlups(cells, args.steps, ms16, ws), "unit": "MLUPS",
                "ms_per_step": ms16 / args.steps, "l2": "512 MB flush between steps",
                "roofline": {"bound": "hbm", "achieved": ach16, "peak": peak, "unit": "GB/s",
                             "frac": ach16 / peak, "kernel_ms": kt16["collide_stream"],
                             "traffic": profiled_traffic(args.workload, "fp16", cells, cx16)},
                "error_vs_fp32": err,
                "error_note": "max |fp16 - fp32| / max|fp32| after the same steps; X as displacement; "
                              "rho absolute; FP32 itself matches the FP64 oracle within 1e-5"}

    nonsph = nonspherical_leg(args, stream, peak, ws) if args.nonspherical else None
    batched = batched_fp16_leg(args, stream, peak, ws) if args.batched else None
    ensemble = ensemble_leg(args, stream, peak, ws) if args.ensemble else None
    if ensemble is not None and args.fp16:
        ensemble["fp16"] = ensemble_leg(args, stream, peak, ws, "fp16")
    phi = phi_matched_leg(args, stream, peak, ws) if args.phi_matched else None
    settling = settling_validation_leg(args, stream) if args.settling_validation else None
    capsules = capsules_leg(args, stream, peak, ws) if args.capsules else None
    grids = grid_shapes_leg(args, stream, peak, ws) if args.grid_shapes else None

    launches_per_step = 3 if npart > 0 else 1
    line = {
        "metric": "MLUPS incl. particle coupling", "value": value, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "cells": cells, "dims": list(w["n"]), "particles": npart,
                   "storage": prec, "tau": w["tau"], "eps": w["eps"], "bc": w["bc"],
                   "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu",
                   "l2": l2_note(prec, cells),
                   "launch": {"tile_y": lat_launch[0], "tile_z": lat_launch[1],
                              "cells_per_thread": lat_launch[2],
                              "momentum_exchange": mea_mode,
                              "autotuned": bool(args.autotune)}},
        "roofline": roofline,
        "step_roofline": step_roofline,
        "coupling": coupling,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "fp16": fp16,
        "nonspherical": nonsph,
        "batched_fp16": batched,
        "ensemble": ensemble,
    }
    if phi is not None:
        line["phi_matched"] = phi
    if settling is not None:
        line["settling_validation"] = settling
    if capsules is not None:
        line["capsules"] = capsules
    if grids is not None:
        line["grid_shapes"] = grids
    return line


def ensemble_leg(args, stream, peak, ws, prec="fp32"):
    """The batched ensemble: 64 independent periodic boxes of 64..96^3 cells,
    10..200 spheres each, all advanced by one captured graph per step with
    the autotuned launch shape, FP32 or FP16 storage (2.4 GB / 1.2 GB of
    populations)."""
    import torch
    from paper_2312_14172_gb300 import hlbm, workloads
    boxes = workloads.ensemble()
    cells = sum(b["n"][0] * b["n"][1] * b["n"][2] for b in boxes)
    npart = sum(len(b["particles"]["shape"]) for b in boxes)
    params = hlbm.make_params(tau=boxes[0]["tau"], eps=boxes[0]["eps"], gravity=boxes[0]["gravity"],
                              max_particles=npart, precision=prec)
    lat = hlbm.Lattice([tuple(b["n"]) + (b["bc"],) for b in boxes], params, stream=stream)
    for k, b in enumerate(boxes):
        lat.add_workload_particles(b["particles"], box_id=[k] * len(b["particles"]["shape"]))
    if args.autotune:
        lat.autotune(nsteps=5)
    elif args.mea_mode:
        lat.set_mea_mode(args.mea_mode)
    lat.step(args.warmup)
    lat.sync()
    steps = max(1, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    lat.sync()
    ms = max_over_ranks(e0.elapsed_time(e1))
    kt = lat.kernel_times(nsteps=10)
    ach = BYTES_PER_CELL[prec] * cells / (kt["collide_stream"] / 1e3) / 1e9
    out = {"value": whole_job_mlups(cells, steps, ms, ws), "unit": "MLUPS", "ms_per_step": ms / steps,
           "storage": prec, "steps": steps, "boxes": len(boxes), "cells": cells, "particles": npart,
           "launch": list(lat.get_launch()), "momentum_exchange": lat.get_mea_mode(), "kernel_ms": kt,
           "l2": f"inputs larger than L2 ({BYTES_PER_CELL[prec] // 2 * cells / 1e6:.0f} MB of populations)",
           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "kernel": "collide_pair_kernel" if lat.get_launch()[2] == 2 else "collide_stream_kernel"}}
    out["coupling"], out["step_roofline"] = coupling_and_step_roofline(lat, cells, npart, steps, ms, ws, prec, peak)
    lat.close()
    return out


def coupling_and_step_roofline(lat, cells, npart, steps, ms, ws, prec, peak):
    """Particle-coupling throughput and the roofline of the whole step.

    The interior cells (cell centre inside a particle) are the cells the
    momentum exchange sums over; the library counts them in the moments
    mode (the mode is switched for one step if another was in use).  Bytes
    of a step: the collision's 2 * 19 * s per cell plus, per interior cell,
    the momentum exchange's 19 arrivals (19 * s) and, in the moments mode,
    the 24-byte list entry written by the collision and read back (in the
    bounding-box mode the 19 departures instead)."""
    mode = lat.get_mea_mode()
    n_int = 0
    if npart > 0:
        if mode != "moments":
            lat.set_mea_mode("moments")
            lat.step(1)
        n_int = lat.interior_cells()
        if mode != "moments":
            lat.set_mea_mode(mode)
    s = BYTES_PER_CELL[prec] // 38
    per_int = 19 * s + (48 if mode == "moments" else 19 * s)
    bpc_mea = BYTES_PER_CELL[prec] + per_int * n_int / cells
    sec = ms / steps / 1e3
    coupling = {"interior_cells_per_step": n_int, "interior_fraction": n_int / cells,
                "mea_cell_updates_per_s": ws * n_int / sec, "particles_per_s": ws * npart / sec,
                "unit": "per second, whole job"}
    step_roofline = {"bound": "hbm", "unit": "GB/s", "peak": peak,
                     "bytes_per_cell_without_mea": BYTES_PER_CELL[prec],
                     "bytes_per_cell_with_mea": bpc_mea,
                     "achieved": bpc_mea * cells / sec / 1e9,
                     "frac": bpc_mea * cells / sec / 1e9 / peak,
                     "mlups_roofline_without_mea": peak * 1e3 / BYTES_PER_CELL[prec],
                     "mlups_roofline_with_mea": peak * 1e3 / bpc_mea,
                     "frac_of_mlups_roofline_without_mea": cells / sec / 1e6 / (peak * 1e3 / BYTES_PER_CELL[prec]),
                     "frac_of_mlups_roofline_with_mea": cells / sec / 1e6 / (peak * 1e3 / bpc_mea),
                     "note": "whole step (momentum exchange, update, collision) per GPU; per interior cell "
                             f"{per_int} B of momentum exchange ({mode} mode)"}
    return coupling, step_roofline


def fp32_fp16_pair(w, args, stream, peak, ws, steps_max=40):
    """One workload with FP32 and with FP16 storage of f - w: step time,
    collision roofline, coupling throughput and whole-step roofline, and the
    FP16 error against FP32 after the same number of steps.  Populations far
    larger than L2, so steps run back to back."""
    import torch
    from paper_2312_14172_gb300 import hlbm
    cells = w["n"][0] * w["n"][1] * w["n"][2]
    npart = len(w["particles"]["shape"])
    steps = max(1, min(args.steps, steps_max))
    out, states = {}, {}
    for prec in ("fp32", "fp16"):
        lat = hlbm.from_workload(w, precision=prec, stream=stream)
        if args.autotune:
            lat.autotune(nsteps=3)
        elif args.mea_mode:
            lat.set_mea_mode(args.mea_mode)
        lat.step(args.warmup)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        lat.sync()
        ms = max_over_ranks(e0.elapsed_time(e1))
        kt = lat.kernel_times(nsteps=4)
        ach = BYTES_PER_CELL[prec] * cells / (kt["collide_stream"] / 1e3) / 1e9
        coupling, step_rl = coupling_and_step_roofline(lat, cells, npart, steps, ms, ws, prec, peak)
        out[prec] = {"value": whole_job_mlups(cells, steps, ms, ws), "unit": "MLUPS", "ms_per_step": ms / steps,
                     "steps": steps, "launch": list(lat.get_launch()), "momentum_exchange": lat.get_mea_mode(),
                     "kernel_ms": kt,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak, "kernel": "collide_stream"},
                     "coupling": coupling, "step_roofline": step_rl}
        states[prec] = (lat.steps_done, lat)
    # error of FP16 against FP32 after the same number of steps
    n32, lat32 = states["fp32"]
    n16, lat16 = states["fp16"]
    if n16 < n32:
        lat16.step(n32 - n16)
    elif n32 < n16:
        lat32.step(n16 - n32)
    s32, s16 = lat32.particle_state(), lat16.particle_state()
    lat32.close()
    lat16.close()
    err = {}
    X0 = w["particles"]["X"]
    for key in ("X", "U", "F", "T"):
        a32 = s32[key] - (X0 if key == "X" else 0)
        a16 = s16[key] - (X0 if key == "X" else 0)
        if key == "X":  # displacement, periodic wrap of a centre next to a face
            L = np.asarray(w["n"], float)
            a32 -= L * np.round(a32 / L)
            a16 -= L * np.round(a16 / L)
        scale = float(np.abs(a32).max()) or 1.0
        err[key] = float(np.abs(a16 - a32).max() / scale)
    out["error_fp16_vs_fp32"] = err
    P = w["particles"]
    out["workload"] = {"name": w["name"], "dims": list(w["n"]), "particles": npart, "cells": cells,
                       "solid_fraction": solid_fraction(P, cells)}
    out["speedup_fp16_over_fp32"] = out["fp16"]["value"] / out["fp32"]["value"]
    return out


def solid_fraction(P, cells):
    """Total particle volume over the lattice volume."""
    from paper_2312_14172_gb300 import workloads
    return float(workloads.particle_volumes(P).sum() / cells)


def nonspherical_leg(args, stream, peak, ws):
    """The non-spherical workload (256^3, 2000 ellipsoids and cuboids, eps =
    1.5) with FP32 and with FP16 storage (populations of 1.27 GB / 0.64 GB)."""
    return fp32_fp16_pair(make_workload("nonspherical"), args, stream, peak, ws, steps_max=100)


def capsules_leg(args, stream, peak, ws):
    """The non-spherical workload's box, counts and size laws with capsules
    only (2000 sphere-swept segments of equal volume, aspect ratio
    U(1, 4), eps = 1.5), FP32 and FP16 storage."""
    return fp32_fp16_pair(make_workload("capsules"), args, stream, peak, ws, steps_max=100)


def grid_shapes_leg(args, stream, peak, ws):
    """The non-spherical workload's box and counts with signed-distance grid
    particles (2000 rounded boxes of equal volume from four grids of aspect
    ratio 1-4, spacing 1/2, random orientations, eps = 1.5), FP32 and FP16
    storage."""
    return fp32_fp16_pair(make_workload("grid_shapes"), args, stream, peak, ws, steps_max=100)


def settling_correlations(phi, re):
    """The three hindered-settling correlations of the paper (Sec. 5) as
    u_bar / u*: Richardson-Zaki (1 - phi)^n with its piecewise expansion
    index in Re, Garside-Al-Dibouni with n = (5.1 + 0.27 Re^0.9) /
    (1 + 0.1 Re^0.9), and Barnea-Mizrahi (1 - phi) / ((1 + phi^(1/3))
    exp(5 phi / (3 (1 - phi))))."""
    if re < 0.2:
        n_rz = 4.65
    elif re < 1.0:
        n_rz = 4.35 * re ** -0.03
    elif re < 500.0:
        n_rz = 4.45 * re ** -0.1
    else:
        n_rz = 2.39
    n_gad = (5.1 + 0.27 * re ** 0.9) / (1.0 + 0.1 * re ** 0.9)
    bm = (1.0 - phi) / ((1.0 + phi ** (1.0 / 3.0)) * np.exp(5.0 * phi / (3.0 * (1.0 - phi))))
    return {"richardson_zaki": (1.0 - phi) ** n_rz, "garside_al_dibouni": (1.0 - phi) ** n_gad,
            "barnea_mizrahi": float(bm), "n_rz": n_rz, "n_gad": n_gad}


def settling_validation_leg(args, stream):
    """Zero-net-flow hindered settling in the set-up of the paper's Sec. 5.1:
    monodisperse spheres of N cells diameter (default 12, the resolution from
    which the paper finds grid-independent results) at random positions in a
    periodic cube of 12 diameters, Archimedes number 1500, density ratio 1.3,
    relaxation time 0.55, solid fractions 0.05 to 0.3, 300 t* with
    t* = D / u*_St and averages taken after 30 t*.  The counter pressure
    gradient is the uniform fluid force of workloads.zero_net_flow, held at
    zero net momentum by feedback once per t* (the paper uses the Ergun
    equation, which it does not print); particles repel through the contact
    extension (hlbm_set_contact, stiffness ten buoyant weights, range 1.5
    cells), without which they overlap at the higher fractions.  Reported
    per fraction: the mean settling velocity relative to the volume-averaged
    velocity, over the reference u* (terminal velocity of an isolated sphere
    with the Schiller-Naumann drag) and over one sphere in the same box,
    beside the three correlations.  A qualitative check, as in the paper."""
    from paper_2312_14172_gb300 import hlbm, workloads
    d = int(args.settling_n)
    tau, rho_r, ar = 0.55, 1.3, 1500.0
    nu = (tau - 0.5) / 3.0
    g = ar * nu * nu / (d ** 3 * (rho_r - 1.0))
    u_st = g * d * d * (rho_r - 1.0) / (18.0 * nu)
    u = u_st
    for _ in range(200):  # u* = sqrt(4 g D (rho_r - 1) / (3 C_d)), C_d of Schiller-Naumann
        re = u * d / nu
        cd = 24.0 / re * (1.0 + 0.15 * re ** 0.687)
        u = 0.5 * u + 0.5 * math.sqrt(4.0 * g * d * (rho_r - 1.0) / (3.0 * cd))
    re = u * d / nu
    t_star = d / u_st
    steps = int(round(args.settling_tstar * t_star))
    sample = max(1, int(round(t_star)))
    avg_from = int(round(0.1 * steps))  # 30 of 300 t*
    weight = (rho_r - 1.0) * math.pi * d ** 3 / 6.0 * g
    k_contact, zeta = 10.0 * weight, 1.5

    def run(w):
        # The momentum exchange does not see the EDM forcing of the smooth
        # zone outside the interior cells (an O(eps / r) share of the
        # coupling), so a constant counter force leaves a small net force and
        # the whole suspension would drift: the counter force is reset every
        # sample interval to cancel the drift rate of the last interval and
        # let the accumulated momentum (lattice plus the particles' mass beyond
        # the fluid's) decay over a few intervals.
        lat = hlbm.from_workload(w, stream=stream)
        lat.set_mea_mode("moments")
        lat.set_contact(k_contact, zeta)
        P = w["particles"]
        extra = (np.asarray(P["rho_p"], float) - 1.0) * workloads.particle_volumes(P)
        ncell = float(np.prod(w["n"]))
        fz = float(w["fluid_force"][2])
        p_prev = 0.0
        vals, drift, stopped = [], [], None
        t0 = time.perf_counter()
        for k in range(0, steps, sample):
            lat.step(sample)
            try:
                U = lat.particle_state()["U"]
                _, J = lat.fluid_momentum()
            except hlbm.HLBMError as e:
                stopped = {"step": k + sample, "t_over_tstar": (k + sample) / t_star, "error": str(e)}
                break
            p_tot = float(J[2] + (extra * U[:, 2]).sum())
            fz -= (p_tot - p_prev) / (ncell * sample) + p_tot / (ncell * 4 * sample)
            p_prev = p_tot
            lat.set_fluid_force((0.0, 0.0, fz))
            if k >= avg_from:
                uz = float(J[2]) / ncell
                vals.append(uz - float(U[:, 2].mean()))
                drift.append(uz)
        dt = time.perf_counter() - t0
        lat.close()
        mean = lambda v: float(np.mean(v)) if v else float("nan")
        return mean(vals), dt, stopped, mean(drift)

    mk = lambda phi: workloads.hindered_settling_periodic(phi, d=d, box_d=12, tau=tau, rho_ratio=rho_r, g=g)
    one = dict(mk(0.05))
    one["particles"] = {k: v[:1] for k, v in one["particles"].items()}
    one = workloads.zero_net_flow(one)
    u1, dt1, stopped1, _ = run(one)
    rows = []
    for phi in (0.05, 0.1, 0.15, 0.2, 0.3):
        w = mk(phi)
        ub, dt, stopped, drift = run(w)
        P = w["particles"]
        phi_r = float(workloads.particle_volumes(P).sum() / np.prod(w["n"]))
        row = {"phi": phi_r, "particles": len(P["shape"]), "u_over_ustar": ub / u, "u_over_u_single": ub / u1,
               "drift_over_ustar": drift / u, "seconds": dt, "stopped": stopped}
        row.update({k: v for k, v in settling_correlations(phi_r, re).items() if not k.startswith("n_")})
        rows.append(row)
    corr = settling_correlations(0.1, re)
    return {"d": d, "box": [12 * d] * 3, "tau": tau, "rho_p_over_rho_f": rho_r, "archimedes": ar, "g": g,
            "u_star": u, "u_star_stokes": u_st, "re": re, "n_rz": corr["n_rz"], "n_gad": corr["n_gad"],
            "t_star_steps": t_star, "steps": steps, "average_from_step": avg_from, "sample_steps": sample,
            "contact": {"k": k_contact, "zeta": zeta, "buoyant_weight": weight},
            "u_single_over_ustar": u1 / u, "single_seconds": dt1, "single_stopped": stopped1, "rows": rows}


def batched_fp16_leg(args, stream, peak, ws):
    """The large dense batch (512 x 512 x 1024 cells, 50 000 lognormal
    spheres, realised solid fraction 0.075) with FP32 and with FP16 storage
    (populations of 20 GB / 10 GB)."""
    return fp32_fp16_pair(make_workload("dense_batch"), args, stream, peak, ws)


def _generate(name):
    from paper_2312_14172_gb300 import workloads
    return getattr(workloads, name)()


def phi_matched_leg(args, stream, peak, ws):
    """The two workloads at the solid fractions their configurations name
    (0.15: 4806 ellipsoids and cuboids in 256^3; 0.2: 50 000 spheres of
    median diameter 11.1 in 512 x 512 x 1024), each with FP32 and FP16
    storage.  Both are drawn in parallel host processes first."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(2) as pool:
        ws_ = pool.map(_generate, ["nonspherical_phi_matched", "dense_batch_phi_matched"])
    return {w["name"]: fp32_fp16_pair(w, args, stream, peak, ws) for w in ws_}


def summary_of(line):
    """Each leg's MLUPS, collision fraction of HBM and whole-step fraction of
    the roofline MLUPS (without the momentum exchange's bytes), and the FP16
    error against FP64, in one small object printed last on the line."""
    def leg(d):
        if not d:
            return None
        sr = d.get("step_roofline") or {}
        return {"mlups": round(d["value"], 1), "collision_frac": round(d["roofline"]["frac"], 4),
                "step_frac": round(sr["frac_of_mlups_roofline_without_mea"], 4) if sr else None}
    out = {"headline": leg(line)}
    out["headline"]["e2e_mlups"] = round(line["e2e"]["value"], 1) if line.get("e2e") else None
    if line.get("e2e") and line["e2e"].get("moved"):
        out["headline"]["e2e_moved_mlups"] = round(line["e2e"]["moved"]["value"], 1)
    if line.get("fp16"):
        out["headline_fp16"] = {"mlups": round(line["fp16"]["value"], 1),
                                "collision_frac": round(line["fp16"]["roofline"]["frac"], 4)}
    for key in ("nonspherical", "batched_fp16", "capsules", "grid_shapes", "phi_matched"):
        d = line.get(key)
        if d and "fp32" in d:
            out[key] = {p: leg(d[p]) for p in ("fp32", "fp16")}
            out[key]["fp16_over_fp32"] = round(d["speedup_fp16_over_fp32"], 3)
    if line.get("ensemble"):
        out["ensemble"] = {"fp32": leg(line["ensemble"]), "fp16": leg(line["ensemble"].get("fp16"))}
    err = (line.get("cpu_baseline") or {}).get("error_vs_fp64")
    if err:
        out["error_vs_fp64_max"] = {p: {q: float(f"{v['max']:.3g}") for q, v in err[p].items()}
                                    for p in ("fp32", "fp16")}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="hindered_settling", choices=WORKLOADS)
    ap.add_argument("--precision", default=None, choices=[None, "fp32", "fp16"])
    ap.add_argument("--no-fp16", dest="fp16", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 512x512x1024 dense-batch FP32/FP16 leg")
    ap.add_argument("--no-ensemble", dest="ensemble", action="store_false",
                    help="skip the 64-box ensemble leg")
    ap.add_argument("--no-nonspherical", dest="nonspherical", action="store_false",
                    help="skip the 256^3 non-spherical FP32/FP16 leg")
    ap.add_argument("--settling-validation", action="store_true",
                    help="add the zero-net-flow hindered-settling check against the paper's three "
                         "correlations (a few minutes)")
    ap.add_argument("--settling-n", type=int, default=12, help="cells per sphere diameter of that check")
    ap.add_argument("--settling-tstar", type=float, default=300.0,
                    help="its duration in t* = D / u*_St (the paper: 300)")
    ap.add_argument("--capsules", action="store_true",
                    help="add the 256^3 box of 2000 capsules with FP32 and FP16 storage")
    ap.add_argument("--grid-shapes", action="store_true",
                    help="add the 256^3 box of 2000 signed-distance grid particles with FP32 and FP16 storage")
    ap.add_argument("--phi-matched", action="store_true",
                    help="add the solid-fraction-matched variants of the non-spherical and dense workloads "
                         "(about two minutes of host time to draw them)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--mea-mode", default=None, choices=[None, "kernel", "moments"])
    ap.add_argument("--launch", default=None, help="collision launch shape TILE_Y,TILE_Z[,CELLS_X] (skips tuning)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = init_dist()
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    line = run_gpu(args, ws, rank, local)
    if rank == 0:
        if args.cpu_baseline:
            w = make_workload(args.workload)
            probe, dt1 = oracle_mlups(w, 1)
            steps = max(1, min(40, int(15.0 / max(dt1, 1e-3))))
            mlups, dt, o = oracle_mlups(w, steps, keep=True)
            line["cpu_baseline"] = {
                "value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                "sample": f"{steps} steps of the full {w['n'][0]}x{w['n'][1]}x{w['n'][2]} workload, "
                          f"FP64, single thread, {dt:.1f} s"}
            # the GPU's FP32 and FP16 runs of the same steps against this
            # FP64 state, per quantity
            line["cpu_baseline"]["error_vs_fp64"] = error_vs_fp64(w, o, steps)
            o.close()
            # the same oracle built with OpenMP: collision and streaming over z
            # slices, momentum exchange over particles, on every host core
            from oracle import oracle
            probe, dt1 = oracle_mlups(w, 1, omp=True)
            steps = max(1, min(100, int(15.0 / max(dt1, 1e-3))))
            mlups, dt = oracle_mlups(w, steps, omp=True)
            line["cpu_baseline"]["openmp"] = {
                "value": mlups, "unit": "MLUPS", "cores": oracle.threads(omp=True), "kind": "oracle",
                "sample": f"{steps} steps of the same workload, FP64, OpenMP, {dt:.1f} s"}
        else:
            line["cpu_baseline"] = None
        line["summary"] = summary_of(line)
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
