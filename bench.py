#!/usr/bin/env python
"""Benchmark of the explicit phase-field fracture step on B300.

Workload (default): the 1000 x 1000-cell glass plate, 100 x 40 mm,
1,002,001 nodes / 2,000,000 P1 triangles with +-0.1h seeded interior
jitter, AT2, spectral split, plane strain, traction 1 MPa with the smooth
ramp, dt = 0.5 x CFL, FP32 kernels with FP64 reductions/history.  A step is
one full staggered step: predictor, element force + history, corrector,
damage right-hand side, the Jacobi-PCG loop to rel. tol 1e-8 and the clamp.

`python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]`
prints one JSON line.  Under torchrun each rank runs an independent replica
of the plate (the method does not shard across GPUs here: "replicas only",
weak scaling); value = all ranks' node-updates / max-over-ranks time.
The reference arm times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pff_synth as S  # noqa: E402

METRIC = "explicit-step node-updates/s at 1M nodes; fwd+adjoint s/step; % HBM roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="plate_1000x1000")
    ap.add_argument("--prec", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--split", choices=["spectral", "amor"], default="spectral")
    ap.add_argument("--model", choices=["AT2", "AT1"], default="AT2")
    ap.add_argument("--operator", choices=["element", "merged"], default="element",
                    help="damage operator form (pff_mesh_set_operator): element-wise "
                         "matrix-free (default) or rows merged per solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=24)
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-plate batched measurement")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the forward+adjoint measurement on the 500x500 plate")
    ap.add_argument("--variant", type=int, default=0,
                    help="gather schedule (0 = autotuned; 1..5 fixed, see pff_options.variant)")
    ap.add_argument("--cg-kernel", choices=["auto", "phases", "persistent", "staged", "fused", "fused_staged", "resident"],
                    default="auto", help="AT2 CG loop (pff_options.cg_kernel; auto = autotuned)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP64 run and the FP32-vs-FP64 error of the benchmark plate")
    ap.add_argument("--no-qs", action="store_true",
                    help="skip the quasi-static single-edge-notched tension measurement")
    ap.add_argument("--qs-only", action="store_true",
                    help="run only the quasi-static measurement and print its line")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the forward + adjoint measurement (checkpoints every 25 steps, damage tape) "
                         "and print its line")
    ap.add_argument("--adjoint-steps", type=int, default=300,
                    help="steps of the forward + adjoint measurement (300 by default)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 64-plate batch measurement and print its line")
    ap.add_argument("--batch-steps", type=int, default=500,
                    help="timed steps of the 64-plate batch (500 by default)")
    ap.add_argument("--qs-increments", type=int, default=100,
                    help="timed load increments of the quasi-static run (all 100 by default)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the 1M-node volumetric-deviatoric and AT1 configurations")
    ap.add_argument("--no-inversion", action="store_true",
                    help="skip the gradient checks and L-BFGS recovery on the 500x500 plate")
    ap.add_argument("--fuse", choices=["auto", "separate", "fused"], default="auto",
                    help="force and damage right-hand side: autotuned, two kernels, or one (pff_options.fuse)")
    ap.add_argument("--nvtx-range", action="store_true",
                    help="wrap the timed steps in the NVTX range 'timed' (for ncu --nvtx-include timed/)")
    ap.add_argument("--loop", choices=["graph", "host"], default="graph",
                    help="host: launch every kernel from the host (ncu cannot profile "
                         "kernels inside graphs with conditional nodes)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes):
    the SM clock, its maximum and the active clock-event reasons."""

    CLOCK_SM = 1

    def __init__(self, index):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError(f"nvmlDeviceGetHandleByIndex_v2({index}) failed")
        self.get_reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _clock(self, fn):
        v = self.C.c_uint()
        if fn(self.h, self.C.c_int(self.CLOCK_SM), self.C.byref(v)) != 0:
            raise RuntimeError("NVML clock query failed")
        return float(v.value)

    def sm_mhz(self):
        return self._clock(self.lib.nvmlDeviceGetClockInfo)

    def max_sm_mhz(self):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo)

    def reasons(self):
        v = self.C.c_ulonglong()
        if self.get_reasons(self.h, self.C.byref(v)) != 0:
            raise RuntimeError("NVML reasons query failed")
        return int(v.value)

    def close(self):
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """Samples the SM clock and the clock-event (throttle) reasons while
    running: through NVML every millisecond when the driver's library loads
    (the timed region of a short run lasts tens of milliseconds), else
    through nvidia-smi every 100 ms.  Read-only queries."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []
        self.stop_flag = False

    def start(self):
        try:
            self.nvml = _Nvml(self.index)
            self.smax = self.nvml.max_sm_mhz()
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return
        except Exception as e:  # no NVML library: nvidia-smi
            self.nvml = None
            self.nvml_error = f"{type(e).__name__}: {e}"
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _poll(self):
        while not self.stop_flag:
            try:
                self.samples.append((self.nvml.sm_mhz(), self.nvml.reasons()))
            except Exception:
                break
            time.sleep(0.001)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.stop_flag = True
            self.t.join(timeout=5)
            sm = [c for c, _ in self.samples]
            reasons = sorted({nm for _, r in self.samples for nm, b in self.BITS.items() if r & b})
            self.nvml.close()
            return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=self.smax,
                        reasons=reasons, samples=len(sm), source="nvml (libnvidia-ml), 1 ms")
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=smax,
                    reasons=sorted(reasons), samples=len(sm), source="nvidia-smi, 100 ms",
                    nvml_error=getattr(self, "nvml_error", None))


# ------------------------------------------------------------- utilities

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def l2_peak_gbs(dev, sizes_mb=(16, 20, 24, 28), k=20, rounds=10):
    """L2-resident bandwidth, measured here: torch.add(a, c, out=b) on FP32
    buffers of each size (three buffers together 48 to 84 MB, inside the 126
    MB L2), k adds captured in one CUDA graph so that launch gaps do not
    count, best round over sizes, bytes = two reads and one write.  The
    denominator of the CG loop's roofline, whose working set stays in L2
    across iterations (on B300 this is about twice the HBM copy rate)."""
    import torch
    best = 0.0
    for mb in sizes_mb:
        n = mb * 2 ** 20 // 4
        a = torch.ones(n, device=dev)
        b = torch.empty_like(a)
        c = torch.ones_like(a)
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            for _ in range(3):
                torch.add(a, c, out=b)
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(k):
                torch.add(a, c, out=b)
        g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(rounds):
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            best = max(best, 12 * n * k / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        del g, a, b, c
    return best


def ncu_traffic(kernel_prefix, summary="ncu_streaming_plate_1000x1000_fp32.md"):
    """DRAM bytes (read + write) from the committed ncu summary: the column of
    the first table whose header names the kernel (per launch, or per CG
    iteration for the CG loop summary), or None when the kernel source
    changed since the capture (the summary records the source hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2606_23458_b300", "csrc", "kernels.cuh")
    try:
        text = open(path).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if f"`{h}`" not in text:
        return None
    lines = text.splitlines()
    for n, ln in enumerate(lines):
        if not ln.startswith("|"):
            continue
        head = [c.strip(" `") for c in ln.strip("|").split("|")]
        col = next((i for i, c in enumerate(head) if kernel_prefix in c), None)
        if col is None:
            continue
        val = {}
        for row in lines[n + 2:]:
            if not row.startswith("|"):
                break
            cells = [c.strip() for c in row.strip("|").split("|")]
            name = cells[0].split(" ")[0]
            if name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                unit = cells[0].split("(")[-1].rstrip(")")
                scale = {"Mbyte": 1e6, "Kbyte": 1e3, "Gbyte": 1e9, "byte": 1.0}.get(unit)
                if scale is None:
                    return None
                val[name] = float(cells[col]) * scale
        return sum(val.values()) if len(val) == 2 else None
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def job_throughput(ms_local, units_per_rank, steps, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's
    timed region (max over ranks when a process group is up) and the units
    all ranks processed.  Returns (value per second, max ms)."""
    import torch
    ws = 1
    t_max = float(ms_local)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    return ws * units_per_rank * steps / (t_max / 1e3), t_max


def algorithmic_bytes(N, Ne, prec):
    """Bytes the method must move, by kernel (FP32_MIXED unless prec=fp64).
    Element data: connectivity 12 B, geometry (4 independent shape
    gradients + area) 5 words, history H 8 B (read + write in the force
    kernel), reaction coefficient 1 word.  Node data per kernel below."""
    w = 8 if prec == "fp64" else 4
    geo = 5 * w
    return {
        # predictor: read u, v, a, write u
        "predict": N * (8 * w),
        # force: T, geometry, H r/w per element; u, d, v, a, 1/m, flags per node; write v, a
        "force": Ne * (12 + geo + 16) + N * (2 * w + w + 4 * w + w + 1 + 4 * w),
        # damage rhs: T, geometry, H per element; d_prev, flags; write x, r (f64), z, p, 1/diag, coef
        "rhs": Ne * (12 + geo + 8 + w) + N * (w + 1 + 16 + 3 * w),
        # CG matvec: T, geometry, coefficient per element; p (as z + beta p) read, q write
        "matvec": Ne * (12 + geo + w) + N * (w + w + 1),
        # CG update: x, r (f64) r/w, q, 1/diag, p read; z, p write
        "update": N * (32 + 3 * w + 2 * w + 1),
        # clamp: x (f64), d_prev read, d write
        "finish": N * (8 + 2 * w + 1),
        # one CG iteration as the method states it: element pass (connectivity
        # 12 B, geometry 20 B, H 8 B), p read and q write, fused vector update
        # (x, r in FP64, p, z, diag) -- multiplied by the iterations of a launch
        "cg_iteration": Ne * (12 + 20 + 8) + N * (8 + 48),
    }


def merged_row_width(tri, N):
    """Width of the damage operator's merged rows on a compact FP32 mesh: 6
    when no node has more than six distinct neighbours, 8 up to eight, else
    None (the per-entry records are used)."""
    t = np.asarray(tri, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [0, 2]]])
    e.sort(axis=1)
    key = np.unique(e[:, 0] * N + e[:, 1])
    deg = np.bincount(np.concatenate([key // N, key % N]), minlength=N).max()
    return 6 if deg <= 6 else 8 if deg <= 8 else None


def format_bytes_cg_iteration(N, form, width, family, fan=False):
    """Bytes one FP32 CG iteration reads and writes in the stored form of the
    damage operator, per row (neighbour values are L2 hits):
    element-wise (entry records): flags, diagonal and per incidence slot a
    16-bit offset pair and two element coefficients (12 B, width = slots);
    element-wise in fan order: flags, diagonal, six 16-bit neighbour offsets
    (12 B), the fan word (4 B) and per fan position two coefficients (8 B);
    merged rows: flags, diagonal, width/2 offset words and width merged
    coefficients.  Two-pass families (persistent, phases): matvec (the row's
    own (p, z) pair read, q written) and vector update (x, r, (p, z) read
    and written; q and 1/diag read, flags again).  Single-reduction family:
    one pass reading the row's (r, w, s, 1/diag) record, p and x, writing
    the new record, p and x.  Resident family: x, p, flags, diagonal and
    the fan tables stay in shared memory for the whole solve, so a pass
    moves the coefficients and the row's record (read and write)."""
    if form == "element" and fan:
        rec = 1 + 4 + 12 + 4 + 8 * width
    else:
        rec = 1 + 4 + (12 * width if form == "element" else 2 * width + 4 * width)
    if family == "resident":
        return N * (8 * width + 16 + 16)
    if family == "fused":
        return N * (rec + 16 + 8 + 8 + 16)
    return N * ((rec + 8 + 4) + (1 + 8 + 8 + 16 + 4 + 4))


def incidence_width(tri, N):
    """Largest number of elements meeting at a node (the entry records'
    slots per row)."""
    return int(np.bincount(np.asarray(tri, dtype=np.int64).ravel(), minlength=N).max())


def host_cores():
    """Host CPU threads this process may run on (the box's core count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count()


# -------------------------------------------------------------- reference

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    c = S.config(args.config, split=args.split, model=args.model)
    m = oracle.Mesh.from_plate(c["mesh"])
    mat = c["material"]
    dt = m.stable_dt(mat, c["cfl"])
    st = m.new_state()
    m.run(mat, st, args.warmup, dt, n0=0)
    t0 = time.perf_counter()
    r = m.run(mat, st, args.steps, dt, n0=args.warmup)
    el = time.perf_counter() - t0
    N = m.N
    val = N * args.steps / el
    line = dict(impl="reference", metric=METRIC, value=val, unit="node-updates/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * el / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config=dict(workload=args.config, nodes=N, elements=m.Ne, split=args.split,
                            model=args.model, precision="fp64", cg_tol=1e-8),
                cpu_baseline=dict(value=val, unit="node-updates/s", cores=1, host_cores=host_cores(), kind="oracle",
                                  sample=f"full {args.config} plate, steps {args.warmup}.."
                                         f"{args.warmup + args.steps - 1} after {args.warmup} untimed"),
                e2e=dict(value=val, unit="node-updates/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                cg_iters_mean=float(r["iters"][:, 0].mean()))
    print(json.dumps(line), flush=True)


def cpu_baseline(args, budget_s=20.0):
    """The oracle as it stands on one host core, on the same plate: warm-up
    steps untimed, then as many of the bench's steps as fit the budget."""
    import oracle
    oracle.build()
    c = S.config(args.config, split=args.split, model=args.model)
    m = oracle.Mesh.from_plate(c["mesh"])
    mat = c["material"]
    dt = m.stable_dt(mat, c["cfl"])
    st = m.new_state()
    m.run(mat, st, args.warmup, dt, n0=0)
    n, el = 0, 0.0
    while n < args.steps and el < budget_s:
        t0 = time.perf_counter()
        m.run(mat, st, 1, dt, n0=args.warmup + n)
        el += time.perf_counter() - t0
        n += 1
    return dict(value=m.N * n / el, unit="node-updates/s", cores=1, host_cores=host_cores(), kind="oracle",
                sample=f"{args.config} full plate, steps {args.warmup}..{args.warmup + n - 1} "
                       f"({n} steps, {el:.1f} s, single thread of {host_cores()} host threads, FP64)")


def batched(pff, dev, steps=500, warmup=5, nvtx=False):
    """The batched workload: 64 independent plates drawn from SplitMix64
    seed 1 (200..700 x 80..280 cells, Gc in [1, 5] J/m^2, traction in
    [0.5, 2] MPa), FP32 with FP64-class reductions, 500 steps, all plates
    advanced by one CUDA graph launch per step, the damage solves of all
    plates in the CG loop form and with the gathers in flight the batch's
    autotuner picked (per-plate persistent launch, the per-plate resident
    loop in waves of plates, or kernels per phase; `tuning`), each plate to
    its own stop."""
    import torch
    plates = []
    for dr in S.batch_draws(64, seed=1):
        p = S.plate(dr["nx"], dr["ny"], jitter=0.1, seed=1, traction=dr["traction"])
        plates.append((p, S.material(2 * p["h"], Gc=dr["Gc"])))
    b = pff.Batch(plates, precision="fp32")
    nodes = sum(inf["N"] for inf in b.info)
    st = b.new_state(device=dev)
    opts = pff.options()
    b.run(st, warmup, opts=opts)
    torch.cuda.synchronize()
    log = torch.zeros(steps, b.nplates, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    b.run(st, steps, step0=warmup, opts=opts, iters_log=log)
    e1.record(stream)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    it = log.cpu().numpy()
    return dict(workload="64 plates, seed 1", plates=b.nplates, nodes=nodes, steps=steps, warmup=warmup,
                value=nodes * steps / (ms / 1e3), unit="node-updates/s", ms_per_step=ms / steps,
                cg_iters_mean=float(it.mean()), cg_iters_max=int(it.max()), cg_iters_min=int(it.min()),
                tuning=b.tuning())


def fwd_adjoint(pff, dev, steps=300, policies=((0, "recompute"), (25, "recompute"), (25, "damage_tape")),
                nvtx=False):
    """Forward + adjoint cost on the differentiation workload: the 500 x 500
    plate (251,001 nodes), FP32 with FP64-class reductions, 300 steps,
    loss = mean((d_T - d*)^2) with d* from Gc* = 3 J/m^2, gradient dL/dGc at
    Gc = 2 (Sec. 4.1-4.2).  Each tape policy is timed: every = 0 tapes the
    whole run in the forward (Sec. 7, the activation tape kept on the GPU);
    every = 25 keeps checkpoints and recomputes each segment, in full
    ("recompute", damage solves included) or its mechanics only
    ("damage_tape": the forward also tapes each step's unclamped damage
    solution, one value per node and step).  The ratio divides by a plain
    forward run (pff_run, no tape) of the same steps."""
    import torch
    c = S.config("plate_500x500")
    mesh = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    mat = c["material"]
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"])
    mesh.set_material(dict(mat, Gc=3.0), c["cfl"])
    st = mesh.new_state(device=dev)
    mesh.run(st, steps, opts=opts)
    dstar = st["d"].clone()
    mesh.set_material(dict(mat, Gc=2.0), c["cfl"])
    stream = torch.cuda.current_stream()

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    # plain forward: the denominator
    log = torch.zeros(steps, 2, dtype=torch.int32, device=dev)
    w = mesh.new_state(device=dev)
    mesh.run(w, 3, opts=opts)
    st = mesh.new_state(device=dev)
    torch.cuda.synchronize()
    e0 = ev()
    mesh.run(st, steps, opts=opts, iters_log=log)
    e1 = ev()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    out = dict(workload="plate_500x500", nodes=mesh.N, steps=steps,
               fwd_s_per_step=t_plain / steps, fwd_cg_iters_mean=float(log[:, 0].float().mean()))
    for every, policy in policies:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ck = pff.Checkpoint(mesh, steps, every, policy)
        torch.cuda.synchronize()
        store_bytes = free0 - torch.cuda.mem_get_info()[0]
        # warm-up: graphs, autotuner, the backward's graphs and the torch ops
        # of the loss gradient (their first use loads kernels)
        w = mesh.new_state(device=dev)
        ckw = pff.Checkpoint(mesh, 3, min(every, 3), policy)
        mesh.run_ckpt(w, ckw, opts=opts)
        gw = (2.0 * (w["d"].double() - dstar.double()) / mesh.N).float().contiguous()
        mesh.backward(ckw, gw, opts=opts)
        ckw.close()
        st = mesh.new_state(device=dev)
        torch.cuda.synchronize()
        e0 = ev()
        mesh.run_ckpt(st, ck, opts=opts)
        e1 = ev()
        d = st["d"]
        gup = (2.0 * (d.double() - dstar.double()) / mesh.N).float().contiguous()
        if nvtx:  # the backward alone (for ncu --nvtx-include timed/)
            torch.cuda.nvtx.range_push("timed")
        g = mesh.backward(ck, gup, opts=opts)
        e2 = ev()
        if nvtx:
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        tf = e0.elapsed_time(e1) / 1e3
        tb = e1.elapsed_time(e2) / 1e3
        loss = float(torch.mean((d.double() - dstar.double()) ** 2))
        name = "full_tape" if every == 0 else (f"ckpt_every_{every}" if policy == "recompute"
                                                else f"ckpt_every_{every}_damage_tape")
        out[name] = dict(
            fwd_taped_s_per_step=tf / steps, bwd_s_per_step=tb / steps,
            fwd_adj_s_per_step=(tf + tb) / steps, ratio=(tf + tb) / t_plain, loss=loss, dL_dGc=g,
            adjoint_cg_iters_mean=ck.adjoint_iters() / steps, store_bytes=int(store_bytes))
        ck.close()
    return out


def subcycled(pff, dev, config, steps=100, warmup=10):
    """Damage subcycling (Sec. 2.4) on the benchmark plate: N_sub = the
    material's limit floor(c_p / (0.6 c_R)) (at least 2), same step and
    tolerance otherwise."""
    import torch
    c = S.config(config)
    ratio, nmax = pff.subcycling_limit(c["material"])
    n_sub = max(2, nmax)
    mesh = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    mesh.set_material(c["material"], c["cfl"])
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], damage_every=n_sub)
    st = mesh.new_state(device=dev)
    mesh.run(st, warmup, opts=opts)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mesh.run(st, steps, step0=warmup, opts=opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return dict(workload=config, n_sub=n_sub, limit_ratio=ratio, limit_n_max=nmax, steps=steps,
                value=mesh.N * steps / (ms / 1e3), unit="node-updates/s", ms_per_step=ms / steps,
                status=int(mesh.sync_status()))


def precision_check(pff, dev, config, steps=997, warmup=3):
    """The precision policy on the benchmark plate: the same steps in FP64
    (the parity mode, itself checked against the oracle by the tests) and in
    FP32_MIXED from the same zero state; the FP64 run is timed (CUDA events
    after `warmup` steps), and the FP32 fields are compared with it at the
    end of the window: relative L2 error of u and max |d32 - d64| (stated
    tolerances 1e-4 and 1e-3 over a pre-branching window)."""
    import torch
    c = S.config(config)
    out = {}
    for prec in ("fp64", "fp32"):
        mesh = pff.Mesh.from_plate(c["mesh"], precision=prec)
        dt = mesh.set_material(c["material"], c["cfl"])
        opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"])
        st = mesh.new_state(device=dev)
        mesh.run(st, warmup, opts=opts)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.run(st, steps, step0=warmup, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = dict(ms_per_step=ms, value=mesh.N / (ms / 1e3), status=int(mesh.sync_status()),
                         u=st["u"].double(), d=st["d"].double())
        del mesh
    u64, u32 = out["fp64"].pop("u"), out["fp32"].pop("u")
    d64, d32 = out["fp64"].pop("d"), out["fp32"].pop("d")
    return dict(workload=config, steps=warmup + steps, window_us=dt * (warmup + steps) * 1e6,
                fp64=out["fp64"], fp32=out["fp32"],
                fp32_vs_fp64=dict(u_rel_l2=float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64)),
                                  d_max_abs=float((d32 - d64).abs().max()), d_max=float(d64.max()),
                                  tolerances=dict(u_rel_l2=1e-4, d_max_abs=1e-3)),
                speedup_fp32_over_fp64=out["fp64"]["ms_per_step"] / out["fp32"]["ms_per_step"])


def quasistatic(pff, dev, increments=100, n=700, compare_increments=2):
    """Quasi-static single-edge-notched tension (Sec. 3.5): the 700 x 700
    unit square, the first `increments` of the 100 equal load increments to
    7e-3 mm (all of them by default, with the reaction curve), each an
    inexact Newton solve (FP64 state and residual; tangent CG in FP32 with
    double-word dots, i.e. FP32 matvecs and FP64-class inner products) on
    the element-wise tangent to |r| <= 1e-8 |f|, history and the damage
    solve (FP64, tol 1e-8).  The first compare_increments are timed beside
    it with the tangent CG in FP64, and with the tangent's rows merged per
    Newton step (the assembled form).  qs_run synchronises, so the events
    bracket whole increments."""
    import torch
    c = S.sent(n)
    out = dict(workload=c["name"], nodes=None, elements=None, increments_total=c["increments"],
               du=c["du"], newton_tol=c["newton_tol"], damage_cg_tol=c["cg_tol"])
    opts = pff.options(cg_tol=c["cg_tol"], cg_max_it=100000)
    stream = torch.cuda.current_stream()
    runs = (("fp32_krylov", "fp32", increments, "element"), ("fp64_krylov", "mesh", compare_increments, "element"),
            ("fp32_krylov_merged", "fp32", compare_increments, "merged"))
    for label, krylov, k, form in runs:
        if k <= 0:
            continue
        mesh = pff.Mesh.from_plate(c["mesh"], precision="fp64")
        mesh.set_material(c["material"], 0.5)
        mesh.set_operator(form)
        out["nodes"], out["elements"] = mesh.N, mesh.Ne
        q = pff.qs_options(newton_tol=c["newton_tol"], krylov=krylov)
        st = mesh.new_state(device=dev)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = mesh.qs_run(st, c["bc"], k, c["du"], qopts=q, opts=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        it = r["iters"]
        out[label] = dict(increments=k, operator=form, s_per_increment=ms / 1e3 / k, newton=it[:, 0].tolist(),
                          tangent_cg=it[:, 1].tolist(), damage_cg=it[:, 2].tolist(),
                          us_per_tangent_cg_iteration=ms * 1e3 / max(int(it[:, 1].sum()), 1),
                          reaction_N_per_m=r["reaction"].tolist(), d_max=float(st["d"].max()))
        del mesh, st
    if "fp32_krylov" in out and "fp64_krylov" in out:
        k = min(len(out["fp32_krylov"]["reaction_N_per_m"]), len(out["fp64_krylov"]["reaction_N_per_m"]))
        out["top_displacement_m"] = [c["du"] * (j + 1) for j in range(len(out["fp32_krylov"]["reaction_N_per_m"]))]
        a = np.array(out["fp32_krylov"]["reaction_N_per_m"][:k])
        b = np.array(out["fp64_krylov"]["reaction_N_per_m"][:k])
        out["reaction_rel_diff_fp32_vs_fp64_krylov"] = float(np.max(np.abs(a - b) / np.abs(b)))
    return out


def mechanics_only(pff, dev, config, steps=200, warmup=10):
    """The explicit step without the damage solve (node-updates per second
    are reported with and without it): the same plate and step graph with the
    damage solve never due (damage_every beyond the run), so each step is
    the predictor, the force kernel with the history update and the
    corrector."""
    import torch
    c = S.config(config)
    mesh = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    mesh.set_material(c["material"], c["cfl"])
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"], damage_every=warmup + steps + 1)
    st = mesh.new_state(device=dev)
    mesh.run(st, warmup, opts=opts)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mesh.run(st, steps, step0=warmup, opts=opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return dict(workload=config, steps=steps, value=mesh.N * steps / (ms / 1e3), unit="node-updates/s",
                ms_per_step=ms / steps, status=int(mesh.sync_status()))


def plate_rate(pff, dev, config, prec="fp32", split="spectral", model="AT2", form="element",
               steps=50, warmup=5, profile=False):
    """Node-updates/s of one plate configuration (CUDA events around `steps`
    full staggered steps after `warmup` untimed ones), its CG iterations and,
    with profile, the persistent CG launch's time per iteration."""
    import torch
    c = S.config(config, split=split, model=model)
    mesh = pff.Mesh.from_plate(c["mesh"], precision=prec)
    mesh.set_material(c["material"], c["cfl"])
    mesh.set_operator(form)
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"])
    st = mesh.new_state(device=dev)
    log = torch.zeros(warmup + steps, 2, dtype=torch.int32, device=dev)
    mesh.run(st, warmup, opts=opts, iters_log=log[:warmup])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mesh.run(st, steps, step0=warmup, opts=opts, iters_log=log[warmup:])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    it = log[warmup:].cpu().numpy()
    out = dict(workload=config, precision=prec, split=split, model=model, operator=form, steps=steps,
               value=mesh.N * steps / (ms / 1e3), unit="node-updates/s", ms_per_step=ms / steps,
               cg_iters_mean=float(it[:, 0].mean()), restarts_mean=float(it[:, 1].mean()),
               status=int(mesh.sync_status()), cg_loop=mesh.cg_choice()[0])
    if profile:
        prof = mesh.profile_kernels(st, reps=5, opts=opts)
        if prof["cg_loop"] > 0:
            out["cg_us_per_iteration"] = 1e3 * prof["cg_loop"] / max(prof["cg_loop_iters"], 1)
        out["kernel_ms"] = prof
    return out


def variants_1m(pff, dev, config, steps=30):
    """The 1M-node plate's other configurations: the volumetric-deviatoric
    split (Eq. amor_split) in FP32 and FP64, and AT1 with that split and the
    bound-projected CG (Sec. 2.4), FP32 and FP64."""
    out = {}
    for prec, split, model in (("fp32", "amor", "AT2"), ("fp64", "amor", "AT2"),
                               ("fp32", "amor", "AT1"), ("fp64", "amor", "AT1")):
        out[f"{model}_{split}_{prec}"] = plate_rate(pff, dev, config, prec, split, model, steps=steps)
    return out


def inversion(pff, dev, steps=300, gcs=(2.0, 2.5, 3.5), gc_star=3.0, max_states=8):
    """Toughness inversion on the differentiation plate (Sec. 4.1, Eq.
    inversion_loss): 500 x 500 cells, FP32 kernels with FP64-class
    reductions, 300 steps, target d* from Gc* = 3 J/m^2.  At each Gc of
    `gcs`: dL/dGc from the adjoint (full tape) beside a central difference of
    the GPU forward with delta = 1e-4 Gc.  Then L-BFGS on log Gc from Gc =
    2.0 (strong-Wolfe line search, one accepted state per step), each
    closure a forward with checkpoints every 25 steps and the adjoint."""
    import torch
    from paper_2606_23458_b300 import inverse
    c = S.config("plate_500x500")
    mat = c["material"]
    mesh = pff.Mesh.from_plate(c["mesh"], precision="fp32")
    mesh.set_material(mat, c["cfl"])
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"])
    f64 = torch.float64
    dstar = inverse.final_damage(torch.tensor(gc_star, dtype=f64), mesh, mat, steps, 0, opts).detach()

    def loss_at(gc, grad):
        g = torch.tensor(gc, dtype=f64, requires_grad=grad)
        L = inverse.mse_loss(inverse.final_damage(g, mesh, mat, steps, 0, opts), dstar)
        if grad:
            L.backward()
            return float(L.detach()), float(g.grad)
        return float(L.detach()), None

    grads = []
    for gc in gcs:
        L, g = loss_at(gc, True)
        h = 1e-4 * gc
        fd = (loss_at(gc + h, False)[0] - loss_at(gc - h, False)[0]) / (2 * h)
        grads.append(dict(Gc=gc, loss=L, dL_dGc_adjoint=g, dL_dGc_central_fd=fd,
                          rel_diff=abs(g - fd) / abs(fd) if fd else None))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gc, hist = inverse.recover_gc(mesh, mat, steps, dstar, 2.0, every=25, opts=opts, max_states=max_states)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    errs = [abs(g - gc_star) / gc_star for g in hist["states"]]
    first = next((k + 1 for k, e in enumerate(errs) if e < 1e-3), None)
    return dict(workload="plate_500x500", nodes=mesh.N, steps=steps, gc_star=gc_star, gradients=grads,
                lbfgs=dict(gc0=2.0, states=hist["states"], rel_err=errs, accepted_states_to_1e_3=first,
                           closure_evaluations=len(hist["evals"]), final_gc=gc,
                           final_rel_err=abs(gc - gc_star) / gc_star, wall_s=el, checkpoint_every=25))


def kernel_rooflines(prof, iters_mean, N, Ne, prec, form, width, peak, peak_kind, fan=False, l2_peak=None):
    """Roofline of the dominant kernel of a step and the HBM fractions of the
    streaming kernels, from pff_profile_kernels' live launch times (CUDA
    events on the launching stream, L2 flushed before every launch).

    achieved = the method's algorithmic bytes per launch / launch time.  For
    the CG loop (one persistent launch per solve) that is the matrix-free
    count of one iteration (element pass 40 B per element, vectors 56 B per
    node) times the launch's iterations; its working set (operator records
    and vectors, about 100 MB on the 1M-node plate) stays in the 126 MB L2
    across iterations, so `traffic` (ncu DRAM bytes) sits far below those
    bytes and `dram_frac` is the fraction of HBM bandwidth the loop really
    draws.  Its bound is then the L2: with l2_peak (l2_peak_gbs) the CG
    loop's roofline is labelled "l2", its fraction taken against that
    measured L2-resident copy bandwidth, and the HBM figures (peak, DRAM
    traffic, dram_frac) move to roofline["hbm"].  The streaming kernels (force with history and corrector, damage
    right-hand side, predictor, clamp) read and write each element and node
    once from HBM; their fractions are the HBM roofline figures proper."""
    ab = algorithmic_bytes(N, Ne, prec)
    per_step = {k: prof[k] for k in ("predict", "force", "rhs", "finish")}
    ms_launch = {k: prof[k] for k in per_step}
    bytes_launch = {k: ab[k] for k in per_step}
    if prof["cg_loop"] > 0:  # the solve's CG loop is one persistent launch
        per_step["cg_loop"] = prof["cg_loop"] * iters_mean / max(prof["cg_loop_iters"], 1)
        ms_launch["cg_loop"] = prof["cg_loop"]
        bytes_launch["cg_loop"] = ab["cg_iteration"] * prof["cg_loop_iters"]
    else:
        for k in ("matvec", "update"):
            per_step[k] = prof[k] * iters_mean
            ms_launch[k] = prof[k]
            bytes_launch[k] = ab[k]
    dom = max(per_step, key=per_step.get)
    achieved = bytes_launch[dom] / (ms_launch[dom] * 1e-3) / 1e9
    kname = {"matvec": "k_cg_matvec_nc", "update": "k_cg_update", "force": "k_force_nc",
             "rhs": "k_dmg_rhs_nc", "cg_loop": "k_cg_"}.get(dom, dom)
    traffic = None
    if prec == "fp32":
        if dom == "cg_loop":
            per_iter = ncu_traffic(kname, f"ncu_full_cg_loop_plate_1000x1000_fp32_{form}.md")
            traffic = per_iter * prof["cg_loop_iters"] if per_iter else None
        else:
            traffic = ncu_traffic(kname)
    roofline = dict(bound="hbm", kernel=dom if dom != "cg_loop" else f"cg_loop ({prof['cg_loop_family']})",
                    operator=form, achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                    peak_kind=peak_kind, traffic=traffic, bytes_per_launch=bytes_launch[dom],
                    ms_per_launch=ms_launch[dom],
                    cg_iterations_per_launch=prof["cg_loop_iters"] if dom == "cg_loop" else None)
    if traffic:
        roofline["dram_frac"] = traffic / (ms_launch[dom] * 1e-3) / 1e9 / peak
    den = peak
    if dom == "cg_loop" and l2_peak:
        hbm = dict(peak=peak, peak_kind=peak_kind, traffic=traffic, dram_frac=roofline.pop("dram_frac", None),
                   method_bytes_over_hbm_peak=achieved / peak)
        roofline.update(bound="l2", peak=l2_peak, frac=achieved / l2_peak,
                        peak_kind="measured here: L2-resident bandwidth (l2_peak_gbs)", hbm=hbm)
        den = l2_peak
    if dom == "cg_loop" and width and prec == "fp32" and prof["cg_loop_family"] in (
            "persistent", "phases", "fused", "resident"):
        fb = format_bytes_cg_iteration(N, form, width, prof["cg_loop_family"], fan) * prof["cg_loop_iters"]
        roofline["format"] = dict(name=("element-wise entry records" + (" in fan order" if fan else "")
                                        if form == "element" else "merged rows")
                                  + f", width {width}", bytes_per_launch=fb,
                                  achieved=fb / (ms_launch[dom] * 1e-3) / 1e9,
                                  frac=fb / (ms_launch[dom] * 1e-3) / 1e9 / den)
        roofline["note"] = ("bytes_per_launch: the method's matrix-free count; format: the bytes the stored "
                            "operator records and vectors move; the loop's working set stays in L2 across "
                            "iterations, so its DRAM traffic (hbm.traffic, hbm.dram_frac) is a small share of "
                            "either and its roofline is the L2's; the HBM roofline figures are the streaming "
                            "kernels'")
    streaming = {}
    for k, kn in (("predict", "k_predict"), ("force", "k_force_nc"), ("rhs", "k_dmg_rhs_nc"),
                  ("finish", "k_dmg_finish")):
        if prof[k] > 0:
            t = ncu_traffic(kn) if prec == "fp32" else None
            streaming[k] = dict(bytes=ab[k], ms=prof[k], gbs=ab[k] / (prof[k] * 1e-3) / 1e9,
                                frac=ab[k] / (prof[k] * 1e-3) / 1e9 / peak, traffic=t,
                                dram_frac=t / (prof[k] * 1e-3) / 1e9 / peak if t else None)
    return roofline, streaming


# ------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    dev = torch.device("cuda", lrank)
    torch.cuda.set_device(dev)
    import paper_2606_23458_b300 as pff

    if args.adjoint_only:
        if rank == 0:
            print(json.dumps(dict(fwd_adjoint=fwd_adjoint(pff, dev, steps=args.adjoint_steps,
                                                          policies=((25, "damage_tape"),), nvtx=args.nvtx_range))),
                  flush=True)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    if args.batch_only:
        if rank == 0:
            print(json.dumps(dict(batched=batched(pff, dev, steps=args.batch_steps, nvtx=args.nvtx_range))),
                  flush=True)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    if args.qs_only:
        if rank == 0:
            print(json.dumps(dict(quasistatic=quasistatic(pff, dev, args.qs_increments, compare_increments=0))),
                  flush=True)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    c = S.config(args.config, split=args.split, model=args.model)
    mesh = pff.Mesh.from_plate(c["mesh"], precision=args.prec)
    dt = mesh.set_material(c["material"], c["cfl"])
    mesh.set_operator(args.operator)
    N, Ne = mesh.N, mesh.Ne
    opts = pff.options(cg_tol=c["cg_tol"], t_ramp=c["t_ramp"],
                       loop_mode=pff.PFF_LOOP_HOST if args.loop == "host" else pff.PFF_LOOP_GRAPH,
                       variant=args.variant,
                       cg_kernel={v: k for k, v in pff.CG_KINDS.items()}[args.cg_kernel],
                       fuse={"auto": 0, "separate": 1, "fused": 2}[args.fuse])
    st = mesh.new_state(device=dev)
    total = args.warmup + args.steps
    log = torch.zeros(total + args.e2e_steps, 2, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # warm-up (also builds and instantiates the step graph)
    mesh.run(st, args.warmup, step0=0, opts=opts, iters_log=log[:args.warmup])
    torch.cuda.synchronize()

    clk = ClockSampler(lrank)
    clk.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if args.nvtx_range:
        torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    mesh.run(st, args.steps, step0=args.warmup, opts=opts, iters_log=log[args.warmup:total])
    e1.record(stream)
    torch.cuda.synchronize()
    if args.nvtx_range:
        torch.cuda.nvtx.range_pop()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    status = mesh.sync_status()
    iters = log[args.warmup:total, 0].cpu().numpy()

    # end-to-end through the public API with host-resident state
    # (pff_run_host, one call for the e2e steps): every step copies the state
    # in from pinned host memory, runs, and copies it back; the copies of u,
    # v, a and H back overlap the step's damage solve, and in the library's
    # pipelined chunks of steps a step's copies in overlap the previous
    # step's damage solve.
    hs = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in st.items()}
    for k in hs:
        hs[k].copy_(st[k])
    bytes_state = sum(v.numel() * v.element_size() for v in st.values())
    mesh.run_host(hs, st, args.e2e_steps, step0=total, opts=opts)  # its graphs, once
    for k in hs:
        hs[k].copy_(st[k])
    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    mesh.run_host(hs, st, args.e2e_steps, step0=total + args.e2e_steps, opts=opts,
                  iters_log=log[total:total + args.e2e_steps])
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1)

    # per-kernel device times on this data (overwrites the state)
    sched_var, sched_ms = mesh.schedule()
    frhs_var, frhs_ms = mesh.fused_schedule()
    cg_kind, cg_U, cg_ms = mesh.cg_choice()
    prof = mesh.profile_kernels(st, reps=5, opts=opts)
    # our kernels in the timed region: the history mirror once per run call,
    # then per step the predictor, the force and right-hand side (one fused
    # kernel, or two), the clamp and the CG loop (one persistent launch, or
    # a matvec and an update per iteration)
    per_solve = 1 if cg_kind not in ("phases", "auto") else None
    per_step = 3 if prof.get("force_rhs_used") else 4
    launches = int(1 + per_step * args.steps + (args.steps * per_solve if per_solve else 2 * iters.sum()))

    # aggregate over ranks
    value, t_max = job_throughput(ms, N, args.steps, device=dev)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = peaks()
    l2_peak = l2_peak_gbs(dev)
    roofline, streaming = kernel_rooflines(prof, iters.mean(), N, Ne, args.prec, args.operator,
                                           incidence_width(c["mesh"]["tri"], N)
                                           if args.operator == "element" else
                                           merged_row_width(c["mesh"]["tri"], N), peak, peak_kind,
                                           fan=args.operator == "element" and mesh.fan_order(), l2_peak=l2_peak)
    ab = algorithmic_bytes(N, Ne, args.prec)
    step_bytes = sum(ab[k] for k in ("predict", "force", "rhs", "finish")) + iters.mean() * ab["cg_iteration"]
    line = dict(
        metric=METRIC, value=value, unit="node-updates/s", n_gpus=ws, steps=args.steps,
        warmup=args.warmup, ms_per_step=t_max / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32" if args.prec == "fp32" else "f64",
        data="synthetic",
        config=dict(workload=args.config, nodes=N, elements=Ne, split=args.split, model=args.model,
                    precision=("FP32 kernels and vectors, double-word FP32 dot products and CG scalars, FP64 history"
                               if args.prec == "fp32" else "FP64"),
                    cg_tol=c["cg_tol"], cg_tol_fp32_floor=2.0 ** -22 if args.prec == "fp32" else None,
                    dt=dt, parallelism=f"replicas x{ws}", loop=args.loop,
                    l2=("no flush between steps: a step streams about 0.3 GB of element and node data "
                        "through HBM (inputs larger than the 126 MB L2); the damage solve's ~100 MB "
                        "working set stays L2-resident within a step"),
                    operator=args.operator),
        roofline=roofline,
        streaming_kernels=streaming,
        # the step's method bytes (streaming kernels from HBM, CG iterations
        # mostly from L2) over the step time: a rate, not an HBM fraction
        step_roofline=dict(bytes=step_bytes, gbs=step_bytes / (t_max / args.steps * 1e-3) / 1e9,
                           hbm_bytes=sum(ab[k] for k in ("predict", "force", "rhs", "finish")),
                           l2_bytes=iters.mean() * ab["cg_iteration"]),
        e2e=dict(value=ws * N * args.e2e_steps / (e2e_ms / 1e3), unit="node-updates/s",
                 h2d_bytes_per_step=bytes_state, d2h_bytes_per_step=bytes_state),
        gpu_launches=launches, clocks=clocks, status=int(status),
        cg_iters=dict(mean=float(iters.mean()), max=int(iters.max()), min=int(iters.min()),
                      per_step=[int(v) for v in iters] if args.steps <= 64 else None),
        kernel_ms=prof,
        schedule=dict(variant=sched_var, tune_ms=sched_ms,
                      force_rhs=dict(variant=frhs_var, tune_ms=frhs_ms),
                      cg_loop=dict(kind=cg_kind, gathers=cg_U, ms_30_iterations=cg_ms)),
    )
    other = "merged" if args.operator == "element" else "element"
    line["operator_forms"] = {
        args.operator: dict(value=value, ms_per_step=t_max / args.steps, cg_iters_mean=float(iters.mean()),
                            cg_us_per_iteration=(1e3 * prof["cg_loop"] / max(prof["cg_loop_iters"], 1)
                                                 if prof["cg_loop"] > 0 else None),
                            roofline=roofline),
        other: plate_rate(pff, dev, args.config, args.prec, args.split, args.model, other,
                          steps=min(args.steps, 100), profile=True),
        "labels": dict(element="matrix-free: every CG product applies each element's own coefficients "
                               "(Eq. matrix_free_fe_operator); the benchmarked default",
                       merged="assembled per solve: the two elements' coefficients of each edge summed "
                              "into one per neighbour by the right-hand side (pff_mesh_set_operator)"),
    }
    if other in line["operator_forms"] and line["operator_forms"][other].get("kernel_ms"):
        pk, pk_kind = peaks()
        line["operator_forms"][other]["roofline"] = kernel_rooflines(
            line["operator_forms"][other].pop("kernel_ms"), line["operator_forms"][other]["cg_iters_mean"],
            N, Ne, args.prec, other,
            merged_row_width(c["mesh"]["tri"], N) if other == "merged" else incidence_width(c["mesh"]["tri"], N),
            pk, pk_kind, l2_peak=l2_peak)[0]
    if args.model == "AT2" and args.split == "spectral" and not args.no_variants:
        line["variants_1m"] = variants_1m(pff, dev, args.config)
    if args.model == "AT2":
        line["subcycled"] = subcycled(pff, dev, args.config)
    line["mechanics_only"] = mechanics_only(pff, dev, args.config)
    if not args.no_adjoint:
        line["fwd_adjoint"] = fwd_adjoint(pff, dev)
    if not args.no_batch:
        line["batched"] = batched(pff, dev)
    if not args.no_qs:
        line["quasistatic"] = quasistatic(pff, dev, args.qs_increments)
    if not args.no_precision:
        line["precision"] = precision_check(pff, dev, args.config)
    if not args.no_inversion:
        line["inversion"] = inversion(pff, dev)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
