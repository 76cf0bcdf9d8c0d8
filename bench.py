#!/usr/bin/env python3
"""Throughput benchmark of the explicit TE/TM solver (Eq. (23)) on one GB300.

Workload (default): the 256 x 256 x 2048 staircase step collimator, pipe
radius 96 -> 32 -> 96 transverse cells, dz = 1 mm, dx = dy = sqrt(2) mm,
c*dt = dz, Gaussian bunch sigma = 6 dz on the axis; float32 fields, float64
wake and balances. One benchmark step is one time step of the whole path:
the bunch current, the ten updates, one wake sample per window point, and
every --balance-every steps the float64 energy and charge balances.

value  = cells * steps / device time of the timed steps, Gcell-updates/s,
         summed over ranks (each rank runs its own replica: weak scaling).
e2e    = the same metric for one complete solve through the C ABI from host
         buffers: tetm_create from a pinned host PEC array, tetm_set_bunch,
         tetm_step(all steps), tetm_wake into host memory.
roofline: the fused step kernel, algorithmic bytes = 12 field words + 1 mask
         byte per cell that carries a field (49 B in float32; cells inside
         PEC hold zero fields and are no work of the method) per launch, over
         its mean launch duration measured with CUDA events on its stream;
         the same figure over the cells of the launched work items is kept
         beside it (achieved_on_processed_cells).
active_gcell_updates_s: the field-carrying cells advanced per second.
balances: the cost of one float64 energy and charge balance (a9), measured
         apart, and its share of a step at the --balance-every cadence.

--impl reference times the FP64 CPU oracle (test infrastructure) on the
host, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s"
UNIT = "Gcell-updates/s"
RZ_FLOPS_PER_CELL = 47
FLOPS_PER_CELL_3D = 48
FP64_PEAK_TFLOPS = 1.25


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="tetm", choices=["tetm", "reference"])
    p.add_argument("--workload", default="collimator",
                   choices=["collimator", "plain_pipe", "batch", "serve", "dielectric", "rz"])
    p.add_argument("--config", default=None,
                   choices=["plain-pipe-fp64", "collimator-fp32", "rz-chain", "batch-64", "serve-2000"],
                   help="a named workload with its precision: the 24x24x96 plain pipe in float64, the "
                        "256x256x2048 step collimator in float32, the 512x16384 nine-cell r-z chain, "
                        "the 64-solve batch, the 2000-request served stream")
    p.add_argument("--rz-chunk", type=int, default=0,
                   help="rz: planes per work item (0 = chosen by the autotuner, untimed)")
    p.add_argument("--rz-kernel", default=None, choices=[None, "async", "register", "bulk", "bulk2"],
                   help="rz: step kernel (default: chosen by the autotuner, untimed)")
    p.add_argument("--rz-start", default="scattered", choices=["cold", "static", "scattered"],
                   help="rz: bunch start (cold: through the entry wall; static: with its TEM "
                        "field in the entry pipe; scattered: the static start with the "
                        "incident TEM field split off, default)")
    p.add_argument("--check", action="store_true",
                   help="Cartesian, float32: also run the full solve in float64 and report the "
                        "error of the longitudinal and transverse wakes against it")
    p.add_argument("--rz-check", action="store_true",
                   help="rz, float32: also run the full solve in float64 (total-field static "
                        "start) and report every wake's error against it")
    p.add_argument("--requests", type=int, default=2000, help="serve: requests in the stream")
    p.add_argument("--rate", type=float, default=40.0, help="serve: mean arrivals per second")
    p.add_argument("--round-steps", type=int, default=16, help="serve: steps per batch call")
    p.add_argument("--solves", type=int, default=64, help="batch: number of solves")
    p.add_argument("--precision", default=None, choices=[None, "fp32", "fp64"])
    p.add_argument("--balance-every", type=int, default=250)
    p.add_argument("--tiling", default=None,
                   help="tile_x,tile_y,chunk_z (default: chosen by the autotuner, untimed)")
    p.add_argument("--no-autotune", action="store_true", help="keep the library's default shape")
    p.add_argument("--kernel", default="fused", choices=["fused", "reference", "twostep"],
                   help="twostep: the block-tiled sweep with two steps per pass (temporal blocking), "
                        "timed in pairs of steps; needs --tiling 32,4,C / 32,8,C / 64,4,C")
    p.add_argument("--scheme", default="tetm", choices=["tetm", "yee"],
                   help="yee: Yee's E/M leapfrog (Eq. (7)) on the same grid at its step bound (8), "
                        "field-only, timed beside the TE/TM scheme per unit of simulated length")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=0, help="0 = the workload's full step count")
    p.add_argument("--nz", type=int, default=0,
                   help="smaller case of the same workload (profiling): number of z cells")
    p.add_argument("--n", type=int, default=0,
                   help="plain_pipe only: transverse cells (profiling a fully active box)")
    args = p.parse_args()
    if args.config:
        args.workload = {"plain-pipe-fp64": "plain_pipe", "collimator-fp32": "collimator", "rz-chain": "rz",
                         "batch-64": "batch", "serve-2000": "serve"}[args.config]
        if args.config == "plain-pipe-fp64" and args.precision is None:
            args.precision = "fp64"
    return args


def make_workload(args):
    from paper_0901_1053_gb300 import workloads as wl
    args.eps = None
    if args.workload == "dielectric":
        w, args.eps = wl.dielectric_collimator(n=256, nz=args.nz or 1024)
        if args.precision:
            w.precision = args.precision
        return w
    if args.workload == "plain_pipe":
        w = wl.plain_pipe(nz=args.nz or 96, n=args.n or 24)
    else:
        w = wl.step_collimator(nz=args.nz or 2048)
    if args.precision:
        w.precision = args.precision
    return w


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """Control plane only (barrier, max of timings): gloo on CPU tensors."""

    def __init__(self, world):
        self.world = world
        if world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
            self.d = dist

    def barrier(self):
        if self.world > 1:
            self.d.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.d.all_reduce(t, op=self.d.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x):
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.d.all_reduce(t, op=self.d.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.d.destroy_process_group()


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) < 10:
                    continue
                if self.uuid and self.uuid not in t[1]:
                    continue
                rows.append(t)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if _num(r[2])]
        mx = [float(r[3]) for r in rows if _num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[4]) for r in rows if _num(r[4])), default=None)}


def _num(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ---------------------------------------------------------------------------
# Roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(names=("kernels_step.cu", "kernels_warp.cu")):
    """Hash of the step-kernel sources (the translation units of the kernel)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_0901_1053_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def fp64_peak(tetm):
    """(TFLOP/s, kind): the device's float64 FMA rate measured by the
    library's microbenchmark, else the part's nominal rate."""
    try:
        return tetm.tetm_measure_fma_rate("fp64"), "measured fp64 FMA rate (tetm_measure_fma_rate)"
    except Exception:
        return FP64_PEAK_TFLOPS, "nominal fp64 rate of the part"


def host_cpu():
    """nproc and the CPU model of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model or __import__("platform").machine()}


def profiled_traffic(name, sources=("kernels_step.cu", "kernels_warp.cu"), tiling=None):
    """DRAM bytes per launch from the committed ncu summary for this kernel
    and workload; None if absent, taken on a different kernel source or (when
    the summary names one) on a different work shape than `tiling`."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash(sources):
        return None
    t = re.search(r"tiling:\s*([0-9]+)\s*,\s*([0-9]+)\s*,\s*([0-9]+)", txt)
    if tiling is not None and t and tuple(int(x) for x in t.groups()) != tuple(tiling):
        return None
    return float(m.group(1))


def balance_cost(s, steps=4):
    """(ms per float64 balance, plain ms per step) on solve s: device time
    of `steps` steps with a balance after every step against the same steps
    without, CUDA events on the solve's stream. Leaves the balances off."""
    import torch
    st = torch.cuda.current_stream()
    out = []
    for every in (1, 0):
        s.set_balance_every(every)
        s.step(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        s.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / steps)
    return out[0] - out[1], out[1]


# ---------------------------------------------------------------------------
# CPU oracle (test infrastructure) on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(w, planes, steps):
    import dataclasses
    from oracle import Oracle
    sub = dataclasses.replace(w, nz=planes, pec=None if w.pec is None else w.pec[:planes].copy())
    o = Oracle(sub.nx, sub.ny, sub.nz, sub.dx, sub.dy, sub.dz, sub.cdt, pec=sub.pec)
    o.set_bunch(sub.sigma, sub.charge, sub.i0, sub.j0)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = sub.nx * sub.ny * sub.nz
    return cells * steps / dt / 1e9, dt, "first %d of %d planes of %s (same transverse grid and " \
        "geometry), %d steps, FP64, 1 thread" % (planes, w.nz, w.name, steps)


def cpu_baseline(w):
    planes = min(w.nz, 256 if w.nx * w.ny >= 256 * 256 else w.nz)
    steps = 20 if w.nx * w.ny >= 256 * 256 else 400
    v, dt, desc = oracle_sample(w, planes, steps)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
            "seconds": round(dt, 2), "host": host_cpu()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args)
    # bounded sample: each benchmark step is one oracle time step on the first
    # planes of the workload, sized so the whole run stays around two minutes
    budget_cells = 2.0e7 * 120.0 / max(1, args.steps + args.warmup)
    planes = int(max(2, min(w.nz, budget_cells // (w.nx * w.ny))))
    import dataclasses
    from oracle import Oracle
    sub = dataclasses.replace(w, nz=planes, pec=None if w.pec is None else w.pec[:planes].copy())
    o = Oracle(sub.nx, sub.ny, sub.nz, sub.dx, sub.dy, sub.dz, sub.cdt, pec=sub.pec)
    o.set_bunch(sub.sigma, sub.charge, sub.i0, sub.j0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    cells = sub.nx * sub.ny * sub.nz
    v = cells * args.steps / dt / 1e9
    desc = "first %d of %d planes of %s, %d timed steps after %d warm-up steps, FP64, 1 thread" % (
        planes, w.nz, w.name, args.steps, args.warmup)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "sample_planes": planes},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_tetm(args):
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world)
    from paper_0901_1053_gb300 import tetm
    w = make_workload(args)
    stream = torch.cuda.current_stream()
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, eps_r=args.eps,
                    pec=w.pec)
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.set_stream(stream.cuda_stream)
    if args.tiling:
        args.tiling_used = tuple(int(x) for x in args.tiling.split(","))
    elif args.kernel == "fused" and not args.no_autotune:
        from paper_0901_1053_gb300.autotune import Autotuner
        args.tiling_used = Autotuner().tune(w, w.precision, eps_r=args.eps)
    else:
        args.tiling_used = None
    if args.kernel == "twostep" and not args.tiling_used:
        args.tiling_used = (32, 8, 32)
    if args.tiling_used:
        s.set_tiling(*args.tiling_used)
    s.set_kernel(args.kernel)
    s.set_balance_every(args.balance_every)
    info = s.info()
    s.step(args.warmup)
    s.sync()

    try:
        uuid = torch.cuda.get_device_properties(local).uuid
        uuid = str(uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.5)
    # steps per timed call: pairs for the two-step kernel (one launch each)
    per_call = 2 if args.kernel == "twostep" else 1
    K = args.steps - args.steps % per_call
    nc = K // per_call
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nc + 1)]
    dist.barrier()
    torch.cuda.synchronize()
    n0 = s.info()["step"]
    for i in range(nc):
        evs[i].record(stream)
        s.step(per_call)
    evs[nc].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    total_ms = evs[0].elapsed_time(evs[nc])
    per = [evs[i].elapsed_time(evs[i + 1]) / per_call for i in range(nc)]
    be = args.balance_every
    bal_steps = [i for i in range(K) if be > 0 and (n0 + i + 1) % be == 0]
    bal_calls = {i // per_call for i in bal_steps}
    plain = [per[i] for i in range(nc) if i not in bal_calls]
    kern_ms = statistics.mean(plain) if plain else total_ms / K
    max_ms = dist.max(total_ms)

    esz = 4 if w.precision == "fp32" else 8
    # 12 field words and either the activity byte or, with per-cell materials,
    # the six coefficient words, per cell that carries a field: the work of
    # the method (a cell in PEC holds zero fields for ever)
    bytes_per_cell = 12 * esz + 1 if args.eps is None else 18 * esz
    if args.kernel == "twostep":  # y^n read and y^{n+2} written once per two steps
        bytes_per_cell = bytes_per_cell / 2
    proc = info["processed_cells"] if args.kernel != "reference" else w.cells
    act = info["active_cells"]
    gbs = bytes_per_cell * act / (kern_ms * 1e-3) / 1e9
    gbs_proc = bytes_per_cell * proc / (kern_ms * 1e-3) / 1e9
    if w.precision == "fp32":
        achieved = gbs
        peak, peak_kind = measured_peak_hbm()
        roof = {"bound": "hbm", "unit": "GB/s", "bytes_per_cell": bytes_per_cell, "basis": "active cells",
                "achieved_on_processed_cells": gbs_proc, "frac_on_processed_cells": gbs_proc / peak}
    else:
        # float64 arithmetic sets the pace on this part: 48 flops per cell
        # and step (the ten updates, a fused multiply-add counted as two)
        achieved = FLOPS_PER_CELL_3D * act / (kern_ms * 1e-3) / 1e12
        peak, peak_kind = fp64_peak(tetm)
        roof = {"bound": "alu", "unit": "TFLOP/s", "flops_per_cell": FLOPS_PER_CELL_3D, "basis": "active cells",
                "achieved_on_processed_cells": FLOPS_PER_CELL_3D * proc / (kern_ms * 1e-3) / 1e12,
                "hbm_gbs": gbs, "bytes_per_cell": bytes_per_cell}
    kname = {28: "fused_step_warp", 56: "fused_step_slab"}.get(info["tile_x"], "fused_step")
    if args.kernel == "twostep":
        kname = "fused_step2"
    if args.eps is not None:
        kname = "fused_step_slab_mat" if info["tile_x"] == 56 else "fused_step_warp_mat"
    prof_name = "%s_%s_%s.md" % (kname, w.precision, w.name)
    sources = ("kernels_slab.cu",) if kname.startswith("fused_step_slab") else ("kernels_step.cu", "kernels_warp.cu")
    traffic = (profiled_traffic(prof_name, sources, (info["tile_x"], info["tile_y"], info["chunk_z"]))
               if args.kernel != "reference" else None)
    wake = s.wake()[0]
    hist = s.balance_history()
    bal_ms, plain_ms = balance_cost(s) if be > 0 else (0.0, kern_ms)
    s.close()

    e2e = None
    if not args.no_e2e:
        steps_e2e = args.e2e_steps or w.steps
        pinned = None
        if w.pec is not None:
            pinned = torch.empty(w.pec.shape, dtype=torch.uint8, pin_memory=True).numpy()
            pinned[...] = w.pec
        out = torch.empty(len(wake), dtype=torch.float64, pin_memory=True).numpy()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, eps_r=args.eps,
                         pec=pinned)
        s2.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        if args.check:
            s2.set_observer(w.i0, w.j0)
        s2.set_kernel(args.kernel)
        if args.tiling_used:
            s2.set_tiling(*args.tiling_used)
        s2.set_balance_every(args.balance_every)   # the same path as the device-timed steps
        s2.step(steps_e2e)
        wk2 = s2.wake()[0]
        out[:] = wk2
        t1 = time.perf_counter()
        twx, twy = s2.transverse_wake() if args.check else (None, None)
        s2.close()
        e2e_s = dist.max(t1 - t0)
        h2d = int(pinned.nbytes if pinned is not None else 0)
        e2e = {"value": world * w.cells * steps_e2e / e2e_s / 1e9, "unit": UNIT,
               "active_gcell_updates_s": world * act * steps_e2e / e2e_s / 1e9,
               "h2d_bytes_per_step": h2d / steps_e2e, "d2h_bytes_per_step": out.nbytes / steps_e2e,
               "h2d_bytes_per_call": h2d, "d2h_bytes_per_call": int(out.nbytes), "steps_per_call": steps_e2e,
               "seconds": round(e2e_s, 3),
               "call": "tetm_create(host pec) + tetm_set_bunch + tetm_set_balance_every + tetm_step + "
                       "tetm_wake(host)"}
        if args.check and w.precision == "fp32" and steps_e2e == w.steps:
            # the same full solve with float64 fields (observer on the bunch
            # line), every wake's error relative to its peak
            r = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", eps_r=args.eps,
                            pec=w.pec)
            r.set_bunch(w.sigma, w.charge, w.i0, w.j0)
            r.set_observer(w.i0, w.j0)
            r.step(steps_e2e)
            rl = r.wake()[0]
            rx, ry = r.transverse_wake()
            r.close()

            def rel(a, b):
                return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
            e2e["wake_error_vs_fp64"] = {"longitudinal": rel(wk2, rl), "transverse_x": rel(twx, rx),
                                         "transverse_y": rel(twy, ry)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    value = world * w.cells * K / (max_ms * 1e-3) / 1e9
    n_bal = len(bal_steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT,
        "active_gcell_updates_s": world * act * K / (max_ms * 1e-3) / 1e9,
        "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz,
                   "dx_mm": round(w.dx * 1e3, 4), "dz_mm": w.dz * 1e3, "cdt": "dz",
                   "sigma_dz": round(w.sigma / w.dz, 3), "fields": w.precision,
                   "wake_and_balances": "f64", "balance_every": be, "kernel": args.kernel,
                   "tiling": [info["tile_x"], info["tile_y"], info["chunk_z"]],
                   "work_items": info["work_items"], "cells": w.cells,
                   "active_cells": info["active_cells"], "processed_cells": proc,
                   "l2": "inputs larger than L2 (two field sets of %.1f GB each)"
                         % (12 * esz * w.cells / 2 / 1e9),
                   "parallelism": "replicas x%d" % world},
        "roofline": dict(roof, achieved=achieved, peak=peak, frac=achieved / peak, traffic=traffic,
                         peak_kind=peak_kind, kernel=kname, kernel_ms=kern_ms,
                         cells_per_launch=proc),
        "cpu_baseline": cpu,
        "e2e": e2e,
        # per balance: the bunch charge, the one fused pass and its second
        # reduction pass (one material); energy and charge passes separately
        # (material arrays)
        "gpu_launches": ((10 * K if args.kernel == "reference" else (K // 2 if args.kernel == "twostep" else K))
                         + (3 if args.eps is None else 6) * n_bal),
        "clocks": clk,
        "balances": {"records": int(hist.shape[0]), "in_timed_region": n_bal,
                     "ms_per_balance": bal_ms,
                     "amortised_ms_per_step": bal_ms / be if be > 0 else 0.0,
                     "share_of_step": (bal_ms / be) / (plain_ms + bal_ms / be) if be > 0 else 0.0,
                     "max_charge_residual_rel": float(np.max(hist[:, 2] / np.maximum(hist[:, 4], 1e-300)))
                     if hist.shape[0] else None,
                     "energy_last_J": float(hist[-1, 1]) if hist.shape[0] else None},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


# ---------------------------------------------------------------------------
# Batched and served workloads (independent solves)
# ---------------------------------------------------------------------------
def _rel(a, b):
    import numpy as np
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def run_batch_mode(args):
    """64 seeded pipe/cavity solves N x N x 4N, N ~ U{32..192}, sigma ~ U[3,10] dz:
    one FP32 batch (autotuned tile, CUDA-graph runs) against the single-solve
    FP64 path, each solve alone in turn."""
    from paper_0901_1053_gb300 import workloads as wl, sharding
    from paper_0901_1053_gb300.autotune import Autotuner
    from paper_0901_1053_gb300.batching import run_batch, run_sequential
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world)
    allw = wl.batch_solves(count=args.solves)
    ws = sharding.shard_workloads(allw, world, rank)
    big = max(ws, key=lambda w: w.cells)
    tuner = Autotuner()
    t32 = tuple(int(x) for x in args.tiling.split(",")) if args.tiling else tuner.tune(big, "fp32", batch=True)
    t64 = tuner.tune(big, "fp64")
    dist.barrier()
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    bstats = {}
    wakes32, t_step, t_total = run_batch(ws, "fp32", t32, graph_steps=32, stats=bstats)
    clk = clocks.stop()
    wakes64, t_seq64 = run_sequential(ws, "fp64", t64)
    err = max(_rel(a, b) for a, b in zip(wakes32, wakes64))
    cs = sum(w.cells * w.steps for w in ws)
    t_step, t_total, t_seq64 = dist.max(t_step), dist.max(t_total), dist.max(t_seq64)
    cs_all = sum(w.cells * w.steps for w in allw)
    line = {"metric": METRIC, "value": cs_all / t_step / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": max(w.steps for w in allw), "warmup": 0, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_%d_pipe_cavity_seed9011053" % len(allw),
                       "n_range": [min(w.nx for w in allw), max(w.nx for w in allw)],
                       "tiling_fp32": list(t32), "tiling_fp64": list(t64), "graph_steps": 32,
                       "cell_steps": cs_all},
            "active_gcell_updates_per_s": dist.sum(bstats["active_cell_steps"]) / t_step / 1e9,
            "solves_per_s": len(allw) / t_total,
            "fp64_single_solve_path_solves_per_s": len(allw) / t_seq64,
            "max_wake_err_vs_fp64_rel_peak": err,
            "e2e": {"value": cs_all / t_total / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(w.pec.nbytes for w in allw)),
                    "d2h_bytes_per_step": int(sum(8 * len(x) for x in wakes32)),
                    "seconds": t_total},
            "seconds": {"batch_steps": t_step, "batch_total": t_total, "fp64_sequential": t_seq64},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def run_serve_mode(args):
    """Poisson stream of solve requests (N ~ U{48..256}, N x N x 4N, pipe /
    cavity / collimator, sigma ~ U[3,10] dz) served with continuous batching
    under a 150 GB device-memory budget: a 64-slot batch advanced in calls of
    round_steps steps, geometry and solve creation and the read-back of
    finished wakes on two worker threads."""
    import numpy as np
    import torch
    from paper_0901_1053_gb300 import workloads as wl, tetm
    from paper_0901_1053_gb300.serve import GpuBackend, Server, latency_stats
    from paper_0901_1053_gb300.autotune import Autotuner
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    reqs = wl.request_stream(count=args.requests, rate=args.rate)
    probe = max(reqs[:32], key=lambda r: r.n).workload("fp32")
    tiling = (tuple(int(x) for x in args.tiling.split(",")) if args.tiling
              else Autotuner().tune(probe, "fp32", batch=True))
    rs = args.round_steps
    be = GpuBackend("fp32", tiling, max_slots=64, round_steps=rs, pool_bytes=150e9)
    srv = Server(be, hbm_budget=150e9, max_slots=64, round_steps=rs, queue_ahead=2, workers=2)
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    res = srv.run_stream(reqs, lambda r: r.spec("fp32"))
    clk = clocks.stop()
    srv.close()
    be.close()
    st = latency_stats(res)
    # accuracy of a sample of served wakes against the FP64 path
    errs = []
    for r in reqs[:6]:
        w = r.workload("fp64")
        s = tetm.Solver.from_workload(w)
        s.step(w.steps)
        errs.append(_rel(res[r.rid].wake, s.wake()[0]))
        s.close()
    mk = st.get("makespan_s")
    line = {"metric": "served solves/s", "value": st.get("solves_per_s"), "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serve_poisson_%d_at_%g_per_s_seed9011054" % (args.requests, args.rate),
                       "hbm_budget_gb": 150, "max_slots": 64, "round_steps": rs, "queue_ahead": 2,
                       "workers": 2, "tiling": list(tiling)},
            "latency": {"p50_s": st.get("p50_s"), "p99_s": st.get("p99_s"), "mean_s": st.get("mean_s")},
            "gcell_updates_per_s": st.get("cell_steps", 0) / mk / 1e9 if mk else None,
            "max_active": srv.max_active, "rounds": srv.rounds,
            "makespan_s": mk, "gpu_busy_s": srv.busy_s, "idle_no_request_s": srv.idle_s,
            "gpu_idle_with_requests_s": (mk - srv.busy_s - srv.idle_s) if mk else None,
            "status_counts": {k: st[k] for k in ("ok", "rejected", "cancelled", "error")},
            "max_wake_err_vs_fp64_rel_peak_sample6": max(errs) if errs else None,
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Rotationally symmetric scheme (Eq. (24)): nine-cell chain, modes 0..4
# ---------------------------------------------------------------------------
def rz_workload(args):
    from paper_0901_1053_gb300 import workloads as wl
    return wl.cavity_chain_rz(nz=args.nz or 16384, precision=args.precision or "fp32")


def rz_start(s, w, start):
    """Starts the bunch; returns the steps of a full solve (the wake window
    complete)."""
    K = 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2
    if start == "cold":
        s.set_bunch(w.sigma, w.charge, w.i0)
        return w.steps
    if start == "static":
        s.set_bunch_static(w.sigma, w.charge, w.i0, K)
    else:
        s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
    return w.steps - K


def rz_source_launches(start, warmup, steps, stride, slots=8):
    """Source launches of the scattered form among `steps` steps taken after
    `warmup` (one launch computes the sources of `slots` steps)."""
    if start != "scattered":
        return 0
    n = until = 0
    count = 0
    for t in range(warmup + steps):
        if t < n:
            continue
        p = stride if t + stride <= warmup + steps else 1
        if n + p > until:
            until = n + slots
            if n >= warmup:
                count += 1
        n += p
    return count


def rz_oracle_sample(w, planes, steps):
    import dataclasses
    from oracle import RzOracle
    sub = dataclasses.replace(w, nz=planes, pec=w.pec[:planes].copy())
    os_ = []
    for m in range(w.m_lo, w.m_hi + 1):
        o = RzOracle(sub.nr, sub.nz, m, sub.dr, sub.dz, sub.cdt, pec=sub.pec)
        o.set_bunch(sub.sigma, sub.charge, sub.i0)
        os_.append(o)
    t0 = time.perf_counter()
    for o in os_:
        o.step(steps)
    dt = time.perf_counter() - t0
    cells = w.n_modes * sub.nr * sub.nz
    desc = ("modes %d..%d, first %d of %d planes of %s (same radial grid and geometry), "
            "%d steps, FP64, 1 thread" % (w.m_lo, w.m_hi, planes, w.nz, w.name, steps))
    return cells * steps / dt / 1e9, dt, desc


def run_rz_mode(args):
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world)
    from paper_0901_1053_gb300 import tetm
    w = rz_workload(args)
    stream = torch.cuda.Stream()
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, w.precision, pec=w.pec)
    full_steps = rz_start(s, w, args.rz_start)
    s.set_stream(stream.cuda_stream)
    if args.rz_chunk and args.rz_kernel:
        kern, chunk = args.rz_kernel, args.rz_chunk
    else:
        from paper_0901_1053_gb300.autotune import tune_rz
        kern, chunk = tune_rz(w)
        kern = args.rz_kernel or kern
        chunk = args.rz_chunk or chunk
    s.set_kernel(kern)
    s.set_tiling(chunk)
    info = s.info()
    s.step(args.warmup)
    s.sync()
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.5)
    # the two-steps-per-pass kernel advances pairs of steps per launch
    stride = 2 if kern == "bulk2" else 1
    K = args.steps - args.steps % stride
    R = K // stride
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(R + 1)]
    dist.barrier()
    torch.cuda.synchronize()
    for i in range(R):
        evs[i].record(stream)
        s.step(stride)
    evs[R].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    total_ms = evs[0].elapsed_time(evs[R])
    per = [evs[i].elapsed_time(evs[i + 1]) / stride for i in range(R)]
    kern_ms = statistics.mean(per)
    max_ms = dist.max(total_ms)
    esz = 4 if w.precision == "fp32" else 8
    bytes_per_cell = 12 * esz + 1
    proc = info["processed_cells"]
    kname = {"async": "rz_step_async_kernel", "bulk": "rz_step_bulk_kernel",
             "bulk2": "rz_step_bulk2_kernel"}.get(kern, "rz_step_kernel")
    launch_ms = kern_ms * stride           # one launch reads y^n and writes y^{n+stride}
    if w.precision == "fp32":
        achieved = bytes_per_cell * proc / (launch_ms * 1e-3) / 1e9
        peak, peak_kind = measured_peak_hbm()
        roof = {"bound": "hbm", "unit": "GB/s", "bytes_per_cell": bytes_per_cell,
                "steps_per_launch": stride, "launch_ms": launch_ms}
    else:
        # float64 arithmetic sets the pace on this part: 47 flops per entry
        # and step (the ten updates, a fused multiply-add counted as two)
        achieved = RZ_FLOPS_PER_CELL * proc / (kern_ms * 1e-3) / 1e12
        peak, peak_kind = fp64_peak(tetm)
        roof = {"bound": "alu", "unit": "TFLOP/s", "flops_per_cell": RZ_FLOPS_PER_CELL,
                "hbm_gbs": bytes_per_cell * proc / (kern_ms * 1e-3) / 1e9}
    traffic = profiled_traffic("%s_%s_%s.md" % (kname, w.precision, w.name), ("rz.cu",))
    s.close()

    e2e = None
    if not args.no_e2e:
        steps_e2e = args.e2e_steps or full_steps
        pinned = torch.empty(w.pec.shape, dtype=torch.uint8, pin_memory=True).numpy()
        pinned[...] = w.pec
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, w.precision, pec=pinned)
        rz_start(s2, w, args.rz_start)
        s2.set_kernel(kern)
        s2.set_tiling(chunk)
        s2.step(steps_e2e)
        wakes = [s2.wake(m)[0] for m in range(w.m_lo, w.m_hi + 1)]
        t1 = time.perf_counter()
        twakes = [s2.transverse_wake(m) for m in range(w.m_lo, w.m_hi + 1)]
        s2.close()
        e2e_s = dist.max(t1 - t0)
        e2e = {"value": world * w.cells * steps_e2e / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(pinned.nbytes),
               "d2h_bytes_per_step": int(sum(x.nbytes for x in wakes)), "steps_per_call": steps_e2e,
               "seconds": round(e2e_s, 3),
               "call": "tetm_rz_create(host pec) + tetm_rz_set_bunch%s + tetm_rz_step + tetm_rz_wake(host)"
                       % ("" if args.rz_start == "cold" else "_" + args.rz_start)}
        if args.rz_check and w.precision == "fp32" and steps_e2e == full_steps:
            # every wake of the float32 solve against the float64 total-field
            # static start (same physics in exact arithmetic for the static
            # and scattered starts; the cold start is checked against a cold
            # float64 solve)
            r = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp64", pec=w.pec)
            rz_start(r, w, "cold" if args.rz_start == "cold" else "static")
            r.set_kernel("bulk")
            r.set_tiling(32)
            r.step(steps_e2e)
            err = []
            for i, m in enumerate(range(w.m_lo, w.m_hi + 1)):
                ref, tref = r.wake(m)[0], r.transverse_wake(m)
                err.append({"m": m,
                            "longitudinal": float(np.max(np.abs(wakes[i] - ref)) / np.max(np.abs(ref))),
                            "transverse": float(np.max(np.abs(twakes[i] - tref)) / np.max(np.abs(tref)))})
            r.close()
            e2e["wake_error_vs_fp64"] = err

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, desc = rz_oracle_sample(w, min(w.nz, 1024), 60)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(dt, 2), "host": host_cpu()}
    value = world * w.cells * K / (max_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nr": w.nr, "nz": w.nz, "modes": [w.m_lo, w.m_hi],
                   "dr_mm": w.dr * 1e3, "dz_mm": w.dz * 1e3, "cdt": "dz",
                   "sigma_dz": round(w.sigma / w.dz, 3), "bunch_ring_i0": w.i0,
                   "fields": w.precision, "wake": "f64", "chunk_z": chunk, "kernel": kern,
                   "start": args.rz_start,
                   "work_items": info["work_items"], "cells": w.cells, "processed_cells": proc,
                   "l2": "inputs larger than L2 (two field sets of %.1f GB each)"
                         % (6 * esz * w.cells / 1e9),
                   "parallelism": "replicas x%d" % world},
        "roofline": dict(roof, achieved=achieved, peak=peak, frac=achieved / peak, traffic=traffic,
                         peak_kind=peak_kind, kernel=kname, kernel_ms=kern_ms,
                         cells_per_launch=proc),
        "cpu_baseline": cpu,
        "e2e": e2e,
        # per pass: the plain step kernel, plus in the scattered form the same
        # kernel over the items meeting the source window, and the sources
        "gpu_launches": R * (2 if args.rz_start == "scattered" else 1)
                        + rz_source_launches(args.rz_start, args.warmup, K, stride),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def run_rz_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = rz_workload(args)
    budget = 2.0e7 * 120.0 / max(1, args.steps + args.warmup)
    planes = int(max(2, min(w.nz, budget // (w.n_modes * w.nr))))
    import dataclasses
    from oracle import RzOracle
    sub = dataclasses.replace(w, nz=planes, pec=w.pec[:planes].copy())
    os_ = []
    for m in range(w.m_lo, w.m_hi + 1):
        o = RzOracle(sub.nr, sub.nz, m, sub.dr, sub.dz, sub.cdt, pec=sub.pec)
        o.set_bunch(sub.sigma, sub.charge, sub.i0)
        o.step(args.warmup)
        os_.append(o)
    t0 = time.perf_counter()
    for o in os_:
        o.step(args.steps)
    dt = time.perf_counter() - t0
    v = w.n_modes * sub.nr * planes * args.steps / dt / 1e9
    desc = "modes %d..%d, first %d of %d planes of %s, %d timed steps, FP64, 1 thread" % (
        w.m_lo, w.m_hi, planes, w.nz, w.name, args.steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "sample_planes": planes},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Yee's scheme (Sec. 3, Eq. (7)) beside the TE/TM scheme
# ---------------------------------------------------------------------------
def yee_cdt(w):
    """The step bound of Yee's scheme, Eq. (8): (dx^-2 + dy^-2 + dz^-2)^-1/2."""
    return 1.0 / math.sqrt(w.dx ** -2 + w.dy ** -2 + w.dz ** -2)


def yee_initial_ex(w):
    """A smooth pulse of e_x along z (canonical layout; the library drops it on
    entries that carry no field). Field-only runs need some initial field."""
    import numpy as np
    k = np.arange(w.nz + 1, dtype=np.float64)
    prof = np.exp(-((k - w.nz / 4.0) / 20.0) ** 2)
    return np.ascontiguousarray(np.broadcast_to(prof[:, None, None], (w.nz + 1, w.ny + 1, w.nx + 1)))


def yee_z_dispersion(tetm, travel=1500, sigma_cells=6.0, n=24, nz=2048):
    """The z-dispersion of both schemes on the GPU (float64): a Gaussian TEM pulse
    (RMS sigma_cells) on a coaxial line n x n x nz (a 4 x 4-cell PEC rod on the axis,
    the paper's sqrt(2) mesh), moved `travel` cells by each scheme at its step
    (TE/TM c*dt = dz, Yee at its bound (8)), against the dispersion-free motion of
    the same initial field: each standing wave sin(r pi k / nz) turning at the
    exact frequency c k. Yee's error is also predicted from its dispersion relation
    (10) (the same sum with sin W = (c dt/dz) sin(r pi / (2 nz)))."""
    import numpy as np
    from paper_0901_1053_gb300 import workloads as wl
    dxy, dz = math.sqrt(2.0) * 1e-3, 1e-3
    rod = (n // 2 - 2, n // 2 + 2, n // 2 - 2, n // 2 + 2)
    pec = wl.coax_pec(n, n, nz, rod)
    e0x, e0y = wl.coax_tem_e(n, n, dxy, dxy, rod)
    k = np.arange(nz + 1)
    a0 = np.exp(-0.5 * ((k - 300.0) / sigma_cells) ** 2)
    a0[0] = a0[-1] = 0.0
    r = np.arange(1, nz)
    modes = np.sin(np.pi * np.outer(r, k) / nz)
    amp = (2.0 / nz) * modes @ a0
    jj, ii = np.unravel_index(np.argmax(np.abs(e0x)), e0x.shape)
    out = {"line": "%dx%dx%d coaxial line, 4x4-cell rod, dx = dy = sqrt(2) dz" % (n, n, nz),
           "pulse_sigma_cells": sigma_cells, "travel_cells": travel, "fields": "f64"}
    for scheme in ("tetm", "yee"):
        cdt = dz if scheme == "tetm" else 1.0 / math.sqrt(2.0 / dxy ** 2 + 1.0 / dz ** 2)
        nu = cdt / dz
        steps = int(round(travel / nu))
        s = tetm.Solver(n, n, nz, dxy, dxy, dz, cdt, "fp64", pec=pec)
        if scheme == "yee":
            s.set_scheme("yee")
        s.set(0, e0x[None] * a0[:, None, None])
        s.set(1, e0y[None] * a0[:, None, None])
        s.step(steps)
        a = s.get(0)[:, jj, ii] / e0x[jj, ii]
        s.close()
        # e^0 and h^{-1/2} = 0 (TE/TM: e at integer times) or e^{-1/2} and h^0 = 0
        # (Yee): each standing wave a_r(t) = A_r cos(omega (t + 1/2)) / cos(omega / 2)
        # or cos(omega t) / cos(omega / 2) at the e time level reached
        m = 2 * steps + 1 if scheme == "tetm" else 2 * steps - 1
        w_exact = nu * np.pi * r / (2 * nz)
        exact = (amp * np.cos(m * w_exact) / np.cos(w_exact)) @ modes
        d = {"cdt_over_dz": round(nu, 6), "steps": steps,
             "max_error_vs_dispersion_free": float(np.max(np.abs(a - exact)) / np.max(np.abs(a0)))}
        if scheme == "yee":
            w = np.arcsin(nu * np.sin(np.pi * r / (2 * nz)))
            pred = (amp * np.cos(m * w) / np.cos(w)) @ modes
            d["predicted_by_eq10"] = float(np.max(np.abs(pred - exact)) / np.max(np.abs(a0)))
            d["max_error_vs_eq10"] = float(np.max(np.abs(a - pred)) / np.max(np.abs(a0)))
        out[scheme] = d
    return out


def run_yee_mode(args):
    """Yee's scheme on the workload's grid at c*dt = the bound (8), one fused
    launch per step, and the TE/TM scheme (c*dt = dz) on the same grid and
    initial field timed beside it: kernel time per step and per dz of simulated
    length (the paper's cost comparison of Sec. 1 and Sec. 4.2)."""
    rank, world, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world)
    from paper_0901_1053_gb300 import tetm
    w = make_workload(args)
    if args.eps is not None:
        raise SystemExit("--scheme yee times the uniform-material workloads")
    cdt = yee_cdt(w)
    stream = torch.cuda.current_stream()
    ex0 = yee_initial_ex(w)
    K = args.steps

    def make(scheme):
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, cdt if scheme == "yee" else w.cdt,
                        w.precision, pec=w.pec)
        if scheme == "yee":
            s.set_scheme("yee")
        s.set_kernel(args.kernel)
        s.set(0, ex0)
        s.set_stream(stream.cuda_stream)
        return s

    def timed(s, clocks=None):
        s.step(args.warmup)
        s.sync()
        if clocks:
            clocks.start()
            time.sleep(0.5)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        dist.barrier()
        torch.cuda.synchronize()
        for i in range(K):
            evs[i].record(stream)
            s.step(1)
        evs[K].record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        clk = clocks.stop() if clocks else None
        total = evs[0].elapsed_time(evs[K])
        return total, total / K, clk

    zdisp = yee_z_dispersion(tetm) if rank == 0 else None

    # the TE/TM scheme first (no balances: kernel against kernel)
    st = make("tetm")
    info_t = st.info()
    _, tetm_ms, _ = timed(st)
    st.close()

    s = make("yee")
    info = s.info()
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    total_ms, kern_ms, clk = timed(s, ClockSampler(uuid))
    max_ms = dist.max(total_ms)
    s.close()

    esz = 4 if w.precision == "fp32" else 8
    bytes_per_cell = 12 * esz + 1
    proc = info["processed_cells"] if args.kernel != "reference" else w.cells
    gbs = bytes_per_cell * proc / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    kname = "yee_fused" if args.kernel != "reference" else "yee_reference"
    traffic = (profiled_traffic("%s_%s_%s.md" % (kname, w.precision, w.name), ("kernels_yee.cu",))
               if args.kernel != "reference" else None)

    e2e = None
    if not args.no_e2e:
        steps_e2e = args.e2e_steps or int(math.ceil(w.steps * w.dz / cdt))
        pinned = torch.empty(w.pec.shape, dtype=torch.uint8, pin_memory=True).numpy()
        pinned[...] = w.pec
        ex_h = torch.empty(ex0.shape, dtype=torch.float64, pin_memory=True).numpy()
        ex_h[...] = ex0
        out = torch.empty(ex0.shape, dtype=torch.float64, pin_memory=True).numpy()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, cdt, w.precision, pec=pinned)
        s2.set_scheme("yee")
        s2.set_kernel(args.kernel)
        s2.set(0, ex_h)
        s2.step(steps_e2e)
        out[...] = s2.get(2)
        t1 = time.perf_counter()
        s2.close()
        e2e_s = dist.max(t1 - t0)
        e2e = {"value": world * w.cells * steps_e2e / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(pinned.nbytes + ex_h.nbytes), "d2h_bytes_per_step": int(out.nbytes),
               "steps_per_call": steps_e2e, "seconds": round(e2e_s, 3),
               "call": "tetm_create(host pec) + tetm_set_scheme(yee) + tetm_set_fields(ex, host) + "
                       "tetm_step + tetm_get_fields(ez, host); the TE/TM solve's simulated length"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, desc = yee_oracle_sample(w, min(w.nz, 256), 20 if w.nx * w.ny >= 256 * 256 else 400)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(dt, 2), "host": host_cpu()}

    yee_per_dz = kern_ms * w.dz / cdt
    line = {
        "metric": METRIC, "value": world * w.cells * K / (max_ms * 1e-3) / 1e9, "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": max_ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if w.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": w.name, "scheme": "yee (Eq. (7))", "nx": w.nx, "ny": w.ny, "nz": w.nz,
                   "dx_mm": round(w.dx * 1e3, 4), "dz_mm": w.dz * 1e3,
                   "cdt_over_dz": round(cdt / w.dz, 6), "cdt": "Eq. (8) bound", "fields": w.precision,
                   "kernel": args.kernel, "tiling": [info["tile_x"], info["tile_y"], info["chunk_z"]],
                   "work_items": info["work_items"], "cells": w.cells, "processed_cells": proc,
                   "l2": "inputs larger than L2 (two field sets of %.1f GB each)"
                         % (12 * esz * w.cells / 2 / 1e9),
                   "parallelism": "replicas x%d" % world},
        "roofline": {"bound": "hbm", "unit": "GB/s", "bytes_per_cell": bytes_per_cell, "achieved": gbs,
                     "peak": peak, "frac": gbs / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": kname, "kernel_ms": kern_ms, "cells_per_launch": proc},
        "versus_tetm": {"tetm_kernel_ms_per_step": tetm_ms, "tetm_cdt_over_dz": 1.0,
                        "tetm_tiling": [info_t["tile_x"], info_t["tile_y"], info_t["chunk_z"]],
                        "yee_kernel_ms_per_step": kern_ms,
                        "tetm_ms_per_dz": tetm_ms, "yee_ms_per_dz": yee_per_dz,
                        "tetm_time_over_yee_time": tetm_ms / yee_per_dz},
        "z_dispersion": zdisp,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": K if args.kernel != "reference" else 2 * K,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def yee_oracle_sample(w, planes, steps):
    import dataclasses
    from oracle import Oracle
    sub = dataclasses.replace(w, nz=planes, pec=None if w.pec is None else w.pec[:planes].copy())
    o = Oracle(sub.nx, sub.ny, sub.nz, sub.dx, sub.dy, sub.dz, yee_cdt(w), pec=sub.pec)
    o.set(0, yee_initial_ex(sub))
    t0 = time.perf_counter()
    o.yee_step(steps)
    dt = time.perf_counter() - t0
    cells = sub.nx * sub.ny * sub.nz
    return cells * steps / dt / 1e9, dt, "Yee's scheme on the first %d of %d planes of %s, %d steps, " \
        "FP64, 1 thread" % (planes, w.nz, w.name, steps)


def run_yee_reference(args):
    """The oracle's Yee scheme on a bounded sample of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args)
    budget_cells = 2.0e7 * 120.0 / max(1, args.steps + args.warmup)
    planes = int(max(2, min(w.nz, budget_cells // (w.nx * w.ny))))
    v, dt, desc = yee_oracle_sample(w, planes, args.steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "scheme": "yee (Eq. (7))",
                                            "sample_planes": planes},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        if args.scheme == "yee":
            return run_yee_reference(args)
        return run_rz_reference(args) if args.workload == "rz" else run_reference(args)
    if args.scheme == "yee":
        return run_yee_mode(args)
    if args.workload == "rz":
        return run_rz_mode(args)
    if args.workload == "batch":
        return run_batch_mode(args)
    if args.workload == "serve":
        return run_serve_mode(args)
    return run_tetm(args)


if __name__ == "__main__":
    sys.exit(main())
