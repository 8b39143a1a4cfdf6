"""Benchmark: gradient throughput of the time-reversible FDTD on one or more GPUs.

One step = one forward run (n_steps leapfrog steps recording the compressed
boundary tape) plus one backward run (time-reversed interior, tape restore,
adjoint, dL/d(eps)) of the waveguide workload: 200 x 200 x 100 cells at
20 nm, 12-cell CPML, 2000 steps, BF16 tape every 4th step with linear
interpolation.  Metric: cell-updates per second of the whole gradient,
nx*ny*nz*n_steps / (T_forward + T_backward), cells including the CPML.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload waveguide200|waveguide600|batched64] [--n-steps N]

N > 1 runs under torchrun: every rank computes its own design (independent
problems, no data-path collective) and rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host cores instead.

Other workloads (not the default line): waveguide600 = 600 x 600 x 300 cells
at 10 nm, 16-cell CPML (10000 steps unless --n-steps); batched64 = 64
independent vacuum cubes of 32..128 cells with 600..1500 steps each, run
concurrently through the group calls (one step = one group forward + one
group backward of all 64).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "fwd+reverse grad Gcell-updates/s & HBM roofline %; tape bytes at stated grad err"
UNIT = "Gcell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--tape", default="bf16:4:linear")
    p.add_argument("--compare-tape", default="f32:1:linear")
    p.add_argument("--kernel", type=int, default=-1, help="0 split, 1 fused, -1 library default")
    p.add_argument("--sample-every", type=int, default=50)
    p.add_argument("--zgroups", type=int, default=0,
                   help="z groups per half-step (0: the library's automatic choice)")
    p.add_argument("--autotune", action="store_true",
                   help="tune the launch shapes first (autotune.tune, cached per GPU type)")
    p.add_argument("--cpu-sample-steps", type=int, default=24)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true")
    p.add_argument("--workload", default="waveguide200",
                   choices=["waveguide200", "waveguide600", "batched64"])
    p.add_argument("--n-steps", type=int, default=0, help="override the workload's step count")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over all ranks (the slowest rank's time); the
    process group must be initialised when ws > 1."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, cell_updates: int, steps: int, seconds: float) -> float:
    """Whole-job Gcell-updates/s: every rank runs its own replica of the
    workload (weak scaling), timed by the slowest rank."""
    return ws * cell_updates * steps / seconds / 1e9


def workload(rank: int, n_steps=None, name: str = "waveguide200"):
    from paper_2603_24027_gb300 import inputs as I
    w = I.waveguide_large(seed=rank) if name == "waveguide600" else I.waveguide_mid(seed=rank)
    return w if not n_steps else w.replace(n_steps=n_steps)


# ------------------------------------------------------------ roofline ---

def cell_classes(w):
    """Counts of cells by (interior?, number of CPML slab axes, in design box?)."""
    P = w.pml_thickness
    ax = []
    for n in (w.nx, w.ny, w.nz):
        s = np.zeros(n, np.int64)
        s[:P] = 1
        s[n - P:] = 1
        ax.append(s)
    slabs = ax[2][:, None, None] + ax[1][None, :, None] + ax[0][None, None, :]
    design = np.zeros(w.shape, bool)
    design[w.design_slice()] = True
    interior = slabs == 0
    return dict(interior=int(interior.sum()), design=int(design.sum()),
                slab_axes=int(slabs.sum()), cells=w.n_cells)


def algorithmic_bytes(w):
    """Minimum HBM bytes per launch of each kernel kind (FP32 = 4 B, FP64 accumulator 8 B).
    Split kernels move one field family per launch; fused kernels read the
    state once and write it once (ping-pong)."""
    c = cell_classes(w)
    n, ni, nd, sa = c["cells"], c["interior"], c["design"], c["slab_axes"]
    npml = n - ni
    return {
        # read E,H; write H (36 B); CPML: 2 psi read + 2 written per slab axis
        "fwd_h": 36 * n + 16 * sa,
        # read H,E,cb; write E (40 B); CPML as above
        "fwd_e": 40 * n + 16 * sa,
        # interior: read H,E,cb,lamE,lamH, write E,lamH (76 B); others 40 B; design 16 B
        "rev_e": 76 * ni + 40 * npml + 16 * nd + 16 * sa,
        # interior: read E,H,lamH,lamE, write H,lamE (72 B); others 36 B
        "rev_h": 72 * ni + 36 * npml + 16 * sa,
        # read E,H,cb, write E,H (52 B); 4 psi read + 4 written per slab axis
        "fused_fwd": 52 * n + 32 * sa,
        # interior: primal 12+12... read E,H,lamE,lamH,cb, write E,H,lamE,lamH (100 B);
        # CPML-side cells adjoint only (52 B); design +16 B; psi 32 B per slab axis
        "fused_rev": 100 * ni + 52 * npml + 16 * nd + 32 * sa,
    }


def tape_values(w):
    """Values of one tape sample: two tangential components on six faces."""
    P = w.pml_thickness
    a, b, c = w.nx - 2 * P, w.ny - 2 * P, w.nz - 2 * P
    return 4 * (b * c + a * c + a * b)


def record_bytes(w, dtype_bytes):
    """One record launch: read every face value (FP32), write its code."""
    return tape_values(w) * (4 + dtype_bytes)


def restore_bytes(w, dtype_bytes, terms):
    """One restore launch: read `terms` samples' codes per face value, write
    the FP32 value; plus the detector seed (read E, H; read and write the
    adjoint) on the detector window."""
    det = (w.det_hi[0] - w.det_lo[0]) * (w.det_hi[1] - w.det_lo[1])
    return tape_values(w) * (terms * dtype_bytes + 4) + det * 4 * 12


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(kernel: str, digest: str, workload: str = "waveguide200"):
    """ncu DRAM bytes per launch recorded for this kernel build, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] == digest and parts[2] == workload:
                return float(parts[3])
    return None


# -------------------------------------------------------------- clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.err = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception as e:  # nvidia-smi missing
            self.err = str(e)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if self.err or not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "note": self.err or "no nvidia-smi samples"}
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names[1:], p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for_smi(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts):
            return parts[local_rank].strip()
    return str(local_rank)


# ---------------------------------------------------------------- ours ---

def tape_cfg(A, spec: str):
    dt, k, interp = spec.split(":")
    return A.record_cfg(dt, int(k), interp)


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2603_24027_gb300 import build as B
    B.build()
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import fdtd

    w = workload(rank, args.n_steps, args.workload)
    rec = tape_cfg(A, args.tape)
    sim = fdtd.Simulation(w, device=dev)
    if args.kernel >= 0:
        sim.set_option(A.OPT_KERNEL, args.kernel)
    sim.set_option(A.OPT_ZGROUPS, args.zgroups)
    eps = torch.from_numpy(w.eps).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned = None
    if args.autotune:
        from paper_2603_24027_gb300 import autotune
        tuned = autotune.tune(sim, eps, rec)

    def barrier():
        if ws > 1:
            dist.barrier()

    def step(s, r):
        s.forward(eps, r)
        return s.backward(1.0)

    for _ in range(max(3, args.warmup)):
        step(sim, rec)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    fwd_ms, bwd_ms = [], []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(gpu_index_for_smi(local)) as clk:
        for i in range(args.steps):
            flush.random_(0, 255)              # evict L2 (129 MB) before each timed step
            starts[i].record()
            g = step(sim, rec)
            ends[i].record()
            t = sim.last_timing()
            fwd_ms.append(t["fwd_ms"])
            bwd_ms.append(t["bwd_ms"])
        torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    launches = sim.last_timing()
    gpu_launches = (launches["fwd_launches"] + launches["bwd_launches"] + 2) * args.steps
    cell_updates = w.n_cells * w.n_steps
    value = job_rate(ws, cell_updates, args.steps, total_ms / 1e3)

    # Per-kernel live timing.  The timed steps run the default schedule, whose
    # half-steps are split into z groups on several streams that overlap, so a
    # launch has no duration of its own there; the per-kernel costs come from a
    # sampled pass of the same steps with one launch per half-step (CUDA events
    # on the library stream, pair-minus-single intervals) right after them.
    zgroups_timed = sim.get_option(A.OPT_ZGROUPS)
    sim.set_option(A.OPT_ZGROUPS, 1)
    sim.set_option(A.OPT_SAMPLE_EVERY, args.sample_every)
    step(sim, rec)                                 # capture the sampled graphs
    torch.cuda.synchronize()
    ktimes, one_ms = {}, []
    for i in range(max(2, min(args.steps, 4))):
        flush.random_(0, 255)
        step(sim, rec)
        t = sim.last_timing()
        one_ms.append(t["fwd_ms"] + t["bwd_ms"])
        for name, (ms, n) in sim.kernel_timing().items():
            ktimes.setdefault(name, []).append((ms, n))
    torch.cuda.synchronize()
    sim.set_option(A.OPT_ZGROUPS, zgroups_timed)
    sim.set_option(A.OPT_SAMPLE_EVERY, 0)
    one_step_ms = statistics.median(one_ms)
    algo = algorithmic_bytes(w)
    peak, peak_kind = read_peaks()
    per_step = {"fwd_h": w.n_steps, "fwd_e": w.n_steps, "rev_e": w.n_steps, "rev_h": w.n_steps,
                "fused_fwd": w.n_steps, "fused_rev": w.n_steps,
                "record": -(-w.n_steps // rec.k), "restore_seed": w.n_steps}
    dtb = {0: 4, 1: 2, 2: 2}.get(rec.dtype, 1)
    tape_algo = {"record": record_bytes(w, dtb),
                 "restore_seed": restore_bytes(w, dtb, 2 if rec.interp == 0 else 4)}
    kern = {}
    for name, lst in ktimes.items():
        n = sum(c for _, c in lst)
        avg = sum(ms * c for ms, c in lst) / max(n, 1)
        share = avg * per_step[name] / one_step_ms
        d = {"avg_ms": avg, "sampled_launches": n, "share_of_step": share}
        ab = algo.get(name, tape_algo.get(name))
        if ab is not None:
            d["algorithmic_bytes"] = ab
            d["achieved_gbs"] = ab / (avg / 1e3) / 1e9
        kern[name] = d
    dom = max((k for k in kern if k in algo), key=lambda k: kern[k]["share_of_step"])
    digest = B.kernel_digest()
    traffic = read_traffic(dom, digest, args.workload)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved_gbs"],
                "peak": peak, "unit": "GB/s", "frac": kern[dom]["achieved_gbs"] / peak,
                "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": algo[dom],
                "launch_timing": "sampled pass with one launch per half-step, after the timed steps"}
    # the whole step: every kernel's algorithmic bytes over the timed step time
    step_bytes = sum(kern[k]["algorithmic_bytes"] * per_step[k] for k in kern
                     if "algorithmic_bytes" in kern[k])
    roofline["step_achieved"] = step_bytes / (total_ms / args.steps / 1e3) / 1e9
    roofline["step_frac"] = roofline["step_achieved"] / peak

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded waveguide: Si strip in SiO2, smoothed random design)",
        "config": {"workload": w.name, "cells": w.n_cells, "n_steps": w.n_steps,
                   "pml": w.pml_thickness, "tape": args.tape,
                   "design_box": list(w.design_shape[::-1]),
                   "parallelism": f"replicas x{ws}", "l2": "flushed before every timed step",
                   "zgroups": args.zgroups or "automatic (4 forward, 3 reverse)",
                   "autotuned": None if tuned is None else
                   {"options": tuned["options"], "cached": tuned["cached"]},
                   "fwd_ms": statistics.median(fwd_ms), "bwd_ms": statistics.median(bwd_ms),
                   "one_launch_per_half_step_ms": one_step_ms,
                   # forward-only and reverse-only rates (cells x steps / phase time)
                   "fwd_gcell_updates_per_s": w.n_cells * w.n_steps / statistics.median(fwd_ms) / 1e6,
                   "bwd_gcell_updates_per_s": w.n_cells * w.n_steps / statistics.median(bwd_ms) / 1e6,
                   "wall_s": wall},
        "gpu_launches": gpu_launches,
        "roofline": roofline,
        "kernels": kern,
        "clocks": clk.summary(),
        "tape_bytes": sim.tape_bytes(rec),
    }

    # the same code with the uncompressed FP32 tape, and gradient agreement
    if not args.no_compare:
        rec32 = tape_cfg(A, args.compare_tape)
        sim32 = fdtd.Simulation(w, device=dev)
        if args.kernel >= 0:
            sim32.set_option(A.OPT_KERNEL, args.kernel)
        for _ in range(2):
            g32 = step(sim32, rec32)
        torch.cuda.synchronize()
        ts = []
        for i in range(args.steps):
            flush.random_(0, 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g32 = step(sim32, rec32)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        v32 = cell_updates / (sum(ts) / args.steps / 1e3) / 1e9
        g64, g3264 = g.double(), g32.double()
        cosv = float((g64 * g3264).sum() / (g64.norm() * g3264.norm()))
        relv = float((g64 - g3264).norm() / g3264.norm())
        out["compare"] = {"tape": args.compare_tape, "value": v32,
                          "tape_bytes": sim32.tape_bytes(rec32),
                          "tape_reduction": sim32.tape_bytes(rec32) / sim.tape_bytes(rec),
                          "speedup_vs_compare": value / ws / v32,
                          "grad_cosine": cosv, "grad_rel_err": relv}
        del sim32

    # end to end through the public host-buffer call
    eps_h = torch.from_numpy(w.eps).pin_memory()
    grad_h = torch.empty(w.design_shape, dtype=torch.float32).pin_memory()
    sim.value_and_grad_host(eps_h, rec, 1.0, grad_h)
    barrier()
    torch.cuda.synchronize()
    te = []
    for i in range(args.steps):
        flush.random_(0, 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.value_and_grad_host(eps_h, rec, 1.0, grad_h)
        te.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(sum(te), ws, dev)
    nd = int(np.prod(w.design_shape))
    out["e2e"] = {"value": job_rate(ws, cell_updates, args.steps, e2e_t), "unit": UNIT,
                  "h2d_bytes_per_step": w.n_cells * 4, "d2h_bytes_per_step": nd * 4 + 8}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps, args.workload)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------- oracle ---

def oracle_step(n_steps: int, name: str = "waveguide200"):
    from oracle import oracle as O
    w = workload(0, n_steps=n_steps, name=name)
    t0 = time.perf_counter()
    O.gradient(w)
    return time.perf_counter() - t0, w


def cpu_baseline(n_steps: int, name: str = "waveguide200"):
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    if name == "waveguide600":          # 27x the cells: keep the sample at a similar CPU time
        n_steps = max(2, n_steps // 12)
    dt, w = oracle_step(n_steps, name)
    return {"value": w.n_cells * w.n_steps / dt / 1e9, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle gradient (forward + stored-history adjoint) of the same "
                      f"{w.nx}x{w.ny}x{w.nz} workload truncated to {n_steps} steps; {dt:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    n = args.cpu_sample_steps
    for _ in range(max(3, args.warmup)):
        oracle_step(max(2, n // 4))
    ts = []
    for _ in range(args.steps):
        dt, w = oracle_step(n)
        ts.append(dt)
    value = w.n_cells * n * len(ts) / sum(ts) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": 1e3 * sum(ts) / len(ts),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "cells": w.n_cells, "n_steps_sample": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                            "kind": "oracle",
                            "sample": f"each step: FP64 oracle gradient of the 200x200x100 "
                                      f"workload over {n} steps"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(args):
    """64 independent problems on one GPU through the group calls."""
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2603_24027_gb300 import build as B
    B.build()
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import fdtd
    from paper_2603_24027_gb300 import inputs as I

    wl = I.batched_cubes(seed=rank)
    rec = tape_cfg(A, args.tape)
    sims = [fdtd.Simulation(w, device=dev) for w in wl]
    for s in sims:
        s.set_option(A.OPT_ZGROUPS, args.zgroups)
    eps = [torch.from_numpy(w.eps).to(dev) for w in wl]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        fdtd.group_forward(sims, eps, rec)
        return fdtd.group_backward(sims)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ts = []
    with ClockSampler(gpu_index_for_smi(local)) as clk:
        for _ in range(args.steps):
            flush.random_(0, 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
    total_ms = max_over_ranks(sum(ts), ws, dev)
    cell_updates = sum(w.n_cells * w.n_steps for w in wl)
    value = job_rate(ws, cell_updates, args.steps, total_ms / 1e3)
    # aggregate algorithmic bytes of one step (all problems, all launches)
    byts = 0
    for w in wl:
        ab = algorithmic_bytes(w)
        byts += w.n_steps * (ab["fwd_h"] + ab["fwd_e"] + ab["rev_e"] + ab["rev_h"])
    peak, peak_kind = read_peaks()
    achieved = byts / (total_ms / args.steps / 1e3) / 1e9
    launches = sum(s.last_timing()["fwd_launches"] + s.last_timing()["bwd_launches"] + 2
                   for s in sims) * args.steps

    # end to end: eps from pinned host memory in, gradients and objectives out
    eps_h = [torch.from_numpy(w.eps).pin_memory() for w in wl]
    grads_h = [torch.empty(w.design_shape, dtype=torch.float32).pin_memory() for w in wl]
    te = []
    for _ in range(args.steps):
        flush.random_(0, 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, hsrc in zip(eps, eps_h):
            d.copy_(hsrc, non_blocking=True)
        objs = fdtd.group_forward(sims, eps, rec)
        gs = fdtd.group_backward(sims)
        for hdst, g in zip(grads_h, gs):
            hdst.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
        te.append(time.perf_counter() - t0)
    assert all(np.isfinite(objs))
    e2e_t = max_over_ranks(sum(te), ws, dev)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (64 seeded vacuum cubes with random design boxes)",
        "config": {"workload": "batched64", "problems": len(wl),
                   "cells": sum(w.n_cells for w in wl), "cell_updates": cell_updates,
                   "tape": args.tape, "zgroups": args.zgroups or "automatic",
                   "parallelism": f"replicas x{ws}, 64 concurrent problems",
                   "l2": "flushed before every timed step"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": "all kernels, aggregate over 64 concurrent problems",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_step": byts},
        "clocks": clk.summary(),
        "e2e": {"value": job_rate(ws, cell_updates, args.steps, e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": sum(w.n_cells * 4 for w in wl),
                "d2h_bytes_per_step": sum(int(np.prod(w.design_shape)) * 4 + 8 for w in wl)},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
