"""Benchmark: gradient throughput of the time-reversible FDTD on one or more GPUs.

One step = one gradient: a forward run (n_steps leapfrog steps recording the
compressed boundary tape) plus a backward run (time-reversed interior, tape
restore, adjoint, dL/d(eps)) of the workload, through the public host-buffer
call fdtd_value_and_grad_host.  Default workload: the large waveguide, 600 x
600 x 300 cells at 10 nm, 16-cell CPML, 10000 steps, FP8 E4M3 tape with a
per-face scale, every 8th step, linear interpolation (32x smaller than the
FP32 tape of every step).

Metric: cell-updates per second of the whole gradient,
nx*ny*nz*n_steps / T, cells including the CPML.
  value: T = device time of each call between its input copy and its output
         copy (CUDA events on the library's stream; eps already in HBM);
  e2e:   T = wall time of the same calls, host copies included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload waveguide600|waveguide200|batched64] [--n-steps N]
                  [--tape dtype:k:interp] [--no-compare]
  python bench.py --profile-run [--workload ...] [--n-steps N] [launch options]

N > 1 runs under torchrun: every rank computes its own design (independent
problems, no data-path collective) and rank 0 prints one JSON line.
--impl reference times the FP64 CPU oracle on the host cores instead, on a
time-truncated sample of the same workload.

Roofline: the algorithmic bytes of a forward time step (52 B per cell, +32 B
per CPML axis of the cell) and of a reverse time step (100 B per interior
cell, 52 B per CPML cell, +32 B per CPML axis, +16 B per design cell), plus
the tape's codes, over the measured time of one step of that phase; the
reverse phase is the dominant one.  Where the forward runs two time steps per
pass over the deep units (the library's choice on the large grid), its
fraction is an effective one: those units' fields cross DRAM once per two
steps.  The per-kernel breakdown comes from a
sampled pass with one launch per half-step on a shortened copy of the
workload (same grid, same per-launch work).

capacity: the workspace of one problem with this tape and with the
comparison tape, and how many such problems fit side by side in the GPU's
memory (where tape compression pays on one GPU: the FP32 tape of every step
bounds the batch, not the speed).

--profile-run: one short forward + backward for profilers (ncu launch lists,
single-kernel captures) and launch-shape sweeps; prints the timings.

Other workloads: waveguide200 = 200 x 200 x 100 cells at 20 nm, 12-cell CPML,
2000 steps; batched64 = 64 independent vacuum cubes of 32..128 cells with
600..1500 steps each, run concurrently through the group calls (one step =
one group forward + one group backward of all 64); the line also reports
the same designs through the batched calls, one launch per half-step over
all of them (one_launch_per_half_step).
"""
from __future__ import annotations

import argparse
import json
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
DEFAULT_TAPE = {"waveguide600": "e4m3:8:linear", "waveguide200": "e4m3:8:linear",
                "batched64": "bf16:4:linear"}
CPU_SAMPLE_STEPS = {"waveguide600": 2, "waveguide200": 24, "batched64": 24}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="waveguide600",
                   choices=["waveguide600", "waveguide200", "batched64"])
    p.add_argument("--n-steps", type=int, default=0, help="override the workload's step count")
    p.add_argument("--tape", default="", help="dtype:k:interp (default per workload)")
    p.add_argument("--compare-tape", default="f32:1:linear")
    p.add_argument("--no-compare", action="store_true")
    p.add_argument("--compare-steps", type=int, default=1)
    p.add_argument("--kernel", type=int, default=-1, help="0 plain loads, 5 staged, -1 default")
    p.add_argument("--reverse", type=int, default=-1,
                   help="reverse step: 1 split phases, 2 fused, -1 the library's choice")
    p.add_argument("--forward", type=int, default=-1,
                   help="forward step: 1 split half-steps, 2 fused, 3 two time steps per "
                        "pass over the deep units, -1 the library's choice")
    p.add_argument("--zgroups", type=int, default=0,
                   help="z groups per half-step (0: the library's automatic choice)")
    p.add_argument("--autotune", action="store_true",
                   help="tune the launch shapes first (autotune.tune, cached per GPU type)")
    p.add_argument("--sample-steps", type=int, default=400,
                   help="time steps of the sampled per-kernel pass")
    p.add_argument("--sample-every", type=int, default=50)
    p.add_argument("--cpu-sample-steps", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    # --profile-run and its launch options
    p.add_argument("--profile-run", action="store_true")
    p.add_argument("--tile-y", type=int, default=0)
    p.add_argument("--tile-x", type=int, default=0)
    p.add_argument("--zchunk", type=int, default=0)
    p.add_argument("--zchunk-fwd", type=int, default=-2,
                   help="-2: library default, -1: automatic")
    p.add_argument("--zchunk-fwd2", type=int, default=-2,
                   help="planes per CTA of the two-step forward pass (-2: library default)")
    p.add_argument("--stages", type=int, default=0)
    p.add_argument("--pdl", type=int, default=-1)
    p.add_argument("--prefetch", type=int, default=-1)
    p.add_argument("--compact", type=int, default=-1)
    p.add_argument("--pml", type=int, default=0, help="profile run: CPML thickness override")
    p.add_argument("--no-graphs", action="store_true")
    a = p.parse_args(argv)
    if not a.tape:
        a.tape = DEFAULT_TAPE[a.workload]
    if not a.cpu_sample_steps:
        a.cpu_sample_steps = CPU_SAMPLE_STEPS[a.workload]
    return a


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


def workload(rank: int, n_steps=None, name: str = "waveguide600"):
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


def tape_values(w):
    """Values of one tape sample: two tangential components on six faces."""
    P = w.pml_thickness
    a, b, c = w.nx - 2 * P, w.ny - 2 * P, w.nz - 2 * P
    return 4 * (b * c + a * c + a * b)


def code_bytes(spec: str) -> float:
    dt = spec.split(":")[0]
    if dt == "f32":
        return 4.0
    if dt in ("bf16", "f16"):
        return 2.0
    if dt.startswith("bdct"):
        K = int(dt[4:]) if len(dt) > 4 else 10
        return (K + 4) / 64.0
    return 1.0


def phase_bytes(w, tape: str):
    """Algorithmic HBM bytes of one forward and one reverse time step (FP32 =
    4 B): forward 52 B per cell (read E, Ht, cb; write E, Ht) + 32 B per CPML
    axis of the cell (4 auxiliaries read and written); reverse 100 B per
    interior cell (read E, Ht, lamE, lamH, cb; write all four), 52 B per CPML
    cell (adjoint only), + 32 B per CPML axis, + 16 B per design cell (FP64
    accumulator read and write).  The tape adds one sample's codes every k-th
    forward step and, per reverse step, the codes of the samples the
    interpolation reads (2 linear, 4 cubic) and the restored FP32 values."""
    c = cell_classes(w)
    n, ni, nd, sa = c["cells"], c["interior"], c["design"], c["slab_axes"]
    _, k, interp = tape.split(":")
    tv, cbytes = tape_values(w), code_bytes(tape)
    terms = 2 if interp == "linear" else 4
    fwd = 52 * n + 32 * sa + tv * (4 + cbytes) / int(k)
    rev = 100 * ni + 52 * (n - ni) + 32 * sa + 16 * nd + tv * (terms * cbytes + 4)
    return {"forward": fwd, "reverse": rev}


def kernel_bytes(w):
    """Per-launch bytes each split half-step kernel moves itself (its own
    reads and writes), for the per-kernel breakdown only: the split reverse
    reads E, Ht and the adjoint in both of its launches.  (The fused steps'
    launches are accounted as their phase.)"""
    c = cell_classes(w)
    n, ni, nd, sa = c["cells"], c["interior"], c["design"], c["slab_axes"]
    npml = n - ni
    return {"fwd_h": 36 * n + 16 * sa, "fwd_e": 40 * n + 16 * sa,
            "rev_e": 76 * ni + 40 * npml + 16 * nd + 16 * sa,
            "rev_h": 72 * ni + 36 * npml + 16 * sa}


PHASE_KERNELS = {"forward": ["fwd_fused", "fwd_2step", "fwd_h", "fwd_e", "record"],
                 "reverse": ["restore_seed", "rev_e", "rev_h", "rev_primal", "rev_adjoint",
                             "rev_adjoint_cpml"]}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(digest: str, workload: str):
    """ncu DRAM bytes per launch recorded for this kernel build:
    {kernel kind: bytes}, from profiles/traffic.txt."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    out = {}
    if not os.path.exists(path):
        return out
    with open(path) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if len(parts) >= 4 and parts[1] == digest and parts[2] == workload:
                out[parts[0]] = float(parts[3])
    return out


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


def apply_options(A, sim, args):
    """Launch options given on the command line (unset ones keep the
    library's defaults)."""
    if args.kernel >= 0:
        sim.set_option(A.OPT_KERNEL, args.kernel)
    if args.reverse >= 0:
        sim.set_option(A.OPT_REVERSE, args.reverse)
    if args.forward >= 0:
        sim.set_option(A.OPT_FORWARD, args.forward)
    sim.set_option(A.OPT_ZGROUPS, args.zgroups)
    for val, opt in ((args.tile_y, A.OPT_TILE_Y), (args.tile_x, A.OPT_TILE_X),
                     (args.zchunk, A.OPT_ZCHUNK), (args.stages, A.OPT_STAGES)):
        if val > 0:
            sim.set_option(opt, val)
    for val, opt in ((args.pdl, A.OPT_PDL), (args.prefetch, A.OPT_PREFETCH),
                     (args.compact, A.OPT_COMPACT_AUX)):
        if val >= 0:
            sim.set_option(opt, val)
    if args.zchunk_fwd != -2:
        sim.set_option(A.OPT_ZCHUNK_FWD, args.zchunk_fwd)
    if args.zchunk_fwd2 != -2:
        sim.set_option(A.OPT_ZCHUNK_FWD2, args.zchunk_fwd2)
    if args.no_graphs:
        sim.set_option(A.OPT_USE_GRAPHS, 0)


def sampled_breakdown(A, fdtd, args, w, rec, dev, flush):
    """Per-kernel in-loop costs from a pass with one launch per half-step on
    the workload shortened to --sample-steps time steps (same grid, same work
    per launch): CUDA events on the library's stream around sampled launches
    (pair-minus-single intervals, see fdtd_kernel_timing)."""
    import torch
    ws_ = w.replace(n_steps=max(1, min(w.n_steps, args.sample_steps)))
    sim = fdtd.Simulation(ws_, device=dev)
    apply_options(A, sim, args)
    sim.set_option(A.OPT_ZGROUPS, 1)
    sim.set_option(A.OPT_SAMPLE_EVERY, args.sample_every)
    eps = torch.from_numpy(ws_.eps).to(dev)
    sim.forward(eps, rec)                   # capture the sampled graphs
    sim.backward(1.0)
    torch.cuda.synchronize()
    ktimes, loop_ms = {}, []
    for _ in range(2):
        flush.random_(0, 255)
        sim.forward(eps, rec)
        sim.backward(1.0)
        t = sim.last_timing()
        loop_ms.append(t["fwd_ms"] + t["bwd_ms"])
        for name, (ms, n) in sim.kernel_timing().items():
            ktimes.setdefault(name, []).append((ms, n))
    torch.cuda.synchronize()
    per_step = {"record": 1.0 / rec.k, "fwd_2step": 0.5}
    kb = kernel_bytes(w)
    other = "fwd_fused" in ktimes or "fwd_2step" in ktimes
    if other:   # the split half-steps ran only the other units
        kb = {k: v for k, v in kb.items() if k not in ("fwd_h", "fwd_e")}
    step_ms = statistics.median(loop_ms) / ws_.n_steps
    kern = {}
    for name, lst in ktimes.items():
        n = sum(c for _, c in lst)
        avg = sum(ms * c for ms, c in lst) / max(n, 1)
        d = {"avg_ms": avg, "sampled_launches": n,
             "share_of_step": avg * per_step.get(name, 1.0) / step_ms}
        if name in kb:
            d["own_bytes"] = kb[name]
            d["own_gbs"] = kb[name] / (avg / 1e3) / 1e9
        if name in ("fwd_h", "fwd_e") and "fwd_fused" in ktimes:
            d["units"] = "the CPML units of the fused forward step"
        if name in ("fwd_h", "fwd_e") and "fwd_2step" in ktimes:
            d["units"] = "the units outside the deep box, one time step per launch"
        if name == "fwd_2step":
            d["units"] = "the deep units, two time steps per launch"
        kern[name] = d
    del sim
    return kern, {"n_steps": ws_.n_steps, "ms_per_time_step": step_ms}


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
    apply_options(A, sim, args)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned = None
    if args.autotune:
        from paper_2603_24027_gb300 import autotune
        tuned = autotune.tune(sim, torch.from_numpy(w.eps).to(dev), rec)
    eps_h = torch.from_numpy(w.eps).pin_memory()
    grad_h = torch.empty(w.design_shape, dtype=torch.float32).pin_memory()

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        sim.value_and_grad_host(eps_h, rec, 1.0, grad_h)
    torch.cuda.synchronize()

    dev_ms, wall_s, fwd_ms, bwd_ms = [], [], [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index_for_smi(local)) as clk:
        for _ in range(args.steps):
            flush.random_(0, 255)              # evict L2 (129 MB) before each timed step
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L, _ = sim.value_and_grad_host(eps_h, rec, 1.0, grad_h)
            wall_s.append(time.perf_counter() - t0)
            dev_ms.append(sim.last_host_call_ms())
            t = sim.last_timing()
            fwd_ms.append(t["fwd_ms"])
            bwd_ms.append(t["bwd_ms"])
    barrier()
    assert np.isfinite(L) and np.isfinite(grad_h.numpy()).all()
    g_main = grad_h.clone()
    total_ms = max_over_ranks(sum(dev_ms), ws, dev)
    total_wall = max_over_ranks(sum(wall_s), ws, dev)
    t = sim.last_timing()
    gpu_launches = (t["fwd_launches"] + t["bwd_launches"] + 2) * args.steps
    cell_updates = w.n_cells * w.n_steps
    value = job_rate(ws, cell_updates, args.steps, total_ms / 1e3)

    # roofline of the two phases: algorithmic bytes of one time step over the
    # measured time of one step of that phase (the loops' CUDA events)
    peak, peak_kind = read_peaks()
    pb = phase_bytes(w, args.tape)
    f_ms = statistics.median(fwd_ms) / w.n_steps
    r_ms = statistics.median(bwd_ms) / w.n_steps
    digest = B.kernel_digest()
    traffic = read_traffic(digest, args.workload)
    kern, sampled = sampled_breakdown(A, fdtd, args, w, rec, dev, flush)
    per_launch = {"record": 1.0 / rec.k, "fwd_2step": 0.5}
    phases = {}
    for ph, ms in (("forward", f_ms), ("reverse", r_ms)):
        ach = pb[ph] / (ms / 1e3) / 1e9
        # ncu DRAM bytes of one time step of the phase: set only when every
        # kernel the phase launched has a capture for the current kernel code
        kinds = [k for k in PHASE_KERNELS[ph] if k in kern]
        tr = (sum(traffic[k] * per_launch.get(k, 1.0) for k in kinds)
              if kinds and all(k in traffic for k in kinds) else None)
        phases[ph] = {"algorithmic_bytes_per_time_step": pb[ph], "ms_per_time_step": ms,
                      "achieved": ach, "frac": ach / peak, "traffic": tr,
                      "kernels": kinds}
        if "fwd_2step" in kinds:
            phases[ph]["note"] = ("two time steps per pass over the deep units: one time "
                                  "step's algorithmic bytes over the time per step is an "
                                  "effective bandwidth (the pass moves the deep units' "
                                  "bytes once per two time steps)")
    dom = max(phases, key=lambda p: phases[p]["ms_per_time_step"])
    roofline = {"bound": "hbm", "kernel": f"{dom} phase (one time step)",
                "achieved": phases[dom]["achieved"], "peak": peak, "unit": "GB/s",
                "frac": phases[dom]["frac"], "traffic": phases[dom]["traffic"],
                "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "timing": "CUDA events on the library stream around each timed step's time "
                          "loops; per time step = loop time / n_steps",
                "kernel_digest": digest, "phases": phases,
                "breakdown": {"kernels": kern, "sampled_pass": sampled}}
    whole = (pb["forward"] + pb["reverse"]) * w.n_steps / (total_ms / args.steps / 1e3) / 1e9
    roofline["gradient_achieved"] = whole
    roofline["gradient_frac"] = whole / peak

    tape_bytes = sim.tape_bytes(rec)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded waveguide: Si strip in SiO2, smoothed random design)",
        "config": {"workload": w.name, "cells": w.n_cells, "n_steps": w.n_steps,
                   "pml": w.pml_thickness, "tape": args.tape,
                   "design_box": list(w.design_shape[::-1]),
                   "parallelism": f"replicas x{ws}",
                   "l2": "state larger than L2; L2 also flushed before every timed step",
                   "zgroups": args.zgroups or "automatic",
                   "forward_step": ("two steps per pass over the deep units" if "fwd_2step" in kern
                                    else "fused" if "fwd_fused" in kern else "split"),
                   "reverse_step": "fused" if "rev_primal" in kern else "split",
                   "autotuned": None if tuned is None else
                   {"options": tuned["options"], "cached": tuned["cached"]},
                   "fwd_ms": statistics.median(fwd_ms), "bwd_ms": statistics.median(bwd_ms),
                   "fwd_gcell_updates_per_s": cell_updates / statistics.median(fwd_ms) / 1e6,
                   "bwd_gcell_updates_per_s": cell_updates / statistics.median(bwd_ms) / 1e6,
                   "timed_through": "fdtd_value_and_grad_host (value: device part; e2e: wall)"},
        "gpu_launches": gpu_launches,
        "roofline": roofline,
        "clocks": clk.summary(),
        "tape_bytes": tape_bytes,
        "tape_reduction_vs_f32_k1": sim.tape_bytes(tape_cfg(A, "f32:1:linear")) / tape_bytes,
    }
    # what the tape buys on one GPU: how many such problems fit side by side
    dev_bytes = torch.cuda.get_device_properties(dev).total_memory
    ws_bytes = sim.workspace_bytes(rec)
    out["capacity"] = {"device_bytes": dev_bytes, "workspace_bytes": ws_bytes,
                       "problems_per_gpu": dev_bytes // ws_bytes}
    nd = int(np.prod(w.design_shape))
    out["e2e"] = {"value": job_rate(ws, cell_updates, args.steps, total_wall), "unit": UNIT,
                  "h2d_bytes_per_step": w.n_cells * 4, "d2h_bytes_per_step": nd * 4 + 8}
    del sim

    # the same code with the uncompressed FP32 tape: speed and gradient agreement
    if not args.no_compare:
        rec32 = tape_cfg(A, args.compare_tape)
        sim32 = fdtd.Simulation(w, device=dev)
        apply_options(A, sim32, args)
        g32 = torch.empty(w.design_shape, dtype=torch.float32).pin_memory()
        sim32.value_and_grad_host(eps_h, rec32, 1.0, g32)
        ts, tw = [], []
        for _ in range(max(1, args.compare_steps)):
            flush.random_(0, 255)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim32.value_and_grad_host(eps_h, rec32, 1.0, g32)
            tw.append(time.perf_counter() - t0)
            ts.append(sim32.last_host_call_ms())
        v32 = cell_updates / (sum(ts) / len(ts) / 1e3) / 1e9
        e32 = cell_updates / (sum(tw) / len(tw)) / 1e9
        a64, b64 = g_main.double(), g32.double()
        ws32 = sim32.workspace_bytes(rec32)
        out["capacity"].update(compare_workspace_bytes=ws32,
                               compare_problems_per_gpu=dev_bytes // ws32)
        out["compare"] = {"tape": args.compare_tape, "value": v32, "e2e": e32,
                          "tape_bytes": sim32.tape_bytes(rec32),
                          "tape_reduction": sim32.tape_bytes(rec32) / tape_bytes,
                          "speedup_vs_compare": value / ws / v32,
                          "e2e_speedup_vs_compare": out["e2e"]["value"] / ws / e32,
                          "grad_cosine": float((a64 * b64).sum() / (a64.norm() * b64.norm())),
                          "grad_rel_err": float((a64 - b64).norm() / b64.norm())}
        del sim32

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps, args.workload)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# --------------------------------------------------------- profile run ---

def run_profile(args):
    """One short forward + backward with the given launch options (one launch
    per half-step unless --zgroups says otherwise), for profilers."""
    import torch
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import build as B
    from paper_2603_24027_gb300 import fdtd
    from paper_2603_24027_gb300 import inputs as I

    B.build()
    w = I.CONFIGS[args.workload]().replace(n_steps=args.n_steps or 12)
    if args.pml:
        w = w.replace(pml_thickness=args.pml)
    rec = tape_cfg(A, args.tape)
    sim = fdtd.Simulation(w)
    if args.zgroups == 0:
        args.zgroups = 1
    apply_options(A, sim, args)
    sim.set_option(A.OPT_SAMPLE_EVERY, args.sample_every if args.sample_every != 50 else 0)
    eps = torch.from_numpy(w.eps).cuda()
    for _ in range(min(args.warmup, 1) + 1):
        L = sim.forward(eps, rec)
        g = sim.backward(1.0)
    torch.cuda.synchronize()
    opts = {name: sim.get_option(getattr(A, name)) for name in
            ("OPT_KERNEL", "OPT_TILE_Y", "OPT_TILE_X", "OPT_ZCHUNK", "OPT_ZCHUNK_FWD",
             "OPT_STAGES", "OPT_ZGROUPS", "OPT_COMPACT_AUX", "OPT_PDL", "OPT_PREFETCH",
             "OPT_REVERSE", "OPT_FORWARD", "OPT_ZCHUNK_FWD2")}
    print(json.dumps(dict(workload=w.name, n_steps=w.n_steps, pml=w.pml_thickness,
                          tape=args.tape, options=opts, L=L, grad_l1=float(g.abs().sum()),
                          timing=sim.last_timing(), kernels=sim.kernel_timing())))


# ------------------------------------------------------------- oracle ---

def oracle_step(n_steps: int, name: str):
    from oracle import oracle as O
    w = workload(0, n_steps=n_steps, name=name)
    t0 = time.perf_counter()
    O.gradient(w)
    return time.perf_counter() - t0, w


def cpu_baseline(n_steps: int, name: str):
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    oracle_step(max(1, n_steps // 2), name)   # warm-up, as the reference arm does
    dt, w = oracle_step(n_steps, name)
    return {"value": w.n_cells * w.n_steps / dt / 1e9, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle gradient (forward + stored-history adjoint) of the same "
                      f"{w.nx}x{w.ny}x{w.nz} workload truncated to {n_steps} steps, after one "
                      f"warm-up run; {dt:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    n = args.cpu_sample_steps
    for _ in range(max(3, args.warmup)):
        oracle_step(max(1, n // 2), args.workload)
    ts = []
    for _ in range(args.steps):
        dt, w = oracle_step(n, args.workload)
        ts.append(dt)
    value = w.n_cells * n * len(ts) / sum(ts) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": 1e3 * sum(ts) / len(ts),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "cells": w.n_cells, "n_steps_sample": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(),
                            "kind": "oracle",
                            "sample": f"each step: FP64 oracle gradient of the "
                                      f"{w.nx}x{w.ny}x{w.nz} workload over {n} steps"},
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
        apply_options(A, s, args)
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
    # aggregate algorithmic bytes of one step (all problems, both phases)
    byts = 0
    for w in wl:
        pb = phase_bytes(w, args.tape)
        byts += w.n_steps * (pb["forward"] + pb["reverse"])
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

    # the same designs in one launch per half-step over all of them
    # (fdtd_batch_forward / backward): measured beside the concurrent loops
    def bstep():
        fdtd.group_forward(sims, eps, rec, batched=True)
        return fdtd.group_backward(sims, batched=True)

    for _ in range(2):
        bstep()
    torch.cuda.synchronize()
    tb = []
    for _ in range(args.steps):
        flush.random_(0, 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        bstep()
        b.record()
        torch.cuda.synchronize()
        tb.append(a.elapsed_time(b))
    batched_ms = max_over_ranks(sum(tb), ws, dev)
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
        "roofline": {"bound": "hbm", "kernel": "whole gradient, all 64 concurrent problems",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_step": byts},
        "clocks": clk.summary(),
        "e2e": {"value": job_rate(ws, cell_updates, args.steps, e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": sum(w.n_cells * 4 for w in wl),
                "d2h_bytes_per_step": sum(int(np.prod(w.design_shape)) * 4 + 8 for w in wl)},
        "one_launch_per_half_step": {
            "value": job_rate(ws, cell_updates, args.steps, batched_ms / 1e3), "unit": UNIT,
            "ms_per_step": batched_ms / args.steps,
            "launches_per_step": sims[0].last_timing()["fwd_launches"]
            + sims[0].last_timing()["bwd_launches"]},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.profile_run:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
