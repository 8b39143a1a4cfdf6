"""Launch-shape autotuner for the default kernels, with a JSON cache.

How fast a gradient runs depends on launch options that leave its results
unchanged: the tile height and ring stages of the one-plane kernels, the z
chunk of the reverse phases, of the forward half-steps and of the two-step
forward pass (a no-op where that pass does not run), and the number of z
groups each half-step is split into.  The library's defaults come from
sweeps on two waveguide grids; other grids may prefer other values.  `tune`
times candidate settings on a shortened copy of the problem itself (same
grid, CPML, source, detector, design box, tape and kernel; fewer time steps),
searching one option at a time from the current settings (coordinate
descent, repeated until a pass changes nothing), applies the fastest to the
simulation and stores it in a JSON cache keyed by the GPU name, the grid,
the CPML thickness, the kernel and the tape configuration, so that a
problem of the same shape is tuned once per GPU type.

    from paper_2603_24027_gb300 import autotune
    best = autotune.tune(sim, eps, rec)          # times, applies, caches
    autotune.tune(other_sim, eps, rec)           # same shape: cache hit, no timing

The search logic and the cache take the timing function as an argument
(`measure(options) -> seconds`), so they run without a GPU.
"""
from __future__ import annotations

import json
import os
import statistics
import time
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

from . import _capi as A

# option name -> (library option id, candidate values in the order tried)
SPACE: List[Tuple[str, int, Sequence[int]]] = [
    ("zgroups", A.OPT_ZGROUPS, (0, 1, 3, 4, 6, 8)),
    ("zchunk", A.OPT_ZCHUNK, (8, 4, 6, 10, 16)),
    ("zchunk_fwd", A.OPT_ZCHUNK_FWD, (-1, 8, 16, 4)),
    ("zchunk_fwd2", A.OPT_ZCHUNK_FWD2, (-1, 64, 256)),
    ("tile_y", A.OPT_TILE_Y, (8, 4, 16, 2)),
    ("stages", A.OPT_STAGES, (2, 3, 4)),
]
OPTION_IDS = {name: oid for name, oid, _ in SPACE}
# tile shape options the exact-reversal variant does not accept
_SHAPE_OPTIONS = ("tile_y", "stages")
# a candidate must beat the current best by this fraction to replace it
MIN_GAIN = 0.01


def default_cache_path() -> str:
    """$FDTD_AUTOTUNE_CACHE, else ~/.cache/fdtd_gb300/autotune.json."""
    p = os.environ.get("FDTD_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "fdtd_gb300", "autotune.json")


def cache_key(gpu_name: str, workload, kernel: int, rec) -> str:
    """GPU type, grid, CPML thickness, kernel and tape configuration."""
    return (f"{gpu_name}|{workload.nx}x{workload.ny}x{workload.nz}|P{workload.pml_thickness}"
            f"|kernel{kernel}|tape{rec.dtype}:{rec.k}:{rec.interp}:{rec.scaled}:{rec.coeffs}")


def load_cache(path: str) -> Dict[str, dict]:
    """The cache's entries; an absent or unreadable file is an empty cache."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def save_entry(path: str, key: str, entry: dict) -> None:
    """Add or replace one entry (read, update, atomic rename)."""
    data = load_cache(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def valid(options: Dict[str, int]) -> bool:
    """Shapes the one-plane kernels are built for: tile heights 2, 4, 8 with
    2-4 stages, height 16 with its own 3 stages; z chunks and groups in the
    library's ranges."""
    ty, s = options.get("tile_y", 8), options.get("stages", 2)
    if ty not in (2, 4, 8, 16) or not 2 <= s <= 4:
        return False
    if ty == 16 and s != 3:
        return False
    if options.get("zchunk", 8) < 0 or options.get("zchunk_fwd", -1) < -1:
        return False
    if options.get("zchunk_fwd2", -1) < -1:
        return False
    return 0 <= options.get("zgroups", 0) <= 16


def search(measure: Callable[[Dict[str, int]], float], start: Dict[str, int],
           space: Iterable[Tuple[str, int, Sequence[int]]] = SPACE, max_passes: int = 3,
           min_gain: float = MIN_GAIN):
    """Coordinate descent from `start`: for each option in turn, time every
    other candidate value with the rest fixed and keep the fastest if it beats
    the current best by `min_gain`; repeat until a pass changes nothing.
    Returns (best options, best seconds, [(options, seconds), ...] tried)."""
    space = list(space)
    best = dict(start)
    if not valid(best):
        raise ValueError(f"starting options are not a valid shape: {best}")
    best_t = measure(dict(best))
    tried = [(dict(best), best_t)]
    seen = {tuple(sorted(best.items()))}
    for _ in range(max_passes):
        changed = False
        for name, _, values in space:
            if name not in best:
                continue
            for v in values:
                cand = dict(best)
                cand[name] = v
                key = tuple(sorted(cand.items()))
                if key in seen or not valid(cand):
                    continue
                seen.add(key)
                t = measure(dict(cand))
                tried.append((dict(cand), t))
                if t < best_t * (1.0 - min_gain):
                    best, best_t, changed = cand, t, True
        if not changed:
            break
    return best, best_t, tried


def current_options(sim, names: Iterable[str]) -> Dict[str, int]:
    return {n: sim.get_option(OPTION_IDS[n]) for n in names}


def apply(sim, options: Dict[str, int]) -> None:
    for name, value in options.items():
        sim.set_option(OPTION_IDS[name], int(value))


def gpu_measure(sim, eps, rec, trial_steps: int = 200, reps: int = 3):
    """A timing function for `search`: forward + backward of a copy of sim's
    problem shortened to trial_steps time steps, with sim's other options,
    timed by the library's CUDA events (median of reps, after one untimed run
    that captures the graphs)."""
    import torch
    from . import fdtd

    w = sim.w.replace(n_steps=max(1, min(sim.w.n_steps, trial_steps)))
    trial = fdtd.Simulation(w, device=eps.device)
    tuned = set(OPTION_IDS.values())
    fixed = [A.OPT_KERNEL, A.OPT_USE_GRAPHS, A.OPT_PDL, A.OPT_PREFETCH,
             A.OPT_TILE_X, A.OPT_COMPACT_AUX, A.OPT_EXACT_REVERSAL]
    for oid in fixed:
        if oid not in tuned:
            trial.set_option(oid, sim.get_option(oid))

    def measure(options: Dict[str, int]) -> float:
        apply(trial, options)
        trial.forward(eps, rec)
        trial.backward(1.0)
        ts = []
        for _ in range(reps):
            trial.forward(eps, rec)
            trial.backward(1.0)
            t = trial.last_timing()
            ts.append((t["fwd_ms"] + t["bwd_ms"]) / 1e3)
        torch.cuda.synchronize()
        return statistics.median(ts)

    measure.trial = trial
    return measure


def tune(sim, eps, rec, cache: Optional[str] = None, trial_steps: int = 200, reps: int = 3,
         measure: Optional[Callable[[Dict[str, int]], float]] = None,
         gpu_name: Optional[str] = None, refresh: bool = False, max_passes: int = 3) -> dict:
    """Tune sim's launch options for (eps's device, rec), apply the result and
    cache it.  A cached entry for the same key is applied without timing
    unless refresh.  Returns the entry: {"options", "seconds", "trials",
    "trial_steps", "cached"}.  Options the kernel does not use are left
    alone (all of them unless kernel 5; tile shapes under exact reversal)."""
    kernel = sim.get_option(A.OPT_KERNEL)
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name(eps.device)
    path = cache if cache is not None else default_cache_path()
    key = cache_key(gpu_name, sim.w, kernel, rec)
    if not refresh:
        hit = load_cache(path).get(key)
        if hit and isinstance(hit.get("options"), dict):
            opts = {k: int(v) for k, v in hit["options"].items() if k in OPTION_IDS}
            if valid(opts):
                apply(sim, opts)
                return dict(hit, cached=True)
    if kernel != 5:
        return {"options": {}, "seconds": None, "trials": 0, "trial_steps": 0,
                "cached": False}
    names = [n for n, _, _ in SPACE]
    if sim.get_option(A.OPT_EXACT_REVERSAL):
        names = [n for n in names if n not in _SHAPE_OPTIONS]
    space = [s for s in SPACE if s[0] in names]
    if measure is None:
        measure = gpu_measure(sim, eps, rec, trial_steps, reps)
    t0 = time.time()
    best, best_t, tried = search(measure, current_options(sim, names), space, max_passes)
    apply(sim, best)
    entry = {"options": best, "seconds": best_t, "trials": len(tried),
             "trial_steps": trial_steps, "tuning_seconds": time.time() - t0,
             "tried": [[o, t] for o, t in tried]}
    save_entry(path, key, entry)
    return dict(entry, cached=False)
