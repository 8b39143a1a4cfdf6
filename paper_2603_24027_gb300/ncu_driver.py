"""Short, self-contained run of the library for profilers (ncu launch lists,
single-kernel captures) and launch-shape sweeps.

  python -m paper_2603_24027_gb300.ncu_driver --workload waveguide200 --steps 12 \
      --kernel 2 --tile-y 4 --zchunk 8 --tape bf16:4:linear [--no-graphs] [--sweep]

Runs one forward + backward (after one warm-up pair when --warmup 1) and
prints the objective and per-kernel sampled timings.  --pml overrides the
CPML thickness, to separate interior and absorbing-layer cost.  It runs one
launch per half-step unless --zgroups says otherwise (0: the library's
automatic z groups), so that a captured launch covers the whole grid.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="waveguide200")
    p.add_argument("--steps", type=int, default=12)
    p.add_argument("--kernel", type=int, default=2)
    p.add_argument("--tile-y", type=int, default=4)
    p.add_argument("--zchunk", type=int, default=8)
    p.add_argument("--rows", type=int, default=2)
    p.add_argument("--stages", type=int, default=2)
    p.add_argument("--pdl", type=int, default=0)
    p.add_argument("--prefetch", type=int, default=0)
    p.add_argument("--tile-x", type=int, default=32)
    p.add_argument("--compact", type=int, default=1)
    p.add_argument("--zchunk-fwd", type=int, default=-2,
                   help="-2: same as --zchunk, -1: the library's automatic choice")
    p.add_argument("--zgroups", type=int, default=1,
                   help="split each half-step launch into this many z-chunk ranges")
    p.add_argument("--tape", default="bf16:4:linear")
    p.add_argument("--pml", type=int, default=0)
    p.add_argument("--warmup", type=int, default=0)
    p.add_argument("--sample-every", type=int, default=0)
    p.add_argument("--no-graphs", action="store_true")
    a = p.parse_args(argv)

    import torch
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import build as B
    from paper_2603_24027_gb300 import fdtd
    from paper_2603_24027_gb300 import inputs as I

    B.build()
    w = I.CONFIGS[a.workload]().replace(n_steps=a.steps)
    if a.pml:
        w = w.replace(pml_thickness=a.pml)
    dt, k, interp = a.tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    sim = fdtd.Simulation(w)
    sim.set_option(A.OPT_KERNEL, a.kernel)
    sim.set_option(A.OPT_TILE_Y, a.tile_y)
    sim.set_option(A.OPT_ZCHUNK, a.zchunk)
    sim.set_option(A.OPT_ROWS, a.rows)
    sim.set_option(A.OPT_STAGES, a.stages)
    sim.set_option(A.OPT_PDL, a.pdl)
    sim.set_option(A.OPT_PREFETCH, a.prefetch)
    sim.set_option(A.OPT_TILE_X, a.tile_x)
    sim.set_option(A.OPT_COMPACT_AUX, a.compact)
    sim.set_option(A.OPT_ZCHUNK_FWD, a.zchunk if a.zchunk_fwd == -2 else a.zchunk_fwd)
    sim.set_option(A.OPT_ZGROUPS, a.zgroups)
    sim.set_option(A.OPT_SAMPLE_EVERY, a.sample_every)
    sim.set_option(A.OPT_USE_GRAPHS, 0 if a.no_graphs else 1)
    eps = torch.from_numpy(w.eps).cuda()
    for _ in range(a.warmup + 1):
        L = sim.forward(eps, rec)
        g = sim.backward(1.0)
    torch.cuda.synchronize()
    out = dict(workload=w.name, steps=w.n_steps, pml=w.pml_thickness, kernel=a.kernel,
               tile_y=a.tile_y, zchunk=a.zchunk, rows=a.rows, stages=a.stages, pdl=a.pdl, prefetch=a.prefetch, tile_x=a.tile_x, compact=a.compact, zchunk_fwd=a.zchunk_fwd, zgroups=a.zgroups, L=L, grad_l1=float(g.abs().sum()),
               timing=sim.last_timing(), kernels=sim.kernel_timing())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
