"""Bounds-checked build (-DFDTD_BOUNDS_CHECK) of the library: every store of
the default two-cells-per-thread kernels (and of the fused reverse step,
into the other buffer of each ping-pong pair) checks that it lands in the
fields, the adjoint fields or an auxiliary set of its launch, and the
gacc reduction that it stays in the design box; a stray store is skipped
and reported (FDTD_ECUDA).  compute-sanitizer is closed on this machine, so
this library build stands in for it: it runs the index arithmetic of the compact
auxiliary layout, the tile shapes, z chunks and ragged grids in a separate
process and checks that no store strays and the gradients stay those of
the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch
from oracle import oracle as O
from paper_2603_24027_gb300 import _capi as A, fdtd as F, inputs as I
assert A.LIB_PATH.endswith("_checked.so"), A.LIB_PATH
grids = {
    "ragged70": I.ragged_box(),
    "ragged86": I.ragged_box(nx=86, ny=50, nz=30, P=7, n_steps=60),
    "ragged45": I.ragged_box(nx=45, ny=27, nz=23, P=5, n_steps=60, det_kind=I.OBJ_E2_PLANE,
                             src_kind=I.SRC_POINT),
    "interior150": I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=50),
}
shapes = [dict(), {A.OPT_TILE_Y: 2, A.OPT_STAGES: 4, A.OPT_ZCHUNK: 1},
          {A.OPT_TILE_Y: 4, A.OPT_STAGES: 3, A.OPT_ZCHUNK: 3},
          {A.OPT_TILE_Y: 16, A.OPT_ZCHUNK: 5}, {A.OPT_TILE_X: 40, A.OPT_STAGES: 3},
          {A.OPT_EXACT_REVERSAL: 22}, {A.OPT_COMPACT_AUX: 0}, {A.OPT_REVERSE: 2},
          {A.OPT_REVERSE: 2, A.OPT_EXACT_REVERSAL: 22}, {A.OPT_REVERSE: 2, A.OPT_ZCHUNK: 3},
          {A.OPT_REVERSE: 2, A.OPT_ZCHUNK: 1, A.OPT_COMPACT_AUX: 0},
          {A.OPT_REVERSE: 1, A.OPT_ZCHUNK: 3}]
# the two-step forward (its pass writes the pair's other buffer and the
# intermediate buffer's frame) on the grid with deep units
deep = {"interior150": [{A.OPT_FORWARD: 3}, {A.OPT_FORWARD: 3, A.OPT_REVERSE: 2},
                        {A.OPT_FORWARD: 3, A.OPT_EXACT_REVERSAL: 22},
                        {A.OPT_FORWARD: 3, A.OPT_ZCHUNK_FWD: 4, A.OPT_ZCHUNK_FWD2: 5}]}
n = 0
for name, w in grids.items():
    ref = {"f32:1:linear": O.gradient(w)[1],
           "bdct10:2:cubic": O.reverse(w, "bdct10", k=2, interp="cubic")[1]}
    eps = torch.from_numpy(w.eps).cuda()
    for kernel in (5,):
        for opts in shapes + deep.get(name, []):
            for tape in ("f32:1:linear", "bdct10:2:cubic"):
                sim = F.Simulation(w)
                sim.set_option(A.OPT_KERNEL, kernel)
                for o, v in opts.items():
                    sim.set_option(o, v)
                dt, k, ip = tape.split(":")
                L = sim.forward(eps, A.record_cfg(dt, int(k), ip))
                g = sim.backward().cpu().numpy().astype(np.float64)
                g0 = ref[tape]
                c = float(g.ravel() @ g0.ravel() / np.linalg.norm(g) / np.linalg.norm(g0))
                assert c > 0.999, (name, kernel, opts, tape, c)
                if dt == "f32" and A.OPT_EXACT_REVERSAL not in opts:
                    assert np.linalg.norm(g - g0) / np.linalg.norm(g0) < 1e-4, (name, kernel, opts)
                n += 1
print(f"bounds-checked runs: {n}, no stray store")
'''


def test_bounds_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2603_24027_gb300 import build as B
    B.build(checked=True)
    env = dict(os.environ, FDTD_BOUNDS_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no stray store" in r.stdout
