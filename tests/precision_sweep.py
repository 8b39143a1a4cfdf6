"""Precision sweep of the compressed boundary tape (Sec. 3, Fig. 3 analogue).

On the 100 x 100 x 50 waveguide device (2000 steps at 20 nm) and for each
seed: the FP64 oracle's exact gradient, then the CUDA path with every tape
configuration {FP32, BF16, FP16 + scale, FP8-E4M3 + scale} x k in
{1, 2, 4, 8, 16} x {linear, cubic}.  Reported per configuration (mean over
seeds): tape bytes and compression factor against FP32 k = 1, the objective's
and gradient's relative error against the oracle, and the gradient's cosine
similarity (Eq. 2) against the CUDA FP32 k = 1 gradient and against the
oracle.  The forward fields' error against the oracle is reported once (the
forward does not depend on the tape).

    python tests/precision_sweep.py --seeds 10 --out results.jsonl --md table.md

--paper-formats runs the paper's own grid instead (Sec. 4, Fig. 3): every
type unscaled (float32, float16, bfloat16 and the five 8-bit formats
e4m3b11fnuz, e5m2fnuz, e4m3fnuz, e4m3 (IEEE-style) and e3m4) for k in
{1, 2, 4, 8, 16, 32} with linear interpolation.

--block-codec runs the block-transform tape (beyond the paper: 8 x 8 DCT
blocks keeping K = 6, 10, 15 or 21 coefficients, int8 codes) for k in
{1, 4, 8, 16} with cubic interpolation, beside FP32 and scaled E4M3.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

DTYPES = ["f32", "bf16", "f16", "e4m3"]
KS = [1, 2, 4, 8, 16]
INTERPS = ["linear", "cubic"]
PAPER_DTYPES = ["f32", "f16", "bf16", "e4m3b11fnuz", "e5m2fnuz", "e4m3fnuz", "e4m3ieee", "e3m4"]
PAPER_KS = [1, 2, 4, 8, 16, 32]
BDCT_DTYPES = ["f32", "e4m3", "bdct6", "bdct10", "bdct15", "bdct21"]
BDCT_KS = [1, 4, 8, 16]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cos(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def run_seed(seed: int, n_steps: int, dtypes=DTYPES, ks=KS, interps=INTERPS, scaled=None,
             oracle=True):
    """One seed of the sweep.  scaled=None keeps each type's default (per-face
    scales for f16 and the hardware e4m3); False stores every type unscaled.
    oracle=False skips the FP64 reference (errors against it are then NaN)."""
    import torch

    from oracle import oracle as O
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import fdtd
    from paper_2603_24027_gb300 import inputs as I

    w = I.waveguide_sweep(seed=seed, n_steps=n_steps)
    t0 = time.perf_counter()
    if oracle:
        L_ref, g_ref, st_ref = O.gradient(w, want_state=True)
    else:
        L_ref, g_ref, st_ref = float("nan"), np.full(w.design_shape, np.nan), None
    t_oracle = time.perf_counter() - t0
    eps = torch.from_numpy(w.eps).cuda()
    sim = fdtd.Simulation(w)
    rows = []
    base = None
    for dt in dtypes:
        for k in ks:
            for interp in interps:
                if dt == "f32" and k == 1 and interp == "cubic" and base is None:
                    interp = "linear"   # the FP32 k = 1 baseline comes first
                elif dt == "f32" and k == 1 and interp == "cubic":
                    continue
                rec = A.record_cfg(dt, k, interp, scaled=scaled)
                L = sim.forward(eps, rec)
                fields = sim.read_fields().cpu().numpy() if base is None else None
                g = sim.backward(1.0).cpu().numpy()
                row = dict(seed=seed, dtype=dt, k=k, interp=interp, tape_bytes=sim.tape_bytes(rec),
                           L=L, L_rel_err=abs(L - L_ref) / abs(L_ref), grad_rel_err=rel(g, g_ref),
                           cos_oracle=cos(g, g_ref))
                if base is None:   # FP32 k = 1 first
                    base = dict(g=g, bytes=row["tape_bytes"])
                    row["E_rel_err"] = rel(fields[:3], st_ref[:3]) if oracle else float("nan")
                    row["H_rel_err"] = rel(fields[3:6], st_ref[3:6]) if oracle else float("nan")
                row["compression"] = base["bytes"] / row["tape_bytes"]
                row["cos_fp32_k1"] = cos(g, base["g"])
                row["rel_fp32_k1"] = rel(g, base["g"])
                rows.append(row)
    return rows, t_oracle


def table(rows):
    import collections
    agg = collections.OrderedDict()
    for r in rows:
        agg.setdefault((r["dtype"], r["k"], r["interp"]), []).append(r)
    lines = ["| tape | k | interp | compression | cos vs FP32 k=1 | rel err vs FP32 k=1 | cos vs oracle | rel err vs oracle |",
             "|---|---|---|---|---|---|---|---|"]
    for (dt, k, interp), rs in agg.items():
        m = lambda key: float(np.mean([r[key] for r in rs]))  # noqa: E731
        mn = lambda key: float(np.min([r[key] for r in rs]))  # noqa: E731
        lines.append(f"| {dt} | {k} | {interp} | {m('compression'):.2f} | {m('cos_fp32_k1'):.7f} "
                     f"(min {mn('cos_fp32_k1'):.7f}) | {m('rel_fp32_k1'):.2e} | "
                     f"{m('cos_oracle'):.7f} | {m('grad_rel_err'):.2e} |")
    return "\n".join(lines)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--seeds", type=int, default=10)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--out", default=None)
    p.add_argument("--md", default=None)
    p.add_argument("--paper-formats", action="store_true")
    p.add_argument("--no-oracle", action="store_true")
    p.add_argument("--block-codec", action="store_true")
    a = p.parse_args()
    from paper_2603_24027_gb300 import build as B
    from oracle import build as OB
    B.build()
    OB.build()
    rows = []
    for s in range(a.seeds):
        if a.paper_formats:
            r, t = run_seed(s, a.steps, dtypes=PAPER_DTYPES, ks=PAPER_KS, interps=["linear"],
                            scaled=False, oracle=not a.no_oracle)
        elif a.block_codec:
            r, t = run_seed(s, a.steps, dtypes=BDCT_DTYPES, ks=BDCT_KS, interps=["cubic"],
                            oracle=not a.no_oracle)
        else:
            r, t = run_seed(s, a.steps, oracle=not a.no_oracle)
        base = r[0]
        print(f"seed {s}: oracle {t:.1f} s, fields E {base['E_rel_err']:.2e} H {base['H_rel_err']:.2e}, "
              f"L {base['L_rel_err']:.2e}, FP32 k=1 grad {base['grad_rel_err']:.2e}", flush=True)
        rows += r
    md = table(rows)
    print(md)
    if a.out:
        with open(a.out, "w") as f:
            for r in rows:
                f.write(json.dumps(r) + "\n")
    if a.md:
        with open(a.md, "w") as f:
            f.write(md + "\n")


if __name__ == "__main__":
    main()
