"""Reduced precision sweep on the 100 x 100 x 50 waveguide (Fig. 3 analogue):
one seed, a few tape configurations, checked against the FP64 oracle."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import precision_sweep as PS  # noqa: E402

pytestmark = pytest.mark.gpu


def test_sweep_waveguide_device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2603_24027_gb300 import build as B
    B.build()
    rows, _ = PS.run_seed(0, 2000, dtypes=["f32", "bf16", "e4m3"], ks=[1, 4, 8, 16],
                          interps=["linear", "cubic"])
    by = {(r["dtype"], r["k"], r["interp"]): r for r in rows}
    base = by[("f32", 1, "linear")]
    assert base["grad_rel_err"] < 1e-4 and base["L_rel_err"] < 1e-5
    # compressed tapes: cosine >= 0.999 up to k = 8, every dtype and interpolation
    for (dt, k, interp), r in by.items():
        if k <= 8:
            assert r["cos_fp32_k1"] >= 0.999, (dt, k, interp, r["cos_fp32_k1"])
    # >= 16x smaller tape at cosine >= 0.999 (FP8 k = 8, BF16 k = 8)
    assert by[("e4m3", 8, "cubic")]["compression"] > 31.9
    assert by[("e4m3", 8, "cubic")]["cos_fp32_k1"] > 0.999
    assert by[("bf16", 8, "linear")]["compression"] == pytest.approx(16.0)
    # Sec. 3: degradation grows with k for linear interpolation; bf16 ~ fp32
    lin = [by[("f32", k, "linear")]["cos_fp32_k1"] for k in (4, 8, 16)]
    assert lin[0] > lin[1] > lin[2]
    assert abs(by[("bf16", 4, "linear")]["cos_fp32_k1"] - by[("f32", 4, "linear")]["cos_fp32_k1"]) < 1e-5
    # cubic interpolation beats linear at every k > 1
    for k in (4, 8, 16):
        assert by[("f32", k, "cubic")]["grad_rel_err"] < by[("f32", k, "linear")]["grad_rel_err"]


def test_paper_format_grid_ordering():
    """Sec. 4 (Fig. 3) with the paper's unscaled formats: float16, bfloat16
    and e4m3b11fnuz stay with float32, e5m2fnuz close behind, and the formats
    with coarse subnormals degrade in the order of their smallest subnormal
    (e4m3fnuz 2^-10, IEEE e4m3 2^-9, e3m4 2^-6) already at k = 1."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2603_24027_gb300 import build as B
    B.build()
    rows, _ = PS.run_seed(0, 2000, dtypes=PS.PAPER_DTYPES, ks=[1, 16], interps=["linear"],
                          scaled=False, oracle=False)
    c = {(r["dtype"], r["k"]): r["cos_fp32_k1"] for r in rows}
    for dt in ("f16", "bf16", "e4m3b11fnuz"):
        assert c[(dt, 1)] > 0.99999, (dt, c[(dt, 1)])
        assert abs(c[(dt, 16)] - c[("f32", 16)]) < 5e-4
    assert c[("e5m2fnuz", 1)] > 0.99995
    assert c[("e4m3b11fnuz", 1)] > c[("e4m3fnuz", 1)] > c[("e4m3ieee", 1)] > c[("e3m4", 1)]
    assert c[("e3m4", 1)] < 0.99
    comp = {(r["dtype"], r["k"]): r["compression"] for r in rows}
    assert comp[("e4m3b11fnuz", 16)] == pytest.approx(64.0)


@pytest.mark.parametrize("tape", ["bf16:4:linear", "e4m3:8:cubic"])
def test_compressed_tape_parity_against_the_oracle_method_at_sweep_size(tape):
    """The 100 x 100 x 50 waveguide, 2000 steps (the size the precision sweep
    is quoted on), compressed tapes against the FP64 oracle's run of the same
    method (same format, scale rule, k and interpolation): relative L2 error
    below 2e-2 and cosine above 0.999 (soft parity: a quantiser may round the
    FP32 and FP64 face values to neighbouring codes)."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from oracle import oracle as O
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import build as B
    from paper_2603_24027_gb300 import fdtd
    from paper_2603_24027_gb300 import inputs as I
    B.build()
    w = I.waveguide_sweep(seed=0, n_steps=2000)
    dt, k, interp = tape.split(":")
    Lm, gm = O.reverse(w, dt, scaled=dt == "e4m3", k=int(k), interp=interp)
    sim = fdtd.Simulation(w)
    eps = torch.from_numpy(w.eps).cuda()
    L = sim.forward(eps, A.record_cfg(dt, int(k), interp))
    g = sim.backward(1.0).cpu().numpy().astype(np.float64)
    assert L == pytest.approx(Lm, rel=1e-5)
    c = float(g.ravel() @ gm.ravel() / (np.linalg.norm(g) * np.linalg.norm(gm)))
    e = float(np.linalg.norm(g - gm) / np.linalg.norm(gm))
    print(f"{tape}: cosine {c:.7f}, rel. error {e:.2e} against the oracle's method run")
    assert c > 0.999 and e < 2e-2, (c, e)
