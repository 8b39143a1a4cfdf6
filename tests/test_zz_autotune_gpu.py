"""The launch-shape autotuner on the GPU: it times candidate shapes on a
shortened copy of the problem, applies the fastest, caches it per GPU type
and problem shape, and leaves the results unchanged (every shape it tries
gives the same fields bit for bit and the same gradient).

Collected after the parity files, like the no-allocation test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_24027_gb300 import build as B
from paper_2603_24027_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_autotune_applies_caches_and_keeps_results(tmp_path):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    from paper_2603_24027_gb300 import _capi as A
    from paper_2603_24027_gb300 import autotune as T
    from paper_2603_24027_gb300 import fdtd

    w = I.ragged_box()
    rec = A.record_cfg("bf16", 2)
    eps = torch.from_numpy(np.ascontiguousarray(w.eps)).cuda()
    base = fdtd.Simulation(w)
    base.forward(eps, rec)
    f0 = base.read_fields().cpu().numpy()
    g0 = base.backward(1.0).cpu().numpy()

    sim = fdtd.Simulation(w)
    path = str(tmp_path / "tune.json")
    r = T.tune(sim, eps, rec, cache=path, trial_steps=20, reps=1, max_passes=1)
    assert not r["cached"] and r["trials"] >= 10 and r["seconds"] > 0
    assert T.valid(r["options"])
    for name, value in r["options"].items():
        assert sim.get_option(T.OPTION_IDS[name]) == value

    sim.forward(eps, rec)
    np.testing.assert_array_equal(sim.read_fields().cpu().numpy(), f0)
    g = sim.backward(1.0).cpu().numpy()
    assert rel(g, g0) < 1e-6

    other = fdtd.Simulation(w)
    r2 = T.tune(other, eps, rec, cache=path)
    assert r2["cached"] and r2["options"] == r["options"]
    assert other.get_option(A.OPT_ZCHUNK) == r["options"]["zchunk"]
