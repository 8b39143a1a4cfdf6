"""Batched designs in one launch per half-step (fdtd_batch_forward/backward)
against the same designs run one by one, and against the FP64 oracle.

The batched path runs the split staged kernels over a list of (design, tile,
z chunk) units, each CTA reading its design's own arguments and tensor maps
from device tables; the per-cell arithmetic is unchanged, so the fields and
gradients must equal each design's own run bit for bit (the objectives to the
order of their FP64 sums across CTAs).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2603_24027_gb300 import build as B
from paper_2603_24027_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    from paper_2603_24027_gb300 import fdtd
    return fdtd


@pytest.fixture(scope="module")
def A(F):
    from paper_2603_24027_gb300 import _capi
    return _capi


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def designs(n=6, seed=1, steps=(300, 420)):
    """Uneven vacuum cubes (32 to 64 cells, ragged against the 32 x 8 tiles)
    with uneven step counts, as in the batched benchmark."""
    return I.batched_cubes(n_sims=n, seed=seed, sizes=(32, 40, 48, 64), steps=steps)


def sims_for(F, A, wl):
    sims = [F.Simulation(w) for w in wl]
    for s in sims:
        s.set_option(A.OPT_FORWARD, 1)
        s.set_option(A.OPT_REVERSE, 1)
    return sims


@pytest.mark.parametrize("tape", ["bf16:4:linear", "f32:1:linear", "f16:3:cubic"])
def test_batched_designs_equal_their_own_runs(F, A, tape):
    wl = designs()
    assert len({w.n_steps for w in wl}) > 1 and len({w.nx for w in wl}) > 1
    dt, k, interp = tape.split(":")
    rec = A.record_cfg(dt, int(k), interp, scaled=False)
    eps = [torch.from_numpy(w.eps).cuda() for w in wl]
    seeds = [1.0 + 0.25 * i for i in range(len(wl))]
    # each design alone
    own = []
    for w, e, sd in zip(wl, eps, seeds):
        s = sims_for(F, A, [w])[0]
        L = s.forward(e, rec)
        fwd = s.read_fields().cpu().numpy()
        g = s.backward(sd).cpu().numpy()
        own.append((L, fwd, g))
    # all of them batched (twice: the second call reuses the plan)
    sims = sims_for(F, A, wl)
    for rep in range(2):
        objs = F.group_forward(sims, eps, rec, batched=True)
        fwds = [s.read_fields().cpu().numpy() for s in sims]
        gs = [g.cpu().numpy() for g in F.group_backward(sims, seeds, batched=True)]
        for (L, fwd, g), Lb, fb, gb in zip(own, objs, fwds, gs):
            assert np.abs(g).max() > 0
            np.testing.assert_array_equal(fb, fwd)
            assert Lb == pytest.approx(L, rel=1e-12)
            np.testing.assert_array_equal(gb, g)


def test_batched_designs_match_the_oracle(F, A):
    """FP32 tape of every step: every design's gradient within 1e-4 of the
    exact discrete gradient, its objective within 1e-5 (runs long enough for
    the pulse, centred at 2 tau = 272 steps, to reach the detector)."""
    wl = designs(n=4, seed=2, steps=(350, 450))
    sims = sims_for(F, A, wl)
    eps = [torch.from_numpy(w.eps).cuda() for w in wl]
    rec = A.record_cfg("f32", 1)
    objs = F.group_forward(sims, eps, rec, batched=True)
    gs = F.group_backward(sims, batched=True)
    for w, L, g in zip(wl, objs, gs):
        Lo, go = O.gradient(w)
        assert np.abs(go).max() > 0
        assert L == pytest.approx(Lo, rel=1e-5)
        assert rel(g.cpu().numpy(), go) < 1e-4


def test_batched_plan_follows_the_list(F, A):
    """A changed list (another order, one design fewer) rebuilds the plan and
    gives each design its own result again."""
    wl = designs(n=5, seed=3)
    sims = sims_for(F, A, wl)
    eps = [torch.from_numpy(w.eps).cuda() for w in wl]
    rec = A.record_cfg("bf16", 4)
    F.group_forward(sims, eps, rec, batched=True)
    g1 = [g.cpu().numpy() for g in F.group_backward(sims, batched=True)]
    order = [3, 0, 4, 1]
    sub = [sims[i] for i in order]
    F.group_forward(sub, [eps[i] for i in order], rec, batched=True)
    g2 = [g.cpu().numpy() for g in F.group_backward(sub, batched=True)]
    for i, g in zip(order, g2):
        np.testing.assert_array_equal(g, g1[i])


def test_batched_designs_refuse_what_they_do_not_run(F, A):
    """Scaled tape formats, exact reversal, and a backward without a batched
    forward are refused with their status; the handles stay usable."""
    wl = designs(n=3, seed=4, steps=(40, 60))
    eps = [torch.from_numpy(w.eps).cuda() for w in wl]
    sims = sims_for(F, A, wl)
    with pytest.raises(A.FdtdError) as e:
        F.group_forward(sims, eps, A.record_cfg("e4m3", 2, scaled=True), batched=True)
    assert e.value.status == A.FDTD_EINVAL
    sims[1].set_option(A.OPT_EXACT_REVERSAL, 22)
    with pytest.raises(A.FdtdError) as e:
        F.group_forward(sims, eps, A.record_cfg("bf16", 2), batched=True)
    assert e.value.status == A.FDTD_EINVAL
    sims[1].set_option(A.OPT_EXACT_REVERSAL, 0)
    with pytest.raises(A.FdtdError) as e:
        F.group_backward(sims, batched=True)
    assert e.value.status == A.FDTD_ESTATE
    objs = F.group_forward(sims, eps, A.record_cfg("bf16", 2), batched=True)
    assert all(np.isfinite(objs))
    assert all(torch.isfinite(g).all() for g in F.group_backward(sims, batched=True))
