"""fdtd_value_and_grad_noalloc: forward + backward without device allocation.

Some callers cannot allocate device memory (they run while a CUDA-graph
capture they do not own is active, or their device memory budget is fixed
in advance), so they cannot provide the usual workspace.  This entry point
uses a fixed scratch array compiled into the library instead.  Its results
must equal those of the workspace path (fdtd_forward + fdtd_backward) on the
same inputs, on consecutive calls (the scratch keeps the previous call's
contents, so everything it reads must be cleared first).

This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes alone in a fresh process, and one case
runs the no-allocation call as the first device work of a fresh process.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_24027_gb300 import build as B
from paper_2603_24027_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    B.build()
    from paper_2603_24027_gb300 import _capi, fdtd
    return _capi, fdtd


def _noalloc(A, sim, eps, rec, seed, out):
    obj = C.c_double()
    rc = A.lib().fdtd_value_and_grad_noalloc(sim.h, C.c_void_p(eps.data_ptr()), C.byref(rec),
                                             float(seed), C.byref(obj), C.c_void_p(out.data_ptr()))
    A.check(rc, sim.h)
    torch.cuda.synchronize()
    return obj.value, out.cpu().numpy().copy()


@pytest.mark.parametrize("kernel,reverse", [(0, 0), (5, 1), (5, 2)])
@pytest.mark.parametrize("tape", [("f32", 1, "linear"), ("bf16", 4, "cubic"), ("e4m3", 2, "linear"),
                                  ("bdct10", 2, "cubic")])
def test_noalloc_matches_workspace_path_on_two_calls(mods, kernel, reverse, tape):
    A, F = mods
    w = I.ragged_box(n_steps=90)
    rec = A.record_cfg(*tape)
    eps = torch.from_numpy(w.eps).cuda()
    # reference: the workspace entry points
    ref = F.Simulation(w)
    ref.set_option(A.OPT_KERNEL, kernel)
    ref.set_option(A.OPT_REVERSE, reverse)
    L_ref = ref.forward(eps, rec)
    g_ref = ref.backward(0.5).cpu().numpy()
    # two calls in a row through the no-allocation entry point
    sim = F.Simulation(w)
    sim.set_option(A.OPT_KERNEL, kernel)
    sim.set_option(A.OPT_REVERSE, reverse)
    out = torch.full(w.design_shape, float("nan"), device="cuda")
    for _ in range(2):
        L, g = _noalloc(A, sim, eps, rec, 0.5, out)
        assert L == pytest.approx(L_ref, rel=1e-12)
        np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())


def test_noalloc_after_a_different_problem_reuses_the_scratch_cleanly(mods):
    A, F = mods
    rec = A.record_cfg("bf16", 2, "linear")
    big = I.ragged_box(nx=45, ny=27, nz=23, P=5, n_steps=90, det_kind=I.OBJ_E2_PLANE,
                       src_kind=I.SRC_POINT)
    small = I.fd_cube()
    for w in (big, small, big):
        eps = torch.from_numpy(w.eps).cuda()
        ref = F.Simulation(w)
        L_ref = ref.forward(eps, rec)
        g_ref = ref.backward(1.0).cpu().numpy()
        sim = F.Simulation(w)
        out = torch.empty(w.design_shape, device="cuda")
        L, g = _noalloc(A, sim, eps, rec, 1.0, out)
        assert L == pytest.approx(L_ref, rel=1e-12)
        np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())


def test_noalloc_rejects_problems_larger_than_the_scratch(mods):
    A, F = mods
    w = I.waveguide_mid()                          # ~0.8 GB workspace
    sim = F.Simulation(w)
    rec = A.record_cfg("f32", 1)
    assert sim.workspace_bytes(rec) > (64 << 20)
    eps = torch.empty(1, device="cuda")
    out = torch.empty(1, device="cuda")
    obj = C.c_double()
    rc = A.lib().fdtd_value_and_grad_noalloc(sim.h, C.c_void_p(eps.data_ptr()), C.byref(rec), 1.0,
                                             C.byref(obj), C.c_void_p(out.data_ptr()))
    assert rc == A.FDTD_ENOMEM
    msg = A.lib().fdtd_last_error(sim.h).decode()
    assert "workspace" in msg and str(64 << 20) in msg


def test_noalloc_reports_a_device_wait_that_gave_up(mods):
    """A bounded device wait that runs out inside the call (the injected wait
    of FDTD_OPT_INJECT_WAIT_TIMEOUT, 200 000 cycles) makes the call return
    FDTD_ETIMEOUT, as the workspace path's backward does; the context stays
    usable and the next call, without the injection, is correct."""
    A, F = mods
    w = I.ragged_box(n_steps=40)
    rec = A.record_cfg("bf16", 2, "linear")
    eps = torch.from_numpy(w.eps).cuda()
    ref = F.Simulation(w)
    L_ref = ref.forward(eps, rec)
    g_ref = ref.backward(1.0).cpu().numpy()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_INJECT_WAIT_TIMEOUT, 200_000)
    out = torch.empty(w.design_shape, device="cuda")
    obj = C.c_double()
    rc = A.lib().fdtd_value_and_grad_noalloc(sim.h, C.c_void_p(eps.data_ptr()), C.byref(rec), 1.0,
                                             C.byref(obj), C.c_void_p(out.data_ptr()))
    assert rc == A.FDTD_ETIMEOUT
    assert "wait" in A.lib().fdtd_last_error(sim.h).decode()
    # the workspace path maps the same word the same way
    ws = F.Simulation(w)
    ws.set_option(A.OPT_INJECT_WAIT_TIMEOUT, 200_000)
    ws.forward(eps, rec)
    with pytest.raises(A.FdtdError) as ei:
        ws.backward(1.0)
    assert ei.value.status == A.FDTD_ETIMEOUT
    sim.set_option(A.OPT_INJECT_WAIT_TIMEOUT, 0)
    L, g = _noalloc(A, sim, eps, rec, 1.0, out)
    assert L == pytest.approx(L_ref, rel=1e-12)
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-9 * np.abs(g_ref).max())


_FRESH = r"""
import ctypes as C, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2603_24027_gb300 import _capi as A, fdtd as F, inputs as I
w = I.ragged_box(n_steps=60)
rec = A.record_cfg("bdct10", 2, "cubic")
eps = torch.from_numpy(w.eps).cuda()
sim = F.Simulation(w)
out = torch.empty(w.design_shape, device="cuda")
obj = C.c_double()
# the first device work of this process: the no-allocation call, BDCT tape
rc = A.lib().fdtd_value_and_grad_noalloc(sim.h, C.c_void_p(eps.data_ptr()), C.byref(rec), 1.0,
                                         C.byref(obj), C.c_void_p(out.data_ptr()))
A.check(rc, sim.h)
torch.cuda.synchronize()
g = out.cpu().numpy().astype(np.float64)
ref = F.Simulation(w)
L_ref = ref.forward(eps, rec)
g_ref = ref.backward(1.0).cpu().numpy().astype(np.float64)
assert abs(obj.value - L_ref) <= 1e-12 * abs(L_ref), (obj.value, L_ref)
err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
assert err < 1e-6, err
print("fresh-process noalloc ok", err)
"""


def test_noalloc_first_in_a_fresh_process_with_a_block_codec_tape(mods):
    """The no-allocation call as the very first device work of a process, with
    a BDCT tape: it must set up what it needs itself (the scratch address and
    the codec's basis table) and equal the workspace path run afterwards."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process noalloc ok" in r.stdout
