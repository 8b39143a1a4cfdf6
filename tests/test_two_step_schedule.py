"""The two-step forward's schedule (FDTD_OPT_FORWARD = 3), on the host.

The pass over the deep units computes time steps n and n + 1 from the
pair's buffer X and writes only E^{n+2}, Ht^{n+3/2} of the deep box into the
other buffer B, plus the intermediate level E^{n+1}, Ht^{n+1/2} on the deep
box's one-cell frame into the third buffer M.  Every other unit runs the
split half-steps one step at a time: H of step n (X -> M), E of step n (E
from X, Ht from M, into M), H of step n + 1 (M -> B), E of step n + 1 (E
from M, Ht from B, into B), the CPML auxiliaries in place; the tape records
E^n (X) and Ht^{n+1/2} (M) at the pass's first step and E^{n+1} (M) and
Ht^{n+3/2} (B) at its second, the objective reads M, then B.

Here the FP64 oracle's single operations play every launch on the full
grid, reading the buffers the schedule names, with every cell of M that no
launch has written set to NaN.  The deep box comes from the library's own
fdtd_deep_units.  The schedule must reproduce the oracle's trajectory bit
for bit (fields, auxiliaries, tape faces, objective) outside the deep box,
where the split half-steps' results are kept; dropping one face of the frame
shows which layers are needed: E^{n+1} on the low faces (the H half-step of
step n + 1 reads E one cell up) and Ht^{n+1/2} on the high faces (the E
half-step of step n reads Ht one cell down).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_2603_24027_gb300 import inputs as I

NAN = float("nan")
FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    return oracle


def deep_box(w, zchunk=8):
    from paper_2603_24027_gb300 import _capi as A
    box = (C.c_int * 6)()
    assert A.lib().fdtd_deep_units(w.nx, w.ny, w.nz, w.pml_thickness, zchunk, box) == 0
    ix0, ix1, iy0, iy1, iz0, iz1 = list(box)
    assert ix1 > ix0 and iy1 > iy0 and iz1 > iz0
    return (32 * ix0, 32 * ix1), (8 * iy0, 8 * iy1), (zchunk * iz0, zchunk * iz1)


def masks(w, box):
    (x0, x1), (y0, y1), (z0, z1) = box
    deep = np.zeros((w.nz, w.ny, w.nx), bool)
    deep[z0:z1, y0:y1, x0:x1] = True
    layer = {}
    for name, (ax, idx) in zip(FACES, ((2, x0), (2, x1 - 1), (1, y0), (1, y1 - 1),
                                       (0, z0), (0, z1 - 1))):
        m = np.zeros_like(deep)
        sl = [slice(z0, z1), slice(y0, y1), slice(x0, x1)]
        sl[ax] = slice(idx, idx + 1)
        m[tuple(sl)] = True
        layer[name] = m
    return deep, layer


def compose(O, E_from, H_from, psi):
    s = np.empty((O.NF,) + E_from.shape[1:])
    s[0:3] = E_from[0:3]
    s[3:6] = H_from[3:6]
    s[6:] = psi
    return s


def faces(O, w, st):
    out = []
    for f in range(6):
        nu = (w.ny if f // 2 == 0 else w.nx) - 2 * w.pml_thickness
        nv = (w.ny if f // 2 == 2 else w.nz) - 2 * w.pml_thickness
        buf = np.zeros(2 * nu * nv)
        O.face_io(w, f, st, buf)
        out.append(buf)
    return out


def run_schedule(O, w, drop=None, seed=0):
    """The forward of w by the two-step schedule from random fields (zero
    auxiliaries, as the library starts); returns the per-step records,
    objectives and final state, and the reference trajectory's."""
    box = deep_box(w)
    deep, layer = masks(w, box)
    comp = ~deep
    frame = np.zeros_like(deep)
    for m in layer.values():
        frame |= m
    shape = (w.nz, w.ny, w.nx)
    ref = np.zeros((O.NF,) + shape)
    ref[:6] = np.random.default_rng(seed).standard_normal((6,) + shape)
    X = ref.copy()
    psi = X[6:].copy()
    got = {"tape": [], "obj": []}
    want = {"tape": [], "obj": []}
    assert w.n_steps % 2 == 0
    for n in range(0, w.n_steps, 2):
        # the reference trajectory, one operation at a time
        r_n = ref.copy()
        O.op(w, "forward_h", n, state=ref)
        want["tape"].append(faces(O, w, compose(O, r_n, ref, ref[6:])))
        O.op(w, "forward_e", n, state=ref)
        want["obj"].append(O.objective(w, ref))
        r_n1 = ref.copy()
        O.op(w, "forward_h", n + 1, state=ref)
        want["tape"].append(faces(O, w, compose(O, r_n1, ref, ref[6:])))
        O.op(w, "forward_e", n + 1, state=ref)
        want["obj"].append(O.objective(w, ref))
        # the pass over the deep units: from X alone; its intermediate level
        # goes to M on the frame (less the dropped layer), its result to B
        T = compose(O, X, X, psi)
        O.op(w, "forward_h", n, state=T)
        O.op(w, "forward_e", n, state=T)
        M = np.full((6,) + shape, NAN)
        keep = frame.copy()
        lvl = None
        if drop is not None:   # one face's layer, less the edges it shares
            name, lvl = drop
            others = np.zeros_like(frame)
            for o, m in layer.items():
                if o != name:
                    others |= m
            keep_lvl = frame & ~(layer[name] & ~others)
        for c in range(6):
            m = keep if drop is None or (lvl == "E1") != (c < 3) else keep_lvl
            M[c][m] = T[c][m]
        T2 = T.copy()
        O.op(w, "forward_h", n + 1, state=T2)
        O.op(w, "forward_e", n + 1, state=T2)
        B = np.full((6,) + shape, NAN)
        B[:, deep] = T2[:6, deep]
        # step n over the other units: H (X -> M), E (E from X, Ht from M)
        U = compose(O, X, X, psi)
        O.op(w, "forward_h", n, state=U)
        M[3:6][:, comp] = U[3:6][:, comp]
        psi[:, comp] = U[6:][:, comp]
        got["tape"].append(faces(O, w, compose(O, X, M, psi)))
        V = compose(O, X, M, psi)
        O.op(w, "forward_e", n, state=V)
        M[0:3][:, comp] = V[0:3][:, comp]
        psi[:, comp] = V[6:][:, comp]
        got["obj"].append(O.objective(w, compose(O, M, M, psi)))
        # step n + 1: H (M -> B), E (E from M, Ht from B)
        W = compose(O, M, M, psi)
        O.op(w, "forward_h", n + 1, state=W)
        B[3:6][:, comp] = W[3:6][:, comp]
        psi[:, comp] = W[6:][:, comp]
        got["tape"].append(faces(O, w, compose(O, M, B, psi)))
        Z = compose(O, M, B, psi)
        O.op(w, "forward_e", n + 1, state=Z)
        B[0:3][:, comp] = Z[0:3][:, comp]
        psi[:, comp] = Z[6:][:, comp]
        got["obj"].append(O.objective(w, compose(O, B, B, psi)))
        X = compose(O, B, B, psi)
    return got, want, X, ref, comp


def workload(n_steps=6):
    # deep units exist; the plane source (x = 7) and the Poynting detector
    # (x = 17) lie in the other units, two cells or more from the deep box;
    # the random initial fields fill the deep box from the first step
    return I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=n_steps)


def test_schedule_reproduces_the_trajectory(O):
    w = workload()
    got, want, X, ref, comp = run_schedule(O, w)
    assert np.abs(ref[:6]).max() > 0 and any(o != 0.0 for o in want["obj"])
    np.testing.assert_array_equal(X[:6], ref[:6])
    np.testing.assert_array_equal(X[6:][:, comp], ref[6:][:, comp])
    for a, b in zip(got["tape"], want["tape"]):
        for fa, fb in zip(a, b):
            np.testing.assert_array_equal(fa, fb)
    assert got["obj"] == want["obj"]


@pytest.mark.parametrize("name", FACES)
@pytest.mark.parametrize("level", ["E1", "H1"])
def test_each_frame_layer_the_other_units_read(O, name, level):
    """E^{n+1} is read on the low faces, Ht^{n+1/2} on the high faces; the
    other level of each face is written by the pass but never read (a face's
    layer is dropped without the edges it shares with other faces)."""
    w = workload(n_steps=2)
    got, want, X, ref, comp = run_schedule(O, w, drop=(name, level))
    needed = (level == "E1") == name.endswith("0")
    if needed:
        assert np.isnan(X[:6][:, comp]).any()
    else:
        np.testing.assert_array_equal(X[:6], ref[:6])
        assert got["obj"] == want["obj"]
