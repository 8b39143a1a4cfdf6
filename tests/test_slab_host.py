"""Slab decomposition over z (paper_2603_24027_gb300.slab), on CPU.

Two and three gloo ranks each run the method of Sec. 2 -- the forward with
the interface slices recorded, then the time-reversed run with the adjoint
-- on their own z planes only: the oracle's single operations are each
rank's arithmetic, and the module's partition, ownership (tape rows, design
rows, detector rows), schedule, exchanges and reductions are everything
around them.  Before every operation, each plane a rank does not own, and
every ghost component its schedule has not just delivered, holds NaN, so a
missing or misplaced exchange turns the result into NaN (the last test
drops each exchange in turn to show it).  The partitioned gradient must equal the
single-rank oracle method's bit for bit, and the objective to rounding.
"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2603_24027_gb300 import inputs as I  # noqa: E402
from paper_2603_24027_gb300 import slab as SL  # noqa: E402

NAN = float("nan")


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def box(det_kind=I.OBJ_POYNTING_PLANE, src_kind=I.SRC_PLANE_GAUSS, n_steps=48):
    """26 x 14 x 18 cells, 4-cell CPML; the design box (the interior) and,
    for the Poynting detector and the plane source, the x-normal planes span
    every slab."""
    return I.ragged_box(nx=26, ny=14, nz=18, P=4, n_steps=n_steps, det_kind=det_kind,
                        src_kind=src_kind)


# ---------------------------------------------------------------- host only --

@pytest.mark.parametrize("nz,P,world", [(18, 4, 2), (18, 4, 3), (11, 4, 2), (300, 16, 8),
                                        (100, 12, 4), (13, 4, 5)])
def test_partition_cuts_keep_the_cpml_whole_and_cover_the_grid(nz, P, world):
    s = SL.partition(40, 30, nz, P, world)
    assert [x.rank for x in s] == list(range(world))
    assert s[0].z0 == 0 and s[-1].z1 == nz
    for a, b in zip(s, s[1:]):
        assert a.z1 == b.z0 and P + 1 <= a.z1 <= nz - P - 1   # cut planes z-lossless
    assert all(x.z1 > x.z0 for x in s)
    assert s[0].cpml_lo and s[-1].cpml_hi
    assert not any(x.cpml_lo for x in s[1:]) and not any(x.cpml_hi for x in s[:-1])


def test_partition_balances_the_cost():
    """600 x 600 x 300 cells on 8 ranks: each slab within one plane's cost of
    the mean (the CPML planes cost more, so the end slabs are thinner)."""
    s = SL.partition(600, 600, 300, 16, 8)
    cost = SL.plane_cost(600, 600, 300, 16)
    per = np.array([cost[x.z0:x.z1].sum() for x in s])
    assert np.all(np.abs(per - per.mean()) <= cost.max())
    assert s[0].z1 - s[0].z0 < s[3].z1 - s[3].z0


def test_plane_cost_matches_the_per_cell_accounting():
    nx, ny, nz, P = 9, 8, 7, 2
    cost = SL.plane_cost(nx, ny, nz, P)
    for z in range(nz):
        tot = 0
        for y in range(ny):
            for x in range(nx):
                axes = sum(int(c < P or c >= n - P) for c, n in ((x, nx), (y, ny), (z, nz)))
                tot += 52 + 32 * axes + (100 if axes == 0 else 52) + 32 * axes
        assert cost[z] == tot


def test_partition_refuses_grids_too_thin():
    with pytest.raises(ValueError):
        SL.partition(20, 20, 12, 4, 5)     # cuts must lie in [5, 7]: three places, four cuts
    assert len(SL.partition(20, 20, 12, 4, 4)) == 4


@pytest.mark.parametrize("world", [1, 2, 3])
def test_tape_rows_cover_every_face_once(world):
    nx, ny, nz, P = 26, 14, 18, 4
    s = SL.partition(nx, ny, nz, P, world)
    rows = {0: nz - 2 * P, 1: nz - 2 * P, 2: nz - 2 * P, 3: nz - 2 * P, 4: ny - 2 * P,
            5: ny - 2 * P}
    for f in range(6):
        hit = np.zeros(rows[f], int)
        for x in s:
            r = x.face_rows(f)
            if r is not None:
                hit[r[0]:r[1]] += 1
        assert np.all(hit == 1), f
    assert s[0].face_rows(4) is not None and s[-1].face_rows(5) is not None


def test_every_operation_follows_its_exchange():
    for sched in (SL.FORWARD_STEP, SL.REVERSE_STEP):
        for i, (kind, name) in enumerate(sched):
            if kind == "op":
                assert sched[i - 1] == ("exchange", name)
    assert {n for k, n in SL.REVERSE_STEP if k == "op"} == {
        "inverse_e", "inverse_h", "adjoint_e", "adjoint_h"}
    # forward differences read the plane above, backward ones the plane below
    assert SL.HALO["forward_h"].side == SL.HALO["inverse_h"].side == "hi"
    assert SL.HALO["forward_e"].side == SL.HALO["inverse_e"].side == "lo"
    assert SL.HALO["adjoint_e"].side == "hi" and SL.HALO["adjoint_h"].side == "lo"


# ------------------------------------------------------- the ranks' method --

def _poison(a, s, psi_ghost_zero=True):
    """NaN on every plane the rank does not own; the auxiliaries of the ghost
    planes are zero (the z-lossless ghost planes multiply them by zero
    coefficients, and NaN * 0 would be NaN)."""
    a[:, :s.z0] = NAN
    a[:, s.z1:] = NAN
    if psi_ghost_zero:
        if s.has_lo:
            a[6:, s.z0 - 1] = 0.0
        if s.has_hi:
            a[6:, s.z1] = 0.0


def _rank_view(w, s):
    """The rank's detector rows and design rows as workloads of their own."""
    wd = None
    a, b = s.rows(w.design_lo[2], w.design_hi[2])
    if b > a:
        wd = w.replace(design_lo=(w.design_lo[0], w.design_lo[1], a),
                       design_hi=(w.design_hi[0], w.design_hi[1], b))
    if w.det_axis == 2:
        wr = w if s.z0 <= w.det_index < s.z1 else w.replace(det_kind=0)
    else:                                   # x- or y-normal plane: v is z
        a2, b2 = s.rows(w.det_lo[1], w.det_hi[1])
        wr = (w.replace(det_lo=(w.det_lo[0], a2), det_hi=(w.det_hi[0], b2)) if b2 > a2
              else w.replace(det_kind=0))
    return wr, wd


def _face_shape(w, f):
    a = f // 2
    ua = 1 if a == 0 else 0
    va = 1 if a == 2 else 2
    dims = (w.nx, w.ny, w.nz)
    return dims[ua] - 2 * w.pml_thickness, dims[va] - 2 * w.pml_thickness   # nu, nv


def partitioned_method(w, s, fmt, k, interp, seed=1.0, drop=None):
    """The method on slab s: returns (L, grad over the whole design box)."""
    from oracle import oracle as O
    T, P = w.n_steps, w.pml_thickness
    shape = (w.nz, w.ny, w.nx)
    st = np.zeros((O.NF,) + shape)
    lam = np.zeros((O.NF,) + shape)
    tmp = np.zeros((6,) + shape)
    dE = np.zeros((3,) + shape)
    wr, wd = _rank_view(w, s)
    gpart = np.zeros(wd.design_shape) if wd is not None else None
    blocks = {"state": torch.from_numpy(st[:6]), "adjoint": torch.from_numpy(lam[:6])}
    r = (T - 1) % k
    J = (T - 1 - r) // k + 1
    tape = {}                                # (j, f) -> [2][rows][nu]

    def xchg(name):
        if name != drop:
            h = SL.HALO[name]
            SL.exchange(s, blocks[h.block], h, z_offset=0)

    def record(faces, j):
        for f in faces:
            rows = s.face_rows(f)
            if rows is None:
                continue
            nu, nv = _face_shape(w, f)
            buf = np.zeros(2 * nu * nv)
            O.face_io(w, f, st, buf)
            tape[(j, f)] = buf.reshape(2, nv, nu)[:, rows[0]:rows[1]].copy()

    _poison(st, s)
    _poison(lam, s)
    L = 0.0
    for n in range(T):
        sample = n >= r and (n - r) % k == 0
        for kind, name in SL.FORWARD_STEP:
            if kind == "record" and sample:
                record((1, 3, 5) if name == "record_e" else (0, 2, 4), (n - r) // k)
            elif kind == "exchange":
                xchg(name)
            elif kind == "op":
                O.op(w, name, n, state=st)
                _poison(st, s)
            elif kind == "objective" and wr.det_kind:
                L += O.objective(wr, st)

    # compress: one scale per face and sample over all ranks' shares
    if fmt != "none":
        keys = [(j, f) for j in range(J) for f in range(6)]
        amax = [float(np.abs(tape[q]).max()) if q in tape else 0.0 for q in keys]
        gmax = SL.reduce_absmax(amax)
        for q, g in zip(keys, gmax):
            if q in tape:
                v = np.concatenate([tape[q].ravel(), [g]])   # the face's absmax rides along
                enc, _ = O.encode_face(fmt, v, scaled=True)
                tape[q] = enc[:-1].reshape(tape[q].shape)

    # the method keeps only the interior of E and Ht
    inside = np.zeros(shape, bool)
    inside[P:w.nz - P, P:w.ny - P, P:w.nx - P] = True
    st[:6, ~inside] = NAN
    st[6:] = NAN
    _poison(st, s, psi_ghost_zero=False)

    # every restored value of the rank, for every step (interpolated in time)
    steps = np.arange(T, dtype=np.float64)
    restored = {}
    for f in range(6):
        rows = s.face_rows(f)
        if rows is None:
            continue
        high = f % 2
        tk = ([0.0] if r > 0 else []) if high else [-1.0]
        tk = np.array(tk + [r + j * k for j in range(J)], np.float64)
        series = np.stack([tape[(j, f)] for j in range(J)], axis=-1)  # [2][rows][nu][J]
        if not high or r > 0:
            series = np.concatenate([np.zeros(series.shape[:-1] + (1,)), series], axis=-1)
        out = np.zeros(series.shape[:-1] + (T,))
        for idx in np.ndindex(series.shape[:-1]):
            out[idx] = O.interp_series(interp, tk, series[idx], steps)
        restored[f] = out

    def restore(faces, n):
        for f in faces:
            if f not in restored:
                continue
            rows = s.face_rows(f)
            nu, nv = _face_shape(w, f)
            buf = np.full((2, nv, nu), NAN)
            buf[:, rows[0]:rows[1]] = restored[f][..., n]
            O.face_io(w, f, st, np.ascontiguousarray(buf).ravel(), to_state=True)

    for n in range(T - 1, -1, -1):
        for kind, name in SL.REVERSE_STEP:
            if kind == "restore":
                restore((0, 2, 4) if name == "restore_h" else (1, 3, 5), n)
            elif kind == "seed" and wr.det_kind:
                O.objective_seed(wr, st, seed, lam)
            elif kind == "exchange":
                xchg(name)
            elif kind == "grad" and wd is not None:
                O.op(wd, "grad", lam=lam, dE=dE, grad=gpart)
            elif kind == "op" and name.startswith("inverse"):
                O.op(w, name, n, state=st, dE=dE)
                _poison(st, s, psi_ghost_zero=False)
            elif kind == "op":
                O.op(w, name, n, lam=lam, tmp=tmp)
                _poison(lam, s)

    L = SL.reduce_sum(L)
    zlo, zhi = w.design_lo[2], w.design_hi[2]
    rows = gpart if gpart is not None else np.zeros((0,) + w.design_shape[1:])
    return L, SL.gather_rows(s, rows, zlo, zhi)


CASES = [
    # (workload kwargs, tape format, k, interpolation)
    (dict(), "none", 1, "linear"),
    (dict(), "none", 3, "cubic"),
    (dict(), "e4m3", 2, "linear"),
    (dict(det_kind=I.OBJ_E2_PLANE, src_kind=I.SRC_POINT), "none", 4, "linear"),
]


def _rank_main(rank, ws, port, out_dir, cases, drop):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    from oracle import oracle as O
    O.set_num_threads(2)
    for i, (kw, fmt, k, interp) in enumerate(cases):
        w = box(**kw)
        s = SL.partition(w.nx, w.ny, w.nz, w.pml_thickness, ws)[rank]
        L, g = partitioned_method(w, s, fmt, k, interp, drop=drop)
        if rank == 0:
            np.save(os.path.join(out_dir, f"case{i}.npy"), np.concatenate([[L], g.ravel()]))
    dist.destroy_process_group()


def _run(ws, cases, tmp_path, drop=None):
    mp.start_processes(_rank_main, args=(ws, free_port(), str(tmp_path), cases, drop),
                       nprocs=ws, start_method="spawn", join=True)
    return [np.load(tmp_path / f"case{i}.npy") for i in range(len(cases))]


def _single(kw, fmt, k, interp):
    from oracle import oracle as O
    w = box(**kw)
    return O.reverse(w, fmt=fmt, scaled=fmt != "none", k=k, interp=interp)


def test_two_ranks_equal_the_single_rank_method(tmp_path):
    got = _run(2, CASES, tmp_path)
    for (kw, fmt, k, interp), v in zip(CASES, got):
        L, g = _single(kw, fmt, k, interp)
        assert np.all(np.isfinite(v))
        assert np.abs(g).max() > 0
        assert v[0] == pytest.approx(L, rel=1e-12, abs=1e-300)
        assert np.array_equal(v[1:], g.ravel()), (kw, fmt, k, interp)


def test_three_ranks_equal_the_single_rank_method(tmp_path):
    cases = [CASES[0], CASES[2]]
    got = _run(3, cases, tmp_path)
    for (kw, fmt, k, interp), v in zip(cases, got):
        L, g = _single(kw, fmt, k, interp)
        assert v[0] == pytest.approx(L, rel=1e-12)
        assert np.array_equal(v[1:], g.ravel())


@pytest.mark.parametrize("name", list(SL.HALO))
def test_every_exchange_is_needed(tmp_path, name):
    """Without any one of the six exchanges, a rank's plane next to the cut
    reads a NaN ghost value and the gradient is lost: the poisoning above
    sees every missing halo."""
    got = _run(2, [CASES[0]], tmp_path, drop=name)
    assert not np.all(np.isfinite(got[0][1:]))
