"""Host-side checks of the C-ABI library (no GPU needed).

The library loads, exports every entry point include/fdtd.h declares, and
its host-computed plan (CPML tables, source waveform, tape interpolation
weights, argument validation, tape sizes) agrees with the independent FP64
oracle.  No compute kernel is called here.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_24027_gb300 import build as B
from paper_2603_24027_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    B.build()
    from paper_2603_24027_gb300 import _capi
    return _capi


@pytest.fixture(scope="module")
def fdtd(capi):
    from paper_2603_24027_gb300 import fdtd
    return fdtd


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(capi):
    names = declared_functions()
    assert len(names) >= 20
    L = C.CDLL(capi.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    # and the binding knows the prototype of each one
    assert set(names) <= set(capi._PROTOS)


def test_library_is_built_for_sm103a_only():
    flags = B.ARCH
    assert flags == ["-gencode", "arch=compute_103a,code=sm_103a"]


WORKLOADS = [I.small_dipole, lambda: I.waveguide_sweep(n_steps=50), I.fd_cube, I.ragged_box]


@pytest.mark.parametrize("make", WORKLOADS)
def test_cpml_tables_match_oracle(fdtd, make):
    w = make()
    sim = fdtd.Simulation(w)
    for ax in range(3):
        ref = O.profiles(w, ax)
        for which, key in enumerate(("b_e", "a_e", "kinv_e", "b_h", "a_h", "kinv_h")):
            got = sim.pml_profile(ax, which).astype(np.float64)
            np.testing.assert_allclose(got, ref[key], rtol=1.2e-7, atol=1e-30)


def test_cpml_tables_with_kappa_grading(fdtd):
    w = I.ragged_box().replace(pml_kappa_max=5.0, pml_alpha_factor=0.2)
    sim = fdtd.Simulation(w)
    for ax in range(3):
        ref = O.profiles(w, ax)
        for which, key in enumerate(("b_e", "a_e", "kinv_e", "b_h", "a_h", "kinv_h")):
            np.testing.assert_allclose(sim.pml_profile(ax, which), ref[key], rtol=1.2e-7, atol=1e-30)


@pytest.mark.parametrize("make", WORKLOADS)
def test_source_waveform_matches_oracle(fdtd, make):
    w = make()
    sim = fdtd.Simulation(w)
    got = sim.source_waveform().astype(np.float64)
    ref = O.waveform(w)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7 * np.abs(ref).max())


@pytest.mark.parametrize("N,k", [(40, 1), (40, 3), (41, 4), (37, 8), (16, 16), (5, 7), (2000, 16)])
@pytest.mark.parametrize("interp", ["linear", "cubic"])
@pytest.mark.parametrize("field", [0, 1])
def test_interpolation_weights_match_oracle(capi, fdtd, N, k, interp, field):
    """The library's per-step weights applied to a random recorded series
    equal the oracle's interpolation of that series, zero knot included."""
    w = I.fd_cube(n_steps=N)
    sim = fdtd.Simulation(w)
    rec = capi.record_cfg("f32", k, interp)
    r = (N - 1) % k
    J = O.n_samples(N, k)
    rng = np.random.default_rng(N * 100 + k)
    vals = rng.standard_normal(J)
    t = [r + j * k for j in range(J)]
    p = list(vals)
    if field == 0:
        t, p = [-1] + t, [0.0] + p
    elif r > 0:
        t, p = [0] + t, [0.0] + p
    steps = list(range(0, N, max(1, N // 60)))
    ref = O.interp_series(interp, np.array(t, float), np.array(p), np.array(steps, float))
    for s, rv in zip(steps, ref):
        slot, wt = sim.interp_weights(rec, s, field)
        got = sum(wt[m] * vals[slot[m]] for m in range(4) if slot[m] >= 0)
        assert got == pytest.approx(rv, abs=2e-6 * (1 + np.abs(vals).max()))


def test_create_rejects_bad_arguments(capi, fdtd):
    good = I.fd_cube()
    bad = [
        good.replace(pml_thickness=0),
        good.replace(dt=good.dt * 1.02),                    # beyond the 3D CFL limit
        good.replace(n_steps=0),
        good.replace(design_lo=(1, 2, 2)),                   # design box in the PML
        good.replace(design_hi=(2, 6, 6)),                   # empty design box
        good.replace(src_pos=(0, 3, 3)),                     # source in the PML
        good.replace(src_component=3),
        good.replace(det_index=1),                           # detector in the PML
        good.replace(det_hi=(7, 6)),
        good.replace(nx=5),                                  # interior too small
    ]
    for w in bad:
        with pytest.raises(capi.FdtdError) as e:
            fdtd.Simulation(w)
        assert e.value.status == capi.FDTD_EINVAL


def test_options_are_validated(capi, fdtd):
    sim = fdtd.Simulation(I.fd_cube())
    lib = capi.lib()
    v = C.c_int()
    for opt, default in [(capi.OPT_KERNEL, 5), (capi.OPT_TILE_Y, 8), (capi.OPT_STAGES, 2),
                         (capi.OPT_USE_GRAPHS, 1), (capi.OPT_TILE_X, 32), (capi.OPT_PDL, 0),
                         (capi.OPT_PREFETCH, 0), (capi.OPT_COMPACT_AUX, 1),
                         (capi.OPT_EXACT_REVERSAL, 0), (capi.OPT_ZCHUNK_FWD, -1),
                         (capi.OPT_ZGROUPS, 0), (capi.OPT_REVERSE, 0),
                         (capi.OPT_INJECT_WAIT_TIMEOUT, 0), (capi.OPT_FORWARD, 0),
                         (capi.OPT_ZCHUNK_FWD2, -1)]:
        assert lib.fdtd_get_option(sim.h, opt, C.byref(v)) == capi.FDTD_OK and v.value == default
    for opt, val in [(capi.OPT_KERNEL, 7), (capi.OPT_KERNEL, -1), (capi.OPT_TILE_Y, 3),
                     (capi.OPT_STAGES, 1), (capi.OPT_STAGES, 5), (capi.OPT_KERNEL, 4),
                     (capi.OPT_KERNEL, 6), (5, 1),
                     (capi.OPT_ZCHUNK, -1), (capi.OPT_TILE_X, 0), (capi.OPT_TILE_X, 36),
                     (capi.OPT_ZCHUNK_FWD, -2), (capi.OPT_EXACT_REVERSAL, 5),
                     (capi.OPT_ZGROUPS, -1), (capi.OPT_ZGROUPS, 17), (capi.OPT_REVERSE, 3),
                     (capi.OPT_REVERSE, -1), (capi.OPT_FORWARD, 4), (capi.OPT_FORWARD, -1),
                     (capi.OPT_ZCHUNK_FWD2, -2),
                     (99, 1)]:
        assert lib.fdtd_set_option(sim.h, opt, val) == capi.FDTD_EINVAL
    assert lib.fdtd_set_option(sim.h, capi.OPT_STAGES, 4) == capi.FDTD_OK
    assert lib.fdtd_get_option(sim.h, capi.OPT_STAGES, C.byref(v)) == capi.FDTD_OK and v.value == 4


def test_forward_without_workspace_is_a_state_error(capi, fdtd):
    sim = fdtd.Simulation(I.fd_cube())
    out = C.c_double()
    rc = capi.lib().fdtd_forward(sim.h, C.c_void_p(1), C.byref(capi.record_cfg()), C.byref(out))
    assert rc == capi.FDTD_ESTATE
    rc = capi.lib().fdtd_backward(sim.h, 1.0, C.c_void_p(1))
    assert rc == capi.FDTD_ESTATE


def test_tape_sizes_and_compression_factors(capi, fdtd):
    """Bytes per sample = 2 tangential values x 6 interior cross-sections x
    dtype bytes; factor = (32/bits) x k relative to FP32 every step (Sec. 3)
    plus 24 bytes of scales per sample for scaled formats."""
    w = I.waveguide_mid()
    sim = fdtd.Simulation(w)
    n = [w.nx - 24, w.ny - 24, w.nz - 24]
    per_sample = 2 * 2 * (n[1] * n[2] + n[0] * n[2] + n[0] * n[1])
    assert per_sample == 230912                      # 200x200x100, P = 12
    f32 = sim.tape_bytes(capi.record_cfg("f32", 1))
    assert f32 == 2000 * per_sample * 4
    bf16k4 = sim.tape_bytes(capi.record_cfg("bf16", 4))
    assert bf16k4 == 500 * per_sample * 2
    assert f32 / bf16k4 == 8.0
    e4k8 = sim.tape_bytes(capi.record_cfg("e4m3", 8))
    assert e4k8 == 250 * (per_sample + 24)
    assert f32 / e4k8 > 31.99
    e4k16 = sim.tape_bytes(capi.record_cfg("e4m3", 16, scaled=True))
    assert f32 / e4k16 > 63.9                        # the paper's 64x at 8 bits, k = 16


def test_compact_auxiliary_workspace(capi, fdtd):
    """The staged kernels keep each axis' CPML auxiliaries only
    over that axis' two slabs (x: cells [0, round_up(P, 4)) and from the
    4-aligned cell round_down(nx - P, 4) on, rows padded to 4; y, z: 2P rows /
    planes), per axis where the grid is long enough (nx >= 2P + 56,
    ny >= 2P + 24, nz >= 2P + 1); the plain-load kernels keep the full grid.
    Three sets (forward + two adjoint) differ; with the fused reverse step
    kernel 5 also holds a second field and adjoint buffer (ping-pong pairs,
    2 x 6 components); everything else is equal."""
    al = lambda b: (b + 255) // 256 * 256

    def full(nx, ny, nz):
        px = (nx + 7) // 8 * 8
        return al(12 * nz * ny * px * 4)

    # 200 x 200 x 100, P = 12: every axis compact
    w = I.waveguide_mid()
    sim = fdtd.Simulation(w)
    rec = capi.record_cfg("bf16", 4)
    sim.set_option(capi.OPT_KERNEL, 0)
    b4 = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_KERNEL, 5)
    sim.set_option(capi.OPT_REVERSE, 2)
    b5 = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_REVERSE, 1)
    b5s = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_REVERSE, 0)   # automatic: split here (70 % of the units in the CPML)
    assert sim.workspace_bytes(rec) == b5s
    compact = al(4 * (24 * 200 * 100 + 200 * 24 * 100 + 200 * 200 * 24) * 4)
    assert b4 - b5s == 3 * (full(200, 200, 100) - compact)
    assert b5 - b5s == 2 * al(6 * 100 * 200 * 200 * 4)
    assert compact / full(200, 200, 100) == pytest.approx(0.16)
    # 70 x 21 x 19, P = 6: x (rows of 8 + 6 cells, pitch 16) and z (12
    # planes) compact, y too short (full rows of px = 72)
    w = I.ragged_box()
    sim = fdtd.Simulation(w)
    sim.set_option(capi.OPT_KERNEL, 0)
    b4 = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_KERNEL, 5)
    sim.set_option(capi.OPT_REVERSE, 1)
    b5 = sim.workspace_bytes(rec)
    compact = al(4 * (16 * 21 * 19 + 72 * 21 * 19 + 72 * 21 * 12) * 4)
    assert b4 - b5 == 3 * (full(70, 21, 19) - compact)


def test_bdct_basis_and_tape_sizes(capi, fdtd):
    """The block-transform codec: the library's basis table equals the
    oracle's bit for bit (both computed on the host from the DCT-II
    definition); tape bytes = samples x blocks x (K codes + 4-byte scale),
    blocks = 2 components x ceil(nu/8) ceil(nv/8) per face; coeffs is
    validated (1..64 for BDCT, 0 = 10; 0 for the other types)."""
    import ctypes as C
    from oracle import oracle as O
    beta = np.zeros(64 * 64, np.float32)
    assert capi.lib().fdtd_bdct_basis(C.c_void_p(beta.ctypes.data)) == capi.FDTD_OK
    np.testing.assert_array_equal(beta.reshape(64, 8, 8), O.bdct_basis())
    w = I.waveguide_mid()                            # faces 176x76 (x, y) and 176x176 (z)
    sim = fdtd.Simulation(w)
    blocks = 2 * 2 * (22 * 10 + 22 * 10 + 22 * 22)
    assert blocks == 3696
    for K, name in ((10, "bdct"), (6, "bdct6"), (21, "bdct21")):
        rec = capi.record_cfg(name, 8)
        assert rec.coeffs == K
        assert sim.tape_bytes(rec) == 250 * blocks * (K + 4)
    f32 = sim.tape_bytes(capi.record_cfg("f32", 1))
    assert f32 / sim.tape_bytes(capi.record_cfg("bdct10", 1)) > 17.8
    lib = capi.lib()
    n = C.c_size_t()
    for dt, k, coeffs in ((9, 1, 65), (9, 1, -1), (1, 1, 10)):
        rec = capi.RecordCfg(dt, k, 0, 0, coeffs)
        assert lib.fdtd_workspace_bytes(sim.h, C.byref(rec), C.byref(n)) == capi.FDTD_EINVAL
    rec = capi.RecordCfg(9, 1, 0, 1, 10)           # no per-face scale for BDCT
    out = C.c_double()
    assert lib.fdtd_forward(sim.h, C.c_void_p(1), C.byref(rec), C.byref(out)) == capi.FDTD_EINVAL


def test_exact_reversal_option_is_validated(capi, fdtd):
    """Grid exponent q: 0 (off) or 8..30; only kernel 5 rounds its increments,
    so a forward with another kernel and q != 0 is refused before any device
    work."""
    import ctypes as C
    sim = fdtd.Simulation(I.fd_cube())
    lib = capi.lib()
    for q in (7, 31, -1):
        assert lib.fdtd_set_option(sim.h, capi.OPT_EXACT_REVERSAL, q) == capi.FDTD_EINVAL
    assert lib.fdtd_set_option(sim.h, capi.OPT_EXACT_REVERSAL, 22) == capi.FDTD_OK
    v = C.c_int()
    assert lib.fdtd_get_option(sim.h, capi.OPT_EXACT_REVERSAL, C.byref(v)) == 0 and v.value == 22
    assert lib.fdtd_set_option(sim.h, capi.OPT_KERNEL, 0) == capi.FDTD_OK
    out = C.c_double()
    rc = lib.fdtd_forward(sim.h, C.c_void_p(1), C.byref(capi.record_cfg()), C.byref(out))
    assert rc == capi.FDTD_EINVAL


def test_checkpoint_header_is_validated(capi, fdtd):
    """fdtd_state_bytes needs a forward; fdtd_load_state refuses a blob that
    is not a state or belongs to another problem before touching the device."""
    import ctypes as C
    lib = capi.lib()
    sim = fdtd.Simulation(I.fd_cube())
    n = C.c_size_t()
    assert lib.fdtd_state_bytes(sim.h, C.byref(n)) == capi.FDTD_ESTATE
    junk = np.zeros(4096, np.uint8)
    assert lib.fdtd_load_state(sim.h, C.c_void_p(junk.ctypes.data), junk.size) == capi.FDTD_EINVAL
    # a header of an 8^3 problem with other step count
    hdr = np.zeros(4096, np.uint8)
    hdr[:8] = np.frombuffer(b"FDTDST01", np.uint8)
    ints = hdr[8:8 + 24].view(np.int32)
    ints[:] = [8, 8, 8, 2, 61, 0]
    assert lib.fdtd_load_state(sim.h, C.c_void_p(hdr.ctypes.data), hdr.size) == capi.FDTD_EINVAL


def test_error_word_maps_to_one_status(capi):
    """The device error word (bits the kernels OR in) maps to the status every
    entry point returns, through one rule: eps invalid (1) -> ENONFINITE,
    wait gave up (4) -> ETIMEOUT, dropped checked store (16) -> ECUDA,
    non-finite gradient (2) -> ENONFINITE, any other bit -> ECUDA; the first
    in that order wins."""
    f = capi.lib().fdtd_status_of_error_word
    assert f(0) == capi.FDTD_OK
    assert f(1) == capi.FDTD_ENONFINITE
    assert f(2) == capi.FDTD_ENONFINITE
    assert f(4) == capi.FDTD_ETIMEOUT
    assert f(16) == capi.FDTD_ECUDA
    assert f(8) == capi.FDTD_ECUDA and f(1 << 31) == capi.FDTD_ECUDA
    assert f(4 | 2) == capi.FDTD_ETIMEOUT          # a timed-out run's result is not trusted
    assert f(16 | 2) == capi.FDTD_ECUDA
    assert f(1 | 4 | 16) == capi.FDTD_ENONFINITE     # invalid input is reported first
    assert f(4 | 16) == capi.FDTD_ETIMEOUT


def test_noalloc_validates_options_like_the_forward(capi, fdtd):
    """Exact reversal is built into kernel 5 only: the no-allocation call
    refuses it with kernel 0 as fdtd_forward does, before any device work."""
    lib = capi.lib()
    sim = fdtd.Simulation(I.fd_cube())
    assert lib.fdtd_set_option(sim.h, capi.OPT_EXACT_REVERSAL, 22) == capi.FDTD_OK
    assert lib.fdtd_set_option(sim.h, capi.OPT_KERNEL, 0) == capi.FDTD_OK
    obj = C.c_double()
    rc = lib.fdtd_value_and_grad_noalloc(sim.h, C.c_void_p(256), C.byref(capi.record_cfg()), 1.0,
                                         C.byref(obj), C.c_void_p(512))
    assert rc == capi.FDTD_EINVAL
    assert "exact reversal" in lib.fdtd_last_error(sim.h).decode()
    rc = lib.fdtd_forward(sim.h, C.c_void_p(256), C.byref(capi.record_cfg()), C.byref(obj))
    assert rc == capi.FDTD_EINVAL


def test_inject_wait_option_is_validated(capi, fdtd):
    lib = capi.lib()
    sim = fdtd.Simulation(I.fd_cube())
    v = C.c_int()
    assert lib.fdtd_get_option(sim.h, capi.OPT_INJECT_WAIT_TIMEOUT, C.byref(v)) == 0 and v.value == 0
    assert lib.fdtd_set_option(sim.h, capi.OPT_INJECT_WAIT_TIMEOUT, -1) == capi.FDTD_EINVAL
    assert lib.fdtd_set_option(sim.h, capi.OPT_INJECT_WAIT_TIMEOUT, 100000) == capi.FDTD_OK
    assert lib.fdtd_get_option(sim.h, capi.OPT_INJECT_WAIT_TIMEOUT, C.byref(v)) == 0
    assert v.value == 100000


@pytest.mark.parametrize("nx,ny,nz,P,zc", [(150, 60, 40, 6, 8), (200, 90, 56, 8, 8),
                                          (170, 75, 61, 7, 4), (200, 200, 100, 12, 8),
                                          (600, 600, 300, 16, 8), (73, 33, 33, 8, 8),
                                          (74, 33, 33, 8, 8), (70, 21, 19, 6, 8),
                                          (130, 40, 60, 5, 7), (66, 34, 34, 1, 1)])
def test_deep_units_against_brute_force(capi, nx, ny, nz, P, zc):
    """The two-step forward's deep units: every 32 x 8 tile and whole zc-plane
    chunk whose cells x0-2 .. x0+33, y0-2 .. y0+8 and planes k0-2 .. k1 (where
    the pass evaluates the intermediate level) all lie in the interior, and
    no other; per axis the qualifying tiles form one run, so the units are
    the box the library reports (all zero when an axis has none)."""
    lib = capi.lib()
    box = (C.c_int * 6)()
    assert lib.fdtd_deep_units(nx, ny, nz, P, zc, box) == capi.FDTD_OK

    def inside(lo, hi_incl, n):
        return lo >= P and hi_incl <= n - P - 1

    xs = [t for t in range(-(-nx // 32)) if inside(32 * t - 2, 32 * t + 33, nx)]
    ys = [t for t in range(-(-ny // 8)) if inside(8 * t - 2, 8 * t + 8, ny)]
    zs = [c for c in range(-(-nz // zc)) if (c + 1) * zc <= nz and
          inside(c * zc - 2, (c + 1) * zc, nz)]
    want = [0] * 6
    if xs and ys and zs:
        for run in (xs, ys, zs):
            assert run == list(range(run[0], run[-1] + 1))
        want = [xs[0], xs[-1] + 1, ys[0], ys[-1] + 1, zs[0], zs[-1] + 1]
    assert list(box) == want
    assert lib.fdtd_deep_units(nx, ny, nz, P, 0, box) == capi.FDTD_EINVAL
    assert lib.fdtd_deep_units(nx, ny, nz, P, zc, None) == capi.FDTD_EINVAL


def test_two_step_forward_workspace(capi, fdtd):
    """FDTD_OPT_FORWARD = 3 holds three field buffers (the pair and the
    intermediate level); with the fused reverse the pair is shared."""
    def al(x):
        return (x + 255) // 256 * 256

    rec = capi.record_cfg("e4m3", 8)
    w = I.waveguide_large(n_steps=10)
    f6 = al(6 * w.nz * w.ny * ((w.nx + 7) // 8 * 8) * 4)
    sim = fdtd.Simulation(w)
    sim.set_option(capi.OPT_REVERSE, 1)
    sim.set_option(capi.OPT_FORWARD, 1)
    split = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_FORWARD, 3)
    assert sim.workspace_bytes(rec) - split == 2 * f6
    sim.set_option(capi.OPT_REVERSE, 2)
    assert sim.workspace_bytes(rec) - split == 3 * f6
    sim.set_option(capi.OPT_FORWARD, 3)
    sim.set_option(capi.OPT_ZCHUNK_FWD2, 5)
    assert sim.workspace_bytes(rec) - split == 3 * f6
    # a grid without deep units gets no third buffer (and is refused at the forward)
    sim = fdtd.Simulation(I.ragged_box())
    sim.set_option(capi.OPT_REVERSE, 1)
    sim.set_option(capi.OPT_FORWARD, 1)
    split = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_FORWARD, 3)
    assert sim.workspace_bytes(rec) == split


@pytest.mark.parametrize("nx,ny,nz,P,zc", [(70, 21, 19, 6, 8), (86, 50, 30, 7, 8), (86, 50, 30, 7, 3),
                                          (200, 200, 100, 12, 8), (120, 77, 41, 9, 0),
                                          (600, 600, 300, 16, 8), (20, 18, 17, 8, 5),
                                          (130, 40, 60, 5, 7)])
def test_fused_reverse_units_partition(capi, nx, ny, nz, P, zc):
    """The fused reverse step's launches (32 x 8 tiles, zc-plane chunks):
    the primal launch covers exactly the units that hold an interior cell;
    the adjoint launch without CPML terms exactly the units whose evaluated
    cells x0-1 .. x0+32, y0-1 .. y0+8 and planes k0-1 .. k1 all lie in the
    interior (so no CPML term is skipped); the adjoint launch with CPML every
    other unit, each once."""
    lib = capi.lib()
    counts = (C.c_int * 3)()
    assert lib.fdtd_reverse_units(nx, ny, nz, P, zc, counts, None, 0) == capi.FDTD_OK
    n = sum(counts)
    buf = np.zeros((n, 3), np.int32)
    assert lib.fdtd_reverse_units(nx, ny, nz, P, zc, counts, buf.ctypes.data, n - 1) == capi.FDTD_EINVAL
    assert lib.fdtd_reverse_units(nx, ny, nz, P, zc, counts, buf.ctypes.data, n) == capi.FDTD_OK
    prim = buf[:counts[0]]
    inner = buf[counts[0]:counts[0] + counts[1]]
    ring = buf[counts[0] + counts[1]:]
    z = zc if zc > 0 else nz
    ntx, nty, nzc = -(-nx // 32), -(-ny // 8), -(-nz // z)

    def interior(lo, hi, nn):           # every cell of [lo, hi] is interior
        return lo >= P and hi <= nn - P - 1

    want_p, want_i = set(), set()
    for cz in range(nzc):
        k0, k1 = cz * z, min(nz, cz * z + z)
        for ty in range(nty):
            for tx in range(ntx):
                x0, y0 = 32 * tx, 8 * ty
                has = (max(x0, P) < min(x0 + 32, nx - P) and max(y0, P) < min(y0 + 8, ny - P)
                       and max(k0, P) < min(k1, nz - P))
                if has:
                    want_p.add((tx, ty, cz))
                if (interior(x0 - 1, x0 + 32, nx) and interior(y0 - 1, y0 + 8, ny)
                        and interior(k0 - 1, k1, nz)):
                    want_i.add((tx, ty, cz))
    assert len(prim) == len(want_p) and set(map(tuple, prim)) == want_p
    assert len(inner) == len(want_i) and set(map(tuple, inner)) == want_i
    allu = {(tx, ty, cz) for cz in range(nzc) for ty in range(nty) for tx in range(ntx)}
    ring_set = set(map(tuple, ring))
    assert len(ring_set) == len(ring)               # each once
    assert ring_set == allu - want_i


def test_automatic_reverse_follows_the_cpml_share(capi, fdtd):
    """FDTD_OPT_REVERSE = 0 takes the fused reverse step (and its second field
    and adjoint buffers) where at most half of the (tile, chunk) units carry
    CPML terms: the 600 x 600 x 300 grid (31 %), not the 200 x 200 x 100 one
    (70 %)."""
    lib = capi.lib()
    counts = (C.c_int * 3)()
    for w, fused in ((I.waveguide_large(n_steps=10), True), (I.waveguide_mid(), False)):
        assert lib.fdtd_reverse_units(w.nx, w.ny, w.nz, w.pml_thickness, 8, counts, None, 0) == 0
        share = counts[2] / (counts[1] + counts[2])
        assert (share <= 0.5) == fused, share
        sim = fdtd.Simulation(w)
        rec = capi.record_cfg("e4m3", 8)
        auto = sim.workspace_bytes(rec)
        sim.set_option(capi.OPT_REVERSE, 2 if fused else 1)
        assert sim.workspace_bytes(rec) == auto


def test_fused_forward_workspace_and_automatic_choice(capi, fdtd):
    """The fused forward step needs the second field buffer only (its
    auxiliaries stay in place); FDTD_OPT_FORWARD = 0 takes the two-step pass
    (second and third buffer) on the 600 x 600 x 300 grid (31 % of the units
    in the CPML, source and detector in the ring) and neither it nor the
    fused step on the 200 x 200 x 100 one (70 %)."""
    def al(x):
        return (x + 255) // 256 * 256

    rec = capi.record_cfg("e4m3", 8)
    w = I.waveguide_large(n_steps=10)
    f6 = al(6 * w.nz * w.ny * ((w.nx + 7) // 8 * 8) * 4)
    sim = fdtd.Simulation(w)
    sim.set_option(capi.OPT_REVERSE, 1)
    sim.set_option(capi.OPT_FORWARD, 1)
    split = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_FORWARD, 2)
    assert sim.workspace_bytes(rec) - split == f6
    sim.set_option(capi.OPT_REVERSE, 2)
    assert sim.workspace_bytes(rec) - split == 2 * f6   # the reverse adds the adjoint's pair
    sim.set_option(capi.OPT_REVERSE, 1)
    sim.set_option(capi.OPT_FORWARD, 0)   # automatic: two steps per pass (a third buffer)
    assert sim.workspace_bytes(rec) - split == 2 * f6
    w = I.waveguide_mid()
    sim = fdtd.Simulation(w)
    sim.set_option(capi.OPT_REVERSE, 1)
    sim.set_option(capi.OPT_FORWARD, 1)
    split = sim.workspace_bytes(rec)
    sim.set_option(capi.OPT_FORWARD, 0)
    assert sim.workspace_bytes(rec) == split


def test_batched_designs_validate_before_any_device_work(capi, fdtd):
    """fdtd_batch_forward / fdtd_batch_backward check their arguments, the
    handles' options and the tape format on the host, before the plan's
    device tables or any launch (handles bound to a placeholder workspace
    address, which nothing dereferences on these paths)."""
    lib = capi.lib()
    wl = I.batched_cubes(n_sims=3, seed=5, sizes=(32, 40), steps=(20, 30))
    sims = [fdtd.Simulation(w) for w in wl]
    base = 1 << 40
    for i, s in enumerate(sims):
        assert lib.fdtd_bind_workspace(s.h, C.c_void_p(base + i * (1 << 32)), 1 << 31) == 0
    n = len(sims)
    hs = (C.c_void_p * n)(*[s.h.value for s in sims])
    eps = (C.c_void_p * n)(*[base] * n)
    objs = (C.c_double * n)()
    bf16 = capi.record_cfg("bf16", 4)
    assert lib.fdtd_batch_forward(hs, 0, eps, C.byref(bf16), objs) == capi.FDTD_EINVAL
    assert lib.fdtd_batch_forward(None, n, eps, C.byref(bf16), objs) == capi.FDTD_EINVAL
    twice = (C.c_void_p * 2)(sims[0].h.value, sims[0].h.value)
    assert lib.fdtd_batch_forward(twice, 2, eps, C.byref(bf16), objs) == capi.FDTD_EINVAL
    scaled = capi.record_cfg("e4m3", 2, scaled=True)
    assert lib.fdtd_batch_forward(hs, n, eps, C.byref(scaled), objs) == capi.FDTD_EINVAL
    assert b"unscaled" in lib.fdtd_last_error(sims[0].h)
    sims[2].set_option(capi.OPT_EXACT_REVERSAL, 22)
    assert lib.fdtd_batch_forward(hs, n, eps, C.byref(bf16), objs) == capi.FDTD_EINVAL
    assert b"split steps" in lib.fdtd_last_error(sims[2].h)
    sims[2].set_option(capi.OPT_EXACT_REVERSAL, 0)
    sims[1].set_option(capi.OPT_REVERSE, 2)
    assert lib.fdtd_batch_forward(hs, n, eps, C.byref(bf16), objs) == capi.FDTD_EINVAL
    sims[1].set_option(capi.OPT_REVERSE, 1)
    seeds = (C.c_double * n)(*[1.0] * n)
    grads = (C.c_void_p * n)(*[base] * n)
    assert lib.fdtd_batch_backward(hs, n, seeds, grads) == capi.FDTD_ESTATE
