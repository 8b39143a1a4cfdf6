"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated targets): forward fields 1e-5 relative L2 (FP32 fields;
the relative L2 of the E vector field and of the H vector field, since a
single component can be near zero by symmetry, e.g. Hz of a z dipole),
uncompressed-tape (FP32, k = 1) gradient 1e-4 relative L2 against the exact
discrete gradient.  Compressed tapes are compared with the oracle's own FP64
run of the method (same quantiser, same interpolation): their difference is
FP32-vs-FP64 field rounding amplified by the quantiser's rounding decisions,
so the bar there is a relative L2 of 2e-2 and a cosine of 0.999.
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


def field_err(gpu, ref):
    """(relative L2 of E, relative L2 of H) over the whole grid."""
    return rel(gpu[:3], ref[:3]), rel(gpu[3:6], ref[3:6])


def cos(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def gpu_run(F, A, w, rec=None, seed=1.0, options=None):
    rec = rec or A.record_cfg("f32", 1)
    sim = F.Simulation(w)
    for k, v in (options or {}).items():
        sim.set_option(k, v)
    eps = torch.from_numpy(np.ascontiguousarray(w.eps)).cuda()
    L = sim.forward(eps, rec)
    fields = sim.read_fields().cpu().numpy()
    hist = sim.objective_history()
    g = sim.backward(seed).cpu().numpy()
    return dict(L=L, fields=fields, hist=hist, g=g, sim=sim)


SMALL = {
    "ragged_poynting": lambda: I.ragged_box(),
    "ragged_e2_point": lambda: I.ragged_box(nx=45, ny=27, nz=23, P=5, n_steps=90,
                                            det_kind=I.OBJ_E2_PLANE, src_kind=I.SRC_POINT),
    "fd_cube": lambda: I.fd_cube(),
}


KERNELS = [0, 5]   # plain-load half-steps (independent cross-check), plane-staged half-steps (default)


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("kernel", KERNELS)
def test_forward_fields_and_objective(F, A, name, kernel):
    w = SMALL[name]()
    r = gpu_run(F, A, w, options={A.OPT_KERNEL: kernel})
    st, obj = O.forward(w)
    eE, eH = field_err(r["fields"], st)
    assert eE < 1e-5 and eH < 1e-5, (eE, eH)
    np.testing.assert_allclose(r["hist"], obj, rtol=0, atol=1e-5 * np.abs(obj).max())
    assert r["L"] == pytest.approx(obj.sum(), rel=1e-5)


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("kernel", KERNELS)
def test_uncompressed_gradient_matches_exact_gradient(F, A, name, kernel):
    w = SMALL[name]()
    r = gpu_run(F, A, w, seed=1.0, options={A.OPT_KERNEL: kernel})
    L, g = O.gradient(w)
    assert r["L"] == pytest.approx(L, rel=1e-5)
    assert rel(r["g"], g) < 1e-4


def test_seed_scales_the_gradient(F, A):
    w = SMALL["ragged_poynting"]()
    r1 = gpu_run(F, A, w, seed=1.0)
    r2 = gpu_run(F, A, w, seed=-2.5)
    np.testing.assert_allclose(r2["g"], -2.5 * r1["g"], rtol=1e-6, atol=1e-30)


def test_dipole48_config(F, A):
    """48^3 at 25 nm, 8-cell CPML, 400 steps, 16^3 random design (FP32 k=1)."""
    w = I.small_dipole()
    r = gpu_run(F, A, w)
    L, g, st = O.gradient(w, want_state=True)
    eE, eH = field_err(r["fields"], st)
    assert eE < 1e-5 and eH < 1e-5, (eE, eH)
    assert r["L"] == pytest.approx(L, rel=1e-5)
    assert rel(r["g"], g) < 1e-4


@pytest.mark.parametrize("dtype,k,interp", [("bf16", 4, "linear"), ("f16", 2, "cubic"),
                                            ("e4m3", 1, "linear"), ("e4m3", 4, "cubic"),
                                            ("f32", 3, "linear"), ("f32", 5, "cubic")])
def test_compressed_tape_matches_oracle_method(F, A, dtype, k, interp):
    w = I.ragged_box(n_steps=120)
    rec = A.record_cfg(dtype, k, interp)
    r = gpu_run(F, A, w, rec=rec)
    L, g = O.reverse(w, dtype, scaled=bool(rec.scaled), k=k, interp=interp)
    assert r["L"] == pytest.approx(L, rel=1e-5)
    assert rel(r["g"], g) < 2e-2
    assert cos(r["g"], g) > 0.999


def test_graphs_and_direct_launches_agree(F, A):
    w = SMALL["ragged_e2_point"]()
    rec = A.record_cfg("bf16", 2, "linear")
    a = gpu_run(F, A, w, rec=rec, options={A.OPT_USE_GRAPHS: 1})
    b = gpu_run(F, A, w, rec=rec, options={A.OPT_USE_GRAPHS: 0})
    np.testing.assert_array_equal(a["fields"], b["fields"])
    np.testing.assert_allclose(a["g"], b["g"], rtol=1e-12, atol=1e-30)


def same_gradient(g, base):
    """Kernel variants agree on the gradient up to the rounding of the adjoint
    sums, which the compiler may contract into fused multiply-adds differently
    in each variant (the forward uses explicitly rounded operations only, so
    its fields are compared bit for bit)."""
    assert rel(g, base) < 1e-6
    np.testing.assert_allclose(g, base, rtol=0, atol=1e-6 * np.abs(base).max())


@pytest.mark.parametrize("zchunk,tile_y,stages", [(1, 4, 3), (3, 8, 2), (0, 2, 4), (16, 1, 3),
                                                  (5, 16, 3), (2, 8, 4), (4, 4, 2)])
def test_launch_shapes_do_not_change_results(F, A, zchunk, tile_y, stages):
    w = SMALL["ragged_poynting"]()
    base = gpu_run(F, A, w)
    for kernel in KERNELS:
        r = gpu_run(F, A, w, options={A.OPT_KERNEL: kernel, A.OPT_ZCHUNK: zchunk,
                                      A.OPT_ZCHUNK_FWD: (zchunk + 5) % 17,
                                      A.OPT_TILE_Y: tile_y, A.OPT_STAGES: stages})
        np.testing.assert_array_equal(r["fields"], base["fields"])
        same_gradient(r["g"], base["g"])


FUSED_GRIDS = {
    "ragged_poynting": lambda: I.ragged_box(),
    "ragged_e2_point": lambda: I.ragged_box(nx=45, ny=27, nz=23, P=5, n_steps=90,
                                            det_kind=I.OBJ_E2_PLANE, src_kind=I.SRC_POINT),
    # CPML-free adjoint units exist and the CPML units take every branch of
    # their enumeration (chunks below / above, rows below / above, columns
    # left / right); 86 x 50 x 30 compacts all three auxiliary axes
    "interior_units": lambda: I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=70),
    "compact86": lambda: I.ragged_box(nx=86, ny=50, nz=30, P=7, n_steps=60),
    # a point source next to the low z-CPML inside the z-only units and an
    # |E|^2 detector nine cells above it: the z-CPML terms of the adjoint
    # there carry a large share of the gradient
    "zcpml_point": lambda: I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=120,
                                        det_kind=I.OBJ_E2_PLANE, src_kind=I.SRC_POINT),
}


def run_both_ways(F, A, w, rec, reverse, options=None):
    sim = F.Simulation(w)
    sim.set_option(A.OPT_REVERSE, reverse)
    for k, v in (options or {}).items():
        sim.set_option(k, v)
    eps = torch.from_numpy(np.ascontiguousarray(w.eps)).cuda()
    L = sim.forward(eps, rec)
    g = sim.backward(1.0).cpu().numpy()
    back = sim.read_fields().cpu().numpy()
    return L, g, back


@pytest.mark.parametrize("name", list(FUSED_GRIDS))
@pytest.mark.parametrize("tape", ["f32:1:linear", "bf16:4:cubic", "e4m3:2:linear", "bdct10:2:cubic"])
def test_fused_reverse_step_matches_the_split_phases(F, A, name, tape):
    """The fused reverse step (a primal and an adjoint launch per step, each
    reading every field once into the other buffer of a ping-pong pair)
    against the split phases: the reconstructed interior fields after the
    whole backward run bit for bit (the primal half-steps repeat the same
    rounded operations), the gradient to the adjoint sums' rounding."""
    w = FUSED_GRIDS[name]()
    dt, k, interp = tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    Ls, gs, bs = run_both_ways(F, A, w, rec, 1)
    Lf, gf, bf = run_both_ways(F, A, w, rec, 2)
    assert Lf == pytest.approx(Ls, rel=1e-12)   # FP64 atomic sums across CTAs
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    np.testing.assert_array_equal(bf[inner], bs[inner])
    assert np.abs(gs).max() > 0
    same_gradient(gf, gs)


def test_fused_reverse_step_with_exact_reversal_returns_to_zero(F, A):
    """Exact reversal through the fused primal kernel: the interior returns to
    the zero initial state bit for bit, and the gradient agrees with the split
    phases' exact-reversal run."""
    w = FUSED_GRIDS["interior_units"]()
    rec = A.record_cfg("f32", 1)
    opts = {A.OPT_EXACT_REVERSAL: 22}
    _, gs, _ = run_both_ways(F, A, w, rec, 1, opts)
    _, gf, bf = run_both_ways(F, A, w, rec, 2, opts)
    P = w.pml_thickness
    assert not np.any(bf[:, P:w.nz - P, P:w.ny - P, P:w.nx - P])
    same_gradient(gf, gs)


def test_fused_reverse_step_with_z_cpml_units_matches_the_oracle(F, A):
    """The fused reverse step against the exact discrete gradient where the
    z-only units' CPML terms matter (a point source in them): every unit
    variant of the adjoint must carry its CPML terms, and a missing one
    leaves the gradient far off (and, over thousands of steps, unbounded)."""
    w = FUSED_GRIDS["zcpml_point"]()
    L, g = O.gradient(w)
    Lf, gf, _ = run_both_ways(F, A, w, A.record_cfg("f32", 1), 2)
    assert Lf == pytest.approx(L, rel=1e-5)
    assert rel(gf, g) < 1e-4


def test_fused_reverse_step_stays_bounded_over_many_steps(F, A):
    """2000 steps on the grid above: the fused step's gradient stays within
    rounding of the split phases' (an adjoint CPML term left out grows
    without bound over such runs)."""
    w = FUSED_GRIDS["zcpml_point"]().replace(n_steps=2000)
    rec = A.record_cfg("e4m3", 8, "linear")
    _, gs, _ = run_both_ways(F, A, w, rec, 1)
    _, gf, _ = run_both_ways(F, A, w, rec, 2)
    assert np.all(np.isfinite(gf))
    assert rel(gf, gs) < 1e-5


# ------------------------------------------------ the fused forward step --

def run_forward_way(F, A, w, rec, forward, reverse, options=None):
    """(L, fields after the forward, gradient, fields after the backward)."""
    sim = F.Simulation(w)
    sim.set_option(A.OPT_FORWARD, forward)
    sim.set_option(A.OPT_REVERSE, reverse)
    for k, v in (options or {}).items():
        sim.set_option(k, v)
    eps = torch.from_numpy(np.ascontiguousarray(w.eps)).cuda()
    L = sim.forward(eps, rec)
    fwd = sim.read_fields().cpu().numpy()
    g = sim.backward(1.0).cpu().numpy()
    back = sim.read_fields().cpu().numpy()
    return L, fwd, g, back


FWD_GRIDS = {
    "interior_units": FUSED_GRIDS["interior_units"],
    # a point source next to the low z-CPML; the Poynting detector (x = 17)
    # and the source lie outside the CPML-free units, as the fused forward needs
    "point_near_zcpml": lambda: I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=120,
                                             src_kind=I.SRC_POINT),
    # odd step count: the forward ends in the second buffer of the pair
    "odd_steps": lambda: I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=71),
    "compact_large": lambda: I.ragged_box(nx=200, ny=90, nz=56, P=8, n_steps=50),
}


@pytest.mark.parametrize("name", list(FWD_GRIDS))
@pytest.mark.parametrize("tape", ["f32:1:linear", "bf16:4:cubic", "e4m3:2:linear"])
@pytest.mark.parametrize("reverse", [1, 2])
def test_fused_forward_step_matches_the_split_half_steps(F, A, name, tape, reverse):
    """The fused forward step (CPML-free units in one launch, the others in
    the split half-steps, all into the other buffer of a ping-pong pair)
    against the split half-steps in place: the fields after the forward and
    after the backward bit for bit (the same rounded operations per cell),
    the objective to the FP64 sums' order, the gradient to the adjoint sums'
    rounding; with both reverse modes, which start from the forward's buffer."""
    w = FWD_GRIDS[name]()
    dt, k, interp = tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    Ls, fs, gs, bs = run_forward_way(F, A, w, rec, 1, reverse)
    Lf, ff, gf, bf = run_forward_way(F, A, w, rec, 2, reverse)
    assert np.abs(fs).max() > 0
    np.testing.assert_array_equal(ff, fs)
    assert Lf == pytest.approx(Ls, rel=1e-12)
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    np.testing.assert_array_equal(bf[inner], bs[inner])
    same_gradient(gf, gs)


@pytest.mark.parametrize("n_steps", [70, 71])
def test_fused_forward_and_reverse_with_exact_reversal_return_to_zero(F, A, n_steps):
    """Exact reversal with both fused steps: the interior returns to zero bit
    for bit from either buffer of the pair, and the gradient (of the scheme
    with increments on the 2^-22 grid) matches the split kernels' run of the
    same scheme."""
    w = FWD_GRIDS["point_near_zcpml"]().replace(n_steps=n_steps)
    rec = A.record_cfg("f32", 1)
    opts = {A.OPT_EXACT_REVERSAL: 22}
    _, fwd, g, back = run_forward_way(F, A, w, rec, 2, 2, opts)
    _, fs, gs, _ = run_forward_way(F, A, w, rec, 1, 1, opts)
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(fwd[inner]).max() > 1e-3
    np.testing.assert_array_equal(fwd, fs)
    assert not np.any(back[inner])
    same_gradient(g, gs)


def test_fused_forward_needs_the_source_outside_its_units(F, A):
    """A source inside the CPML-free units: FDTD_OPT_FORWARD = 2 is refused at
    the forward, automatic (0) runs the split half-steps, and the gradient
    matches the oracle."""
    w = I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=120, src_kind=I.SRC_POINT)
    w = w.replace(src_pos=(40, 30, 20))   # tile 1, chunk 2: a CPML-free unit
    eps = torch.from_numpy(w.eps).cuda()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_FORWARD, 2)
    with pytest.raises(A.FdtdError) as e:
        sim.forward(eps, A.record_cfg("f32", 1))
    assert e.value.status == A.FDTD_EINVAL
    sim.set_option(A.OPT_FORWARD, 0)
    sim.forward(eps, A.record_cfg("f32", 1))
    _, g = O.gradient(w)
    assert np.abs(g).max() > 0
    assert rel(sim.backward(1.0).cpu().numpy(), g) < 1e-4


# grids with deep units for the two-step forward (source and detectors two
# cells or more away from them); "ragged_chunks" cuts the deep z range into
# 5-plane chunks of the pass over 4-plane chunks of the split half-steps
FWD2_GRIDS = {
    "interior_units": (FUSED_GRIDS["interior_units"], {}),
    "odd_steps": (FWD_GRIDS["odd_steps"], {}),
    "compact_large": (FWD_GRIDS["compact_large"], {}),
    "ragged_chunks": (lambda: I.ragged_box(nx=170, ny=75, nz=61, P=7, n_steps=33),
                      {"zf": 4, "zf2": 5}),
}


def fwd2_opts(A, extra):
    o = {}
    if "zf" in extra:
        o[A.OPT_ZCHUNK_FWD] = extra["zf"]
    if "zf2" in extra:
        o[A.OPT_ZCHUNK_FWD2] = extra["zf2"]
    return o


@pytest.mark.parametrize("name", list(FWD2_GRIDS))
@pytest.mark.parametrize("tape", ["f32:1:linear", "bf16:3:cubic", "e4m3:2:linear"])
@pytest.mark.parametrize("reverse", [1, 2])
def test_two_step_forward_matches_the_split_half_steps(F, A, name, tape, reverse):
    """Two time steps per pass over the deep units (the other units in split
    half-steps through the intermediate buffer) against the split half-steps
    in place: the fields after the forward and after the backward bit for
    bit, the objective to the FP64 sums' order, the gradient to the adjoint
    sums' rounding (so the tape, sampled at the pass's first and second step
    alike, is the same); odd step counts run their first step split."""
    make, extra = FWD2_GRIDS[name]
    w = make()
    dt, k, interp = tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    opts = fwd2_opts(A, extra)
    Ls, fs, gs, bs = run_forward_way(F, A, w, rec, 1, reverse, opts)
    Lt, ft, gt, bt = run_forward_way(F, A, w, rec, 3, reverse, opts)
    assert np.abs(fs).max() > 0
    np.testing.assert_array_equal(ft, fs)
    assert Lt == pytest.approx(Ls, rel=1e-12)
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    np.testing.assert_array_equal(bt[inner], bs[inner])
    same_gradient(gt, gs)


@pytest.mark.parametrize("n_steps", [70, 71])
def test_two_step_forward_with_exact_reversal_returns_to_zero(F, A, n_steps):
    """Exact reversal after a two-step forward: the fields equal the split
    kernels' run of the same scheme bit for bit, and the fused reverse brings
    the interior back to zero bit for bit from either buffer."""
    w = FWD2_GRIDS["interior_units"][0]().replace(n_steps=n_steps)
    rec = A.record_cfg("f32", 1)
    opts = {A.OPT_EXACT_REVERSAL: 22}
    _, fwd, g, back = run_forward_way(F, A, w, rec, 3, 2, opts)
    _, fs, gs, _ = run_forward_way(F, A, w, rec, 1, 1, opts)
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(fwd[inner]).max() > 1e-3
    np.testing.assert_array_equal(fwd, fs)
    assert not np.any(back[inner])
    same_gradient(g, gs)


def test_two_step_forward_matches_the_oracle(F, A):
    """FP32 tape of every step after a two-step forward: the gradient within
    1e-4 of the exact discrete gradient, the objective within 1e-5."""
    w = FWD2_GRIDS["interior_units"][0]().replace(n_steps=121)
    sim = F.Simulation(w)
    sim.set_option(A.OPT_FORWARD, 3)
    eps = torch.from_numpy(w.eps).cuda()
    L = sim.forward(eps, A.record_cfg("f32", 1))
    g = sim.backward(1.0).cpu().numpy()
    Lo, go = O.gradient(w)
    assert np.abs(go).max() > 0
    assert L == pytest.approx(Lo, rel=1e-5)
    assert rel(g, go) < 1e-4


def test_two_step_forward_needs_the_source_away_from_its_units(F, A):
    """A point source inside the deep units: FDTD_OPT_FORWARD = 3 is refused
    at the forward and the handle stays usable."""
    w = I.ragged_box(nx=150, ny=60, nz=40, P=6, n_steps=40, src_kind=I.SRC_POINT)
    w = w.replace(src_pos=(60, 30, 20))
    eps = torch.from_numpy(w.eps).cuda()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_FORWARD, 3)
    with pytest.raises(A.FdtdError) as e:
        sim.forward(eps, A.record_cfg("f32", 1))
    assert e.value.status == A.FDTD_EINVAL
    sim.set_option(A.OPT_FORWARD, 1)
    assert np.isfinite(sim.forward(eps, A.record_cfg("f32", 1)))


@pytest.mark.parametrize("reverse", [1, 2])
def test_exact_reversal_on_a_grid_of_many_waves(F, A, reverse):
    """300 x 120 x 80 cells, 200 steps, exact reversal: every one of the many
    waves of CTAs must read each staged plane only after its copy landed and
    refill a stage only after every thread's reads of it are ordered before
    the copy (a proxy fence between the shared-memory reads and the TMA
    write); any stale or early read leaves the interior off zero."""
    w = I.ragged_box(nx=300, ny=120, nz=80, P=8, n_steps=200)
    sim = F.Simulation(w)
    sim.set_option(A.OPT_REVERSE, reverse)
    sim.set_option(A.OPT_EXACT_REVERSAL, 22)
    eps = torch.from_numpy(w.eps).cuda()
    sim.forward(eps, A.record_cfg("f32", 1))
    fwd = sim.read_fields().cpu().numpy()
    sim.backward(1.0)
    back = sim.read_fields().cpu().numpy()
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(fwd[inner]).max() > 1e-3
    assert not np.any(back[inner])


@pytest.mark.parametrize("zchunk", [1, 3, 0])
def test_fused_reverse_step_chunks_and_two_detectors(F, A, zchunk):
    """z chunks of 1 and 3 planes and whole columns (every chunk boundary
    passes the lag planes between CTAs), and a second detector seeded in the
    same run: the fused step against the oracle's exact gradient."""
    w = I.coupler_small(n_steps=70)
    L, M, g = O.gradient2(w, 0.7, -1.3)
    sim = F.Simulation(w)
    sim.set_option(A.OPT_REVERSE, 2)
    sim.set_option(A.OPT_ZCHUNK, zchunk)
    eps = torch.from_numpy(w.eps).cuda()
    sim.forward(eps, A.record_cfg("f32", 1))
    gf = sim.backward(0.7, seed2=-1.3).cpu().numpy()
    assert rel(gf, g) < 1e-4


def test_fused_reverse_step_needs_its_tiles(F, A):
    """FDTD_OPT_REVERSE = 2 with other tiles than 32 x 8 is refused at the
    forward; automatic (0) falls back to the split phases there."""
    w = SMALL["fd_cube"]()
    eps = torch.from_numpy(w.eps).cuda()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_REVERSE, 2)
    sim.set_option(A.OPT_TILE_Y, 4)
    with pytest.raises(A.FdtdError) as e:
        sim.forward(eps, A.record_cfg("f32", 1))
    assert e.value.status == A.FDTD_EINVAL
    sim.set_option(A.OPT_REVERSE, 0)
    sim.forward(eps, A.record_cfg("f32", 1))
    L, g = O.gradient(w)
    assert rel(sim.backward(1.0).cpu().numpy(), g) < 1e-4


@pytest.mark.parametrize("zgroups,zchunk,zfwd,tape,graphs", [
    (2, 4, -1, "bf16:2", 1), (0, 3, -1, "f16:2", 0), (3, 2, 3, "f32:1", 1), (5, 1, 2, "bf16:3", 0),
    (16, 4, 4, "e4m3:2", 1), (4, 8, 0, "bdct:2", 1)])
def test_zgroups_do_not_change_results(F, A, zgroups, zchunk, zfwd, tape, graphs):
    """Split half-step launches over z-chunk ranges on their own streams (the
    scheduling only changes which launches may overlap): the same fields bit for
    bit, the same gradient, including more groups than z chunks (16 on the
    whole-column forward) and tape samples (record joins every group)."""
    w = SMALL["ragged_poynting"]()
    dt, k = tape.split(":")
    rec = A.record_cfg(dt, int(k))
    opts = {A.OPT_ZCHUNK: zchunk, A.OPT_ZCHUNK_FWD: zfwd, A.OPT_USE_GRAPHS: graphs}
    base = gpu_run(F, A, w, rec=rec, options={**opts, A.OPT_ZGROUPS: 1})
    r = gpu_run(F, A, w, rec=rec, options={**opts, A.OPT_ZGROUPS: zgroups})
    np.testing.assert_array_equal(r["fields"], base["fields"])
    np.testing.assert_allclose(r["hist"], base["hist"], rtol=1e-12, atol=1e-300)
    same_gradient(r["g"], base["g"])
    if tape == "f32:1":
        L, g = O.gradient(w)
        assert rel(r["g"], g) < 1e-4


def test_zgroups_benchmark_grid_matches_single_launches(F, A):
    """The 200 x 200 x 100 waveguide (400 steps, BF16 k = 4): the default z
    groups leave the forward fields bit for bit and the gradient unchanged."""
    w = I.waveguide().replace(n_steps=400)
    rec = A.record_cfg("bf16", 4)
    base = gpu_run(F, A, w, rec=rec, options={A.OPT_ZGROUPS: 1})
    r = gpu_run(F, A, w, rec=rec)   # automatic: 4 groups forward, 3 reverse
    np.testing.assert_array_equal(r["fields"], base["fields"])
    same_gradient(r["g"], base["g"])


@pytest.mark.parametrize("dtype", ["bf16", "f16", "e4m3"])
@pytest.mark.parametrize("scaled", [False, True])
def test_codec_is_bit_exact_against_torch_casts(F, A, dtype, scaled):
    import ctypes as C
    if scaled and dtype == "bf16":
        pytest.skip("bf16 shares FP32's exponent range: no scale")
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "e4m3": torch.float8_e4m3fn}[dtype]
    rng = np.random.default_rng(3)
    n = 100003
    x = (rng.standard_normal(n) * np.exp(rng.uniform(-12, 6, n))).astype(np.float32)
    if not scaled and dtype == "e4m3":
        x = np.clip(x, -448, 448)
    if not scaled and dtype == "f16":
        x = np.clip(x, -65504, 65504)
    xd = torch.from_numpy(x).cuda()
    code = torch.empty(n, dtype=tdt, device="cuda")
    scale = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    code_id = A.TAPE[dtype]
    A.check(A.lib().fdtd_encode(code_id, int(scaled), C.c_void_p(xd.data_ptr()), n,
                                C.c_void_p(code.data_ptr()), C.c_void_p(scale.data_ptr()), None))
    A.check(A.lib().fdtd_decode(code_id, C.c_void_p(code.data_ptr()), n,
                                C.c_void_p(scale.data_ptr()), C.c_void_p(out.data_ptr()), None))
    s = np.float32(1.0)
    if scaled:
        fmax = {"f16": 65504.0, "e4m3": 448.0}[dtype]
        s = np.float32(np.abs(x).max()) / np.float32(fmax)
        assert scale.item() == s
    ref_code = torch.from_numpy((x / s).astype(np.float32)).to(tdt)
    assert torch.equal(code.cpu().view(torch.uint8 if dtype == "e4m3" else torch.int16),
                       ref_code.view(torch.uint8 if dtype == "e4m3" else torch.int16))
    ref = (ref_code.to(torch.float32) * torch.tensor(s)).numpy()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("tile_x,stages", [(32, 2), (40, 2), (40, 3)])
@pytest.mark.parametrize("name", ["ragged_poynting", "ragged_e2_point"])
def test_tile_widths_do_not_change_results(F, A, tile_x, stages, name):
    """Two-cells-per-thread kernels with 32- and 40-wide tiles (8 rows)
    against the reference kernel variant."""
    w = SMALL[name]()
    rec = A.record_cfg("bf16", 2, "linear")
    base = gpu_run(F, A, w, rec=rec, options={A.OPT_KERNEL: 0})
    r = gpu_run(F, A, w, rec=rec, options={A.OPT_KERNEL: 5, A.OPT_TILE_Y: 8,
                                           A.OPT_TILE_X: tile_x, A.OPT_STAGES: stages})
    np.testing.assert_array_equal(r["fields"], base["fields"])
    same_gradient(r["g"], base["g"])


@pytest.mark.parametrize("ty,stages,tile_x", [(8, 2, 32), (8, 3, 40), (16, 3, 32), (2, 4, 32),
                                           (4, 2, 32)])
def test_compact_auxiliaries_match_the_full_grid_layout(F, A, ty, stages, tile_x):
    """86 x 50 x 30 cells, 7-cell CPML: the staged kernels keep the CPML
    auxiliaries of all three axes compact (x: 8 + 10 cells per row, the high
    slab from the 4-aligned cell 76; y and z: 14 rows / planes), or the full
    grid with FDTD_OPT_COMPACT_AUX = 0.  Same fields bit for bit, same
    gradient, for tile shapes whose boxes reach the mapped part of the
    arrays from different starts."""
    w = I.ragged_box(nx=86, ny=50, nz=30, P=7, n_steps=70)
    rec = A.record_cfg("bf16", 2, "linear")
    base = gpu_run(F, A, w, rec=rec, options={A.OPT_KERNEL: 5, A.OPT_COMPACT_AUX: 0})
    r = gpu_run(F, A, w, rec=rec, options={A.OPT_KERNEL: 5, A.OPT_TILE_Y: ty,
                                           A.OPT_STAGES: stages, A.OPT_TILE_X: tile_x})
    np.testing.assert_array_equal(r["fields"], base["fields"])
    same_gradient(r["g"], base["g"])
    assert r["sim"].workspace_bytes(rec) < base["sim"].workspace_bytes(rec)


@pytest.mark.parametrize("kernel,tape", [(5, "bf16:4:linear"), (5, "bdct10:2:cubic"),
                                         (0, "e4m3:2:cubic")])
def test_checkpoint_resumes_the_backward_in_another_handle(F, A, kernel, tape):
    """Forward in one handle, save its state to host memory, load it into a
    fresh handle of the same problem: the fresh handle's backward gives the
    original's gradient and objectives bit for bit."""
    w = SMALL["ragged_poynting"]()
    dt, k, interp = tape.split(":")
    rec = A.record_cfg(dt, int(k), interp)
    eps = torch.from_numpy(w.eps).cuda()
    a = F.Simulation(w)
    a.set_option(A.OPT_KERNEL, kernel)
    a.forward(eps, rec)
    blob = a.save_state()
    ga = a.backward().cpu().numpy()
    b = F.Simulation(w)
    b.set_option(A.OPT_KERNEL, kernel)
    b.load_state(blob, rec)
    np.testing.assert_array_equal(b.objective_history(), a.objective_history())
    gb = b.backward().cpu().numpy()
    np.testing.assert_array_equal(gb, ga)


@pytest.mark.parametrize("nx,ny,nz,tile_x", [(70, 38, 16, 32), (69, 37, 16, 32), (70, 38, 17, 40),
                                             (69, 39, 16, 40)])
def test_compact_auxiliaries_at_the_eligibility_thresholds(F, A, nx, ny, nz, tile_x):
    """7-cell CPML: x is compacted from nx = 2P + 56 = 70 and y from ny = 2P +
    24 = 38, one cell less keeps the axis full (z from 2P + 1, below the
    smallest valid grid, 2P + 2).  Grids at and just below each threshold,
    32- and 40-wide tiles: the fields equal the full-grid layout's bit for
    bit and the gradient agrees."""
    w = I.ragged_box(nx=nx, ny=ny, nz=nz, P=7, n_steps=50)
    rec = A.record_cfg("bf16", 2, "linear")
    opts = {A.OPT_TILE_X: tile_x, A.OPT_STAGES: 2}
    base = gpu_run(F, A, w, rec=rec, options={**opts, A.OPT_COMPACT_AUX: 0})
    r = gpu_run(F, A, w, rec=rec, options=opts)
    np.testing.assert_array_equal(r["fields"], base["fields"])
    same_gradient(r["g"], base["g"])


@pytest.mark.parametrize("graphs", [0, 1])
def test_dependent_launch_and_l2_prefetch_do_not_change_results(F, A, graphs):
    w = SMALL["ragged_poynting"]()
    rec = A.record_cfg("bf16", 2, "linear")
    a = gpu_run(F, A, w, rec=rec, options={A.OPT_PDL: 1, A.OPT_USE_GRAPHS: graphs,
                                           A.OPT_PREFETCH: 1})
    b = gpu_run(F, A, w, rec=rec, options={A.OPT_PDL: 0, A.OPT_USE_GRAPHS: graphs})
    np.testing.assert_array_equal(a["fields"], b["fields"])
    np.testing.assert_array_equal(a["g"], b["g"])
    assert a["L"] == b["L"]


@pytest.mark.parametrize("reverse,kinds", [(1, ("rev_e", "rev_h")),
                                           (2, ("rev_primal", "rev_adjoint", "rev_adjoint_cpml"))])
def test_sampled_kernel_timing_accounts_for_the_loop(F, A, reverse, kinds):
    """Differential in-loop timing (pair of launches minus single launch):
    every kernel kind gets a positive cost, the costs times the launch counts
    add up to the measured loop times, and sampling does not change results;
    for the split reverse phases and for the fused reverse step (its primal
    launch and its two adjoint launches)."""
    w = I.waveguide_sweep(n_steps=200)
    rec = A.record_cfg("bf16", 4, "linear")
    one = {A.OPT_ZGROUPS: 1, A.OPT_REVERSE: reverse}   # sampling records one launch per half-step
    base = gpu_run(F, A, w, rec=rec, options=one)
    r = gpu_run(F, A, w, rec=rec, options={**one, A.OPT_SAMPLE_EVERY: 7})
    np.testing.assert_array_equal(r["fields"], base["fields"])
    np.testing.assert_array_equal(r["g"], base["g"])
    sim = r["sim"]
    sim.forward(torch.from_numpy(w.eps).cuda(), rec)   # warm graphs, then measure
    sim.backward(1.0)
    kt, t = sim.kernel_timing(), sim.last_timing()
    for name in ("fwd_h", "fwd_e", "record", "restore_seed") + kinds:
        assert name in kt and kt[name][0] > 0 and kt[name][1] >= 1, (name, kt)
    n, nrec = w.n_steps, -(-w.n_steps // 4)
    fwd = n * (kt["fwd_h"][0] + kt["fwd_e"][0]) + nrec * kt["record"][0]
    bwd = n * (kt["restore_seed"][0] + sum(kt[k][0] for k in kinds))
    assert 0.7 < fwd / t["fwd_ms"] < 1.3, (fwd, t)
    assert 0.7 < bwd / t["bwd_ms"] < 1.3, (bwd, t)


@pytest.mark.parametrize("kernel", KERNELS)
def test_two_detector_gradient_matches_oracle(F, A, kernel):
    """Coupler layout (plane-wave source, flux through the output waveguide L
    and above the device M): objectives and the gradient of s L + s2 M from
    one time-reversed run against the oracle's stored-history gradient."""
    w = I.coupler_small(n_steps=110)
    s1, s2 = 0.7, -1.3
    Lr, Mr, gr = O.gradient2(w, s1, s2)
    sim = F.Simulation(w)
    sim.set_option(A.OPT_KERNEL, kernel)
    eps = torch.from_numpy(w.eps).cuda()
    L = sim.forward(eps, A.record_cfg("f32", 1))
    L2, M = sim.objectives()
    assert L2 == L
    assert L == pytest.approx(Lr, rel=1e-5) and M == pytest.approx(Mr, rel=1e-5)
    g = sim.backward(s1, seed2=s2).cpu().numpy()
    assert rel(g, gr) < 1e-4


@pytest.mark.parametrize("tape", ["bf16:4:linear", "e4m3:2:cubic"])
def test_two_detector_compressed_tape_and_seed_errors(F, A, tape):
    """Both detectors seeded through a compressed tape (the transmission ratio
    of Sec. 4) against the oracle's FP64 run of the same method with the same
    tape settings and seeds: soft parity (a quantiser may round FP32 and FP64
    inputs to neighbouring codes)."""
    w = I.coupler_small(n_steps=110)
    dt, k, interp = tape.split(":")
    scaled = dt == "e4m3"
    Lm, Mm, gm = O.reverse2(w, dt, scaled=scaled, k=int(k), interp=interp, seed=1.0, seed2=-2.0)
    sim = F.Simulation(w)
    eps = torch.from_numpy(w.eps).cuda()
    L = sim.forward(eps, A.record_cfg(dt, int(k), interp))
    M = sim.objectives()[1]
    assert L == pytest.approx(Lm, rel=1e-5) and M == pytest.approx(Mm, rel=1e-5)
    g = sim.backward(1.0, seed2=-2.0).cpu().numpy()
    assert cos(g, gm) > 0.999
    assert rel(g, gm) < 2e-2
    # seed2 without a second detector is a state error
    w1 = w.replace(det2_kind=0)
    sim1 = F.Simulation(w1)
    sim1.forward(eps, A.record_cfg("f32", 1))
    with pytest.raises(A.FdtdError) as e:
        sim1.backward(1.0, seed2=1.0)
    assert e.value.status == A.FDTD_ESTATE


PAPER_FP8 = ["e4m3b11fnuz", "e5m2fnuz", "e4m3fnuz", "e4m3ieee", "e3m4"]


@pytest.mark.parametrize("fmt", PAPER_FP8)
@pytest.mark.parametrize("scaled", [False, True])
def test_paper_fp8_codec_is_bit_exact_against_oracle(F, A, fmt, scaled):
    """The software codec of the Sec. 4 formats equals the oracle's RNE
    quantiser (pinned by brute force over all codes) bit for bit, on values
    spanning subnormals, normals, ties and out-of-range magnitudes."""
    import ctypes as C
    rng = np.random.default_rng(5)
    fmax = O.format_max(fmt)
    n = 50021
    x = (rng.choice([-1, 1], n) * np.exp(rng.uniform(np.log(fmax) - 30, np.log(fmax) + 3, n)))
    # exact midpoints between neighbouring codes (ties)
    grid = np.unique(np.abs(O.quantize(fmt, np.exp(np.linspace(np.log(fmax) - 30,
                                                                np.log(fmax), 4000)))))
    mids = (grid[:-1] + grid[1:]) / 2
    x = np.concatenate([x, mids, -mids, [0.0, fmax, -fmax]]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    code = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    scale = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    A.check(A.lib().fdtd_encode(A.TAPE[fmt], int(scaled), C.c_void_p(xd.data_ptr()), x.size,
                                C.c_void_p(code.data_ptr()), C.c_void_p(scale.data_ptr()), None))
    A.check(A.lib().fdtd_decode(A.TAPE[fmt], C.c_void_p(code.data_ptr()), x.size,
                                C.c_void_p(scale.data_ptr()), C.c_void_p(out.data_ptr()), None))
    s32 = np.float32(1.0)
    if scaled:
        s32 = max(np.float32(np.abs(x).max()) / np.float32(fmax), np.float32(2.0 ** -126))
        assert scale.item() == s32
    q = O.quantize(fmt, (x / s32).astype(np.float32).astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(out.cpu().numpy(), q * s32)


@pytest.mark.parametrize("fmt,k", [("e4m3b11fnuz", 4), ("e5m2fnuz", 2), ("e3m4", 1)])
def test_paper_fp8_tape_matches_oracle_method(F, A, fmt, k):
    """Unscaled tape in the Sec. 4 formats against the oracle's run of the
    method with the same format."""
    w = I.ragged_box(n_steps=120)
    rec = A.record_cfg(fmt, k, "linear")
    assert rec.scaled == 0
    r = gpu_run(F, A, w, rec=rec)
    L, g = O.reverse(w, fmt, scaled=False, k=k, interp="linear")
    assert r["L"] == pytest.approx(L, rel=1e-5)
    assert rel(r["g"], g) < 2e-2
    assert cos(r["g"], g) > 0.999


@pytest.mark.parametrize("K", [1, 6, 10, 21, 64])
def test_bdct_codec_is_bit_exact_against_oracle(F, A, K):
    """Block-transform codec on raw planes (ragged sizes, values over many
    decades, all-zero and constant blocks): codes, scales and decoded values
    equal the oracle's float32 implementation bit for bit."""
    import ctypes as C
    rng = np.random.default_rng(K)
    for nv, nu in [(1, 1), (8, 8), (5, 11), (76, 176), (129, 37)]:
        x = (rng.standard_normal((nv, nu)) * np.exp(rng.uniform(-20, 3, (nv, nu))))
        x = x.astype(np.float32)
        if nu >= 16 and nv >= 16:
            x[:8, :8] = 0.0                    # an all-zero block
            x[8:16, 8:16] = 0.25               # a constant block
        nb = ((nu + 7) // 8) * ((nv + 7) // 8)
        xd = torch.from_numpy(x).cuda()
        codes = torch.zeros((nb, K), dtype=torch.int8, device="cuda")
        scales = torch.zeros(nb, dtype=torch.float32, device="cuda")
        out = torch.zeros((nv, nu), dtype=torch.float32, device="cuda")
        A.check(A.lib().fdtd_bdct_encode(C.c_void_p(xd.data_ptr()), nu, nv, K,
                                         C.c_void_p(codes.data_ptr()),
                                         C.c_void_p(scales.data_ptr()), None))
        A.check(A.lib().fdtd_bdct_decode(C.c_void_p(codes.data_ptr()),
                                         C.c_void_p(scales.data_ptr()), nu, nv, K,
                                         C.c_void_p(out.data_ptr()), None))
        oc, osc = O.bdct_encode(x, K)
        np.testing.assert_array_equal(codes.cpu().numpy(), oc)
        np.testing.assert_array_equal(scales.cpu().numpy(), osc)
        np.testing.assert_array_equal(out.cpu().numpy(), O.bdct_decode(oc, osc, nu, nv))


@pytest.mark.parametrize("name,k,interp", [("bdct10", 2, "cubic"), ("bdct21", 1, "linear"),
                                           ("bdct6", 4, "cubic")])
def test_bdct_tape_matches_oracle_method(F, A, name, k, interp):
    """Gradient with the block-transform tape against the oracle's run of the
    method with the same codec (its quantisation decisions are taken on the
    oracle's own FP64 fields rounded to float32, so a few codes may differ
    by one step: soft parity), for the default and the one-cell kernels."""
    w = I.ragged_box(n_steps=120)
    rec = A.record_cfg(name, k, interp)
    L, g = O.reverse(w, name, k=k, interp=interp)
    for kernel in (5, 0):
        r = gpu_run(F, A, w, rec=rec, options={A.OPT_KERNEL: kernel})
        assert r["L"] == pytest.approx(L, rel=1e-5)
        assert rel(r["g"], g) < 2e-2
        assert cos(r["g"], g) > 0.999


def test_bdct_coefficient_counts_are_not_mixed_up_by_cached_graphs(F, A):
    """One handle running the block codec with K = 6, then K = 21 (captured
    time-loop graphs are keyed by K too): the K = 21 results equal a fresh
    handle's bit for bit and differ from K = 6."""
    w = I.ragged_box(n_steps=60)
    eps = torch.from_numpy(w.eps).cuda()
    sim = F.Simulation(w)
    out = {}
    for name in ("bdct6", "bdct21"):
        sim.forward(eps, A.record_cfg(name, 2, "cubic"))
        out[name] = sim.backward().cpu().numpy()
    fresh = gpu_run(F, A, w, rec=A.record_cfg("bdct21", 2, "cubic"))
    np.testing.assert_array_equal(out["bdct21"], fresh["g"])
    assert not np.array_equal(out["bdct6"], out["bdct21"])


def test_autograd_function_against_central_differences(F, A):
    """FDTDGrad's backward vs central differences of its own forward (FP32
    fields, FP64 objective).  Along the gradient direction the derivative is
    |g|, large against the FP32 rounding noise of L; along a random direction
    it is ~1e-2 |g| and the difference step is widened accordingly."""
    w = I.ragged_box(n_steps=100)
    sim = F.Simulation(w)
    rec = A.record_cfg("f32", 1)
    eps_bg = torch.from_numpy(w.eps).cuda()
    d = torch.from_numpy(w.eps[w.design_slice()].copy()).cuda().requires_grad_(True)
    L = F.objective(d, eps_bg, sim, rec)
    L.backward()
    g = d.grad.double()
    rnd = torch.from_numpy(np.random.default_rng(5).standard_normal(w.design_shape)).cuda()
    # perturb only cells whose eps stays >= 1 under the step (eps >= 1 is required)
    mask = (d.detach() >= 1.6).double()
    vg, vr = g * mask, rnd * mask
    for v, h, tol in ((vg / vg.norm(), 0.05, 2e-3), (vr / vr.norm(), 0.3, 5e-2)):
        Lp = F.objective((d.detach().double() + h * v).float(), eps_bg, sim, rec).item()
        Lm = F.objective((d.detach().double() - h * v).float(), eps_bg, sim, rec).item()
        fd = (Lp - Lm) / (2 * h)
        an = float((g * v).sum())
        assert abs(fd - an) <= tol * abs(an), (fd, an)


def test_host_buffer_path_matches_device_path(F, A):
    w = SMALL["ragged_poynting"]()
    rec = A.record_cfg("bf16", 2, "cubic")
    r = gpu_run(F, A, w, rec=rec, seed=0.75)
    sim = F.Simulation(w)
    eps_h = torch.from_numpy(w.eps).pin_memory()
    L, gh = sim.value_and_grad_host(eps_h, rec, seed=0.75)
    assert L == pytest.approx(r["L"], rel=1e-12)
    np.testing.assert_allclose(gh.numpy(), r["g"], rtol=1e-12, atol=1e-30)


def test_group_calls_match_single_calls(F, A):
    ws = I.batched_cubes(n_sims=3, sizes=(32, 36, 40), steps=(60, 90))
    rec = A.record_cfg("bf16", 4, "linear")
    sims = [F.Simulation(w) for w in ws]
    eps = [torch.from_numpy(w.eps).cuda() for w in ws]
    objs = F.group_forward(sims, eps, rec)
    grads = F.group_backward(sims, seeds=[1.0, 2.0, -1.0])
    for w, o, g, s in zip(ws, objs, grads, [1.0, 2.0, -1.0]):
        r = gpu_run(F, A, w, rec=rec, seed=s)
        assert o == pytest.approx(r["L"], rel=1e-12)
        np.testing.assert_allclose(g.cpu().numpy(), r["g"], rtol=1e-10, atol=1e-30)


def _degenerate_cases():
    cube = I.fd_cube()
    rb = I.ragged_box(nx=35, ny=17, nz=15, P=3, n_steps=40)
    P = rb.pml_thickness
    return {
        # one time step: a single recorded sample
        "one_step": cube.replace(n_steps=1, det_index=3),
        # smallest grid the API accepts: 2P+2 cells per axis (a 2-cell interior)
        "min_grid": cube.replace(nx=6, ny=6, nz=6, eps=np.ones((6, 6, 6), np.float32),
                                 design_lo=(2, 2, 2), design_hi=(4, 4, 4), src_pos=(2, 3, 2),
                                 det_index=3, det_lo=(2, 2), det_hi=(4, 4)),
        # a one-cell design box and a one-cell detector window
        "one_cell": rb.replace(design_lo=(P + 4, P + 2, P + 3), design_hi=(P + 5, P + 3, P + 4),
                               det_lo=(P + 1, P + 1), det_hi=(P + 2, P + 2)),
    }


@pytest.mark.parametrize("name", ["one_step", "min_grid", "one_cell"])
@pytest.mark.parametrize("kernel", [0, 5])
def test_degenerate_problems(F, A, name, kernel):
    w = _degenerate_cases()[name]
    L, g = O.gradient(w)
    r = gpu_run(F, A, w, options={A.OPT_KERNEL: kernel})
    assert r["L"] == pytest.approx(L, rel=1e-5, abs=1e-30)
    if np.abs(g).max() > 0:
        assert rel(r["g"], g) < 1e-4
    else:
        assert np.abs(r["g"]).max() == 0.0


@pytest.mark.parametrize("k", [7, 100])
def test_subsampling_longer_than_the_run(F, A, k):
    """k >= n_steps keeps only the last step (plus the known zero state) and
    still matches the oracle's run of the method."""
    w = I.ragged_box(n_steps=40)
    r = gpu_run(F, A, w, rec=A.record_cfg("f32", k, "linear"))
    Lm, gm = O.reverse(w, "f32", k=k, interp="linear")
    assert r["L"] == pytest.approx(Lm, rel=1e-5)
    assert rel(r["g"], gm) < 1e-3


@pytest.mark.parametrize("kernel", [0, 5])
def test_time_reversal_returns_to_the_initial_state(F, A, kernel):
    """After the backward run the reconstructed interior state is the zero
    initial state (E^0 = 0, Ht^{-1/2} = 0) up to the FP32 drift of the
    reversal (Sec. 1-2: the interior is stepped backwards exactly in exact
    arithmetic).  The drift is reported relative to the peak field."""
    w = SMALL["ragged_poynting"]()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_KERNEL, kernel)
    eps = torch.from_numpy(w.eps).cuda()
    sim.forward(eps, A.record_cfg("f32", 1))
    end = sim.read_fields().cpu().numpy()
    sim.backward()
    back = sim.read_fields().cpu().numpy()
    P = w.pml_thickness
    interior = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    peak = np.abs(end[interior]).max()
    drift = np.abs(back[interior]).max() / peak
    print(f"kernel {kernel}: reversal drift {drift:.2e} of the peak field")
    assert peak > 0 and drift < 1e-4


def rounding_bound(w, q):
    """Bound on the L2 error of the final fields of the scheme with
    increments rounded to multiples of 2^-q against the unrounded one: each
    step adds at most 2^-(q+1) per field value, and the leapfrog does not
    amplify an error by more than a constant (taken as 4, generous for
    S = 0.99/sqrt(3) with the CPML damping)."""
    return 4.0 * w.n_steps * 2.0 ** -(q + 1) * np.sqrt(6 * w.nx * w.ny * w.nz)


@pytest.mark.parametrize("name", ["ragged_poynting", "ragged_e2_point"])
def test_exact_reversal_retraces_the_forward_bit_for_bit(F, A, name):
    """With increments rounded to multiples of 2^-22 every float32 update of
    the leapfrog is exact, so after the backward run the reconstructed
    interior is the zero initial state bit for bit (plain float32 increments
    leave a drift of ~1e-7 of the peak).  The rounded scheme differs from the
    FP64 oracle's unrounded one by at most the accumulated rounding, and its
    gradient stays within the FP32 parity bounds of the full-size test."""
    q = 22
    w = SMALL[name]()
    sim = F.Simulation(w)
    sim.set_option(A.OPT_EXACT_REVERSAL, q)
    eps = torch.from_numpy(w.eps).cuda()
    L = sim.forward(eps, A.record_cfg("f32", 1))
    end = sim.read_fields().cpu().numpy()
    g = sim.backward().cpu().numpy()
    back = sim.read_fields().cpu().numpy()
    P = w.pml_thickness
    interior = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(end[interior]).max() > 0
    np.testing.assert_array_equal(back[interior], np.zeros_like(back[interior]))
    Lr, gr, st = O.gradient(w, want_state=True)
    err = np.linalg.norm((end[:6] - st[:6]).ravel())
    print(f"{name}: field error {err:.2e} (bound {rounding_bound(w, q):.2e}), "
          f"L rel {abs(L - Lr) / abs(Lr):.1e}, grad rel {rel(g, gr):.2e}, cos {cos(g, gr):.7f}")
    assert err < rounding_bound(w, q)
    assert L == pytest.approx(Lr, rel=1e-4)
    assert rel(g, gr) < 1e-3 and cos(g, gr) > 0.99999


def test_exact_reversal_on_the_benchmark_grid(F, A):
    """The 200 x 200 x 100 grid in the default launch configuration (100
    steps): the interior returns to zero bit for bit and the fields stay
    within the accumulated rounding of the FP64 oracle's unrounded scheme.
    The objective of this early-pulse case (L ~ 3.5e-7) comes from detector
    fields ~1e-3 of the peak, where an absolute grid of 2^-22 is coarse:
    its L and gradient are reported, not held to the FP32 parity bounds."""
    q = 22
    w = I.waveguide_mid().replace(n_steps=100, t0_over_tau=0.3, det_index=60)
    L, g, st = O.gradient(w, want_state=True)
    r = gpu_run(F, A, w, options={A.OPT_EXACT_REVERSAL: q})
    back = r["sim"].read_fields().cpu().numpy()
    P = w.pml_thickness
    interior = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    np.testing.assert_array_equal(back[interior], np.zeros_like(back[interior]))
    err = np.linalg.norm((r["fields"][:6] - st[:6]).ravel())
    print(f"benchmark grid: field error {err:.2e} (bound {rounding_bound(w, q):.2e}), "
          f"L rel {abs(r['L'] - L) / abs(L):.1e}, grad rel {rel(r['g'], g):.2e}, "
          f"cos {cos(r['g'], g):.7f}")
    assert err < rounding_bound(w, q)


def test_large_grid_properties_at_full_size(F, A):
    """The 600 x 600 x 300 grid (108 M cells, 16-cell CPML) in the default
    launch configuration, 200 steps of an early pulse with the BF16 k = 4
    tape of the benchmark: the compact auxiliary layout gives the same fields
    bit for bit and the same gradient as the full-grid layout in less memory,
    and with exact reversal (FP32 k = 1 tape) the interior returns to zero
    bit for bit."""
    # the pulse from x = 20 reaches the design region (x >= 100) and the
    # detector plane at x = 120 within 200 steps
    w = I.waveguide_large(n_steps=200).replace(t0_over_tau=0.3, det_index=120)
    rec = A.record_cfg("bf16", 4, "linear")
    a = gpu_run(F, A, w, rec=rec)
    b = gpu_run(F, A, w, rec=rec, options={A.OPT_COMPACT_AUX: 0})
    np.testing.assert_array_equal(a["fields"], b["fields"])
    assert np.abs(a["g"]).max() > 0
    same_gradient(a["g"], b["g"])
    assert a["sim"].workspace_bytes(rec) < b["sim"].workspace_bytes(rec)
    del a, b
    r = gpu_run(F, A, w, options={A.OPT_EXACT_REVERSAL: 22})
    back = r["sim"].read_fields().cpu().numpy()
    P = w.pml_thickness
    interior = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(r["fields"][interior]).max() > 0
    assert not np.any(back[interior])


def test_full_size_waveguide_in_the_benchmark_configuration(F, A):
    """The 200 x 200 x 100 benchmark grid with its own source (the Gaussian
    pulse centred at 3 tau) in the default launch configuration, shortened to
    700 steps and with the detector moved into the design region's x range
    (x = 60), so that the FP64 oracle computes every output and both L and
    dL/d(eps) are non-zero (79 % of the design cells above 1e-6 of the
    maximum): forward fields, objective and the uncompressed-tape gradient at
    the stated tolerances."""
    w = I.waveguide_mid().replace(n_steps=700, det_index=60)
    L, g, st = O.gradient(w, want_state=True)
    assert L != 0.0 and np.abs(g).max() > 0
    r = gpu_run(F, A, w)
    eE, eH = field_err(r["fields"], st)
    assert eE < 1e-5 and eH < 1e-5, (eE, eH)
    assert r["L"] == pytest.approx(L, rel=1e-5)
    assert rel(r["g"], g) < 1e-4, rel(r["g"], g)
    r0 = gpu_run(F, A, w, options={A.OPT_KERNEL: 0})
    np.testing.assert_array_equal(r0["fields"], r["fields"])
    same_gradient(r["g"], r0["g"])


def test_largest_grid_in_the_bench_configuration(F, A):
    """600 x 600 x 300 cells, 10 000 steps, the E4M3 tape every 8th step: the
    bench's line, with the library's default steps (two time steps per pass
    forward, fused reverse), against the split half-steps and phases.  The oracle cannot run
    this grid, so properties that hold at any size stand in: forward fields
    bit for bit, the objective to the FP64 sums' order, the gradient finite
    and within 1e-5 of the split kernels' over a run long enough for an
    adjoint term left out to grow without bound."""
    w = I.waveguide_large(n_steps=10000)
    rec = A.record_cfg("e4m3", 8, "linear")
    Lf, ff, gf, _ = run_forward_way(F, A, w, rec, 0, 0)
    torch.cuda.empty_cache()
    Ls, fs, gs, _ = run_forward_way(F, A, w, rec, 1, 1)
    torch.cuda.empty_cache()
    assert np.abs(fs).max() > 0 and np.abs(gs).max() > 0
    np.testing.assert_array_equal(ff, fs)
    assert Lf == pytest.approx(Ls, rel=1e-12)
    assert np.all(np.isfinite(gf))
    assert rel(gf, gs) < 1e-5


def test_largest_grid_against_the_oracle_near_the_source(F, A):
    """All 108 M cells of the 600 x 600 x 300 grid in the bench's launch
    configuration (two time steps per pass forward, fused reverse, FP32
    tape of every step), against the FP64 oracle: the Poynting detector moved
    to x = 28 and the design box to x in [21, 28) around the strip, between
    the source plane (x = 20) and the detector, so that L and dL/d(eps) are
    non-zero within 120 steps.  Source and detector stay two cells or more
    away from the deep units (x >= 32), as the two-step pass needs.  Fields after the forward within 1e-5, the objective within 1e-5,
    the gradient within 1e-4."""
    w = I.waveguide_large(n_steps=120)
    P, yc, zc = w.pml_thickness, w.ny // 2, w.nz // 2
    w = w.replace(det_index=28, design_lo=(21, yc - 16, zc - 11), design_hi=(28, yc + 16, zc + 11))
    L, g, st = O.gradient(w, want_state=True)
    assert L != 0.0 and np.abs(g).max() > 0
    sim = F.Simulation(w)
    for opt in (A.OPT_FORWARD, A.OPT_REVERSE):
        assert sim.get_option(opt) == 0
    eps = torch.from_numpy(w.eps).cuda()
    Lg = sim.forward(eps, A.record_cfg("f32", 1))
    # per pair of steps: the pass, 2 x 4 split launches over the other units, 2 records
    assert sim.last_timing()["fwd_launches"] == 11 * w.n_steps // 2
    fields = sim.read_fields().cpu().numpy()
    eE, eH = field_err(fields, st)
    del st
    assert eE < 1e-5 and eH < 1e-5, (eE, eH)
    assert Lg == pytest.approx(L, rel=1e-5)
    gg = sim.backward(1.0).cpu().numpy()
    assert sim.last_timing()["bwd_launches"] == 5 * w.n_steps   # fused: restore, primal, 3 adjoint
    assert rel(gg, g) < 1e-4, rel(gg, g)
    del sim
    torch.cuda.empty_cache()


def test_largest_grid_compressed_tape_against_the_oracle_method(F, A):
    """The same full-size case with the bench's tape (E4M3 with per-face
    scales, every 8th step, linear): the GPU gradient against the oracle's
    FP64 run of the method with the same quantiser and interpolation, at the
    compressed-tape bar (relative L2 2e-2, cosine 0.999)."""
    w = I.waveguide_large(n_steps=120)
    yc, zc = w.ny // 2, w.nz // 2
    w = w.replace(det_index=28, design_lo=(21, yc - 16, zc - 11), design_hi=(28, yc + 16, zc + 11))
    Lm, gm = O.reverse(w, fmt="e4m3", scaled=True, k=8, interp="linear")
    assert np.abs(gm).max() > 0
    sim = F.Simulation(w)
    eps = torch.from_numpy(w.eps).cuda()
    Lg = sim.forward(eps, A.record_cfg("e4m3", 8, "linear"))
    gg = sim.backward(1.0).cpu().numpy()
    assert Lg == pytest.approx(Lm, rel=1e-5)
    assert rel(gg, gm) < 2e-2, rel(gg, gm)
    assert cos(gg, gm) > 0.999
    del sim
    torch.cuda.empty_cache()


def test_largest_grid_exact_reversal_returns_to_zero(F, A):
    """The same grid, 300 steps, exact reversal through the default steps:
    the interior returns to the zero initial state bit for bit."""
    w = I.waveguide_large(n_steps=300)
    _, fwd, _, back = run_forward_way(F, A, w, A.record_cfg("f32", 1), 0, 0,
                                      {A.OPT_EXACT_REVERSAL: 22})
    torch.cuda.empty_cache()
    P = w.pml_thickness
    inner = (slice(None), slice(P, w.nz - P), slice(P, w.ny - P), slice(P, w.nx - P))
    assert np.abs(fwd[inner]).max() > 0
    assert not np.any(back[inner])


def test_reversal_drift_report_with_an_abruptly_switched_source(F, A):
    """Drift report, not parity: a source switched on at 0.3 tau (not the
    benchmark's pulse) drives content up to the grid's Nyquist limit, where
    float32 time reversal of 100 steps reproduces the gradient only to ~2e-4
    (printed).  The bound checked is that drift's order; the plain-load
    kernels, an independent variant, agree with the default ones to
    rounding."""
    w = I.waveguide_mid().replace(n_steps=100, t0_over_tau=0.3, det_index=60)
    L, g = O.gradient(w)
    r = gpu_run(F, A, w)
    drift = rel(r["g"], g)
    print(f"reversal drift, abrupt source, 100 steps: gradient rel. error {drift:.2e}")
    assert drift < 1e-3
    r0 = gpu_run(F, A, w, options={A.OPT_KERNEL: 0})
    same_gradient(r["g"], r0["g"])


def test_full_length_benchmark_forward(F, A):
    """The benchmark workload itself (200 x 200 x 100, 2000 steps, BF16 tape
    k = 4, default launch configuration) against the FP64 oracle's forward:
    the objective of every step (the detector plane sampled 2000 times) and
    the final fields.  After 2000 steps the pulse has left the grid and the
    final state is a residue of ~1e-3 of the peak field, whose relative error
    is correspondingly larger than mid-run."""
    w = I.waveguide_mid()
    st, obj = O.forward(w)
    r = gpu_run(F, A, w, rec=A.record_cfg("bf16", 4, "linear"))
    np.testing.assert_allclose(r["hist"], obj, rtol=0, atol=1e-5 * np.abs(obj).max())
    assert r["L"] == pytest.approx(obj.sum(), rel=1e-5)
    eE, eH = field_err(r["fields"], st)
    assert eE < 1e-2 and eH < 1e-2, (eE, eH)


def test_bounded_device_wait_reports_a_timeout(F, A):
    """Failure detection without a fault: a wait that nothing completes gives
    up after its limit, the host reads FDTD_ETIMEOUT, and the context stays
    usable for a normal run afterwards."""
    import ctypes as C
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = A.lib().fdtd_selftest_wait(C.c_void_p(flag.data_ptr()), 20_000_000, None)
    assert rc == A.FDTD_ETIMEOUT
    assert int(flag.item()) & 4
    assert A.lib().fdtd_selftest_wait(C.c_void_p(flag.data_ptr()), 0, None) == A.FDTD_EINVAL
    assert A.lib().fdtd_selftest_wait(None, 1000, None) == A.FDTD_EINVAL
    w = SMALL["fd_cube"]()
    r = gpu_run(F, A, w)
    L, g = O.gradient(w)
    assert rel(r["g"], g) < 1e-4


def test_error_statuses(F, A):
    import ctypes as C
    w = SMALL["fd_cube"]()
    sim = F.Simulation(w)
    rec = A.record_cfg("f32", 1)
    sim.ensure_workspace(rec)
    g = torch.empty(w.design_shape, device="cuda")
    rc = A.lib().fdtd_backward(sim.h, 1.0, C.c_void_p(g.data_ptr()))
    assert rc == A.FDTD_ESTATE
    bad = torch.from_numpy(w.eps).cuda()
    bad[4, 4, 4] = 0.5
    with pytest.raises(A.FdtdError) as e:
        sim.forward(bad, rec)
    assert e.value.status == A.FDTD_ENONFINITE
    bad[4, 4, 4] = float("nan")
    with pytest.raises(A.FdtdError) as e:
        sim.forward(bad, rec)
    assert e.value.status == A.FDTD_ENONFINITE
    # a valid run afterwards still works and a second backward is refused
    sim.forward(torch.from_numpy(w.eps).cuda(), rec)
    sim.backward()
    rc = A.lib().fdtd_backward(sim.h, 1.0, C.c_void_p(g.data_ptr()))
    assert rc == A.FDTD_ESTATE


@pytest.mark.parametrize("dtype", ["f16", "e4m3"])
def test_scaled_codec_on_vanishing_faces_stays_finite(F, A, dtype):
    """A face whose absmax is far below FP32's normal range must not produce a
    zero scale (0/0 would encode NaN): the scale is at least 2^-126."""
    import ctypes as C
    x = np.array([1e-43, -5e-44, 0.0, 3e-45], np.float32)
    xd = torch.from_numpy(x).cuda()
    tdt = {"f16": torch.float16, "e4m3": torch.float8_e4m3fn}[dtype]
    code = torch.empty(x.size, dtype=tdt, device="cuda")
    scale = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    A.check(A.lib().fdtd_encode(A.TAPE[dtype], 1, C.c_void_p(xd.data_ptr()), x.size,
                                C.c_void_p(code.data_ptr()), C.c_void_p(scale.data_ptr()), None))
    A.check(A.lib().fdtd_decode(A.TAPE[dtype], C.c_void_p(code.data_ptr()), x.size,
                                C.c_void_p(scale.data_ptr()), C.c_void_p(out.data_ptr()), None))
    assert scale.item() == np.float32(2.0 ** -126)
    o = out.cpu().numpy()
    assert np.isfinite(o).all() and np.abs(o).max() <= 1e-37


def test_compressed_tape_with_vanishing_boundary_fields(F, A):
    """Early in a run most boundary faces carry only the tiny leading edge of
    the field; the scaled FP8 tape must still give a finite gradient that
    agrees with the oracle's run of the method."""
    w = I.ragged_box(n_steps=24)
    rec = A.record_cfg("e4m3", 1, "linear")
    r = gpu_run(F, A, w, rec=rec)
    L, g = O.reverse(w, "e4m3", scaled=True, k=1, interp="linear")
    assert np.isfinite(r["g"]).all()
    assert cos(r["g"], g) > 0.999
