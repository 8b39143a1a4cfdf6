"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to something the paper or the
mathematics fixes: the paper's printed numbers (Eq. 1 and the text after it),
the Yee dispersion relation (closed form), the discrete leapfrog energy
(invariant), exact time reversal, the transpose identity <v, F u> = <F^T v, u>,
brute-force central differences, library float casts and polynomial
exactness of the interpolants.
"""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import oracle as O
from paper_2603_24027_gb300 import inputs as I

C0 = 299792458.0


def box(nx, ny, nz, P=0, n_steps=10, eps=None, **kw):
    eps = np.ones((nz, ny, nx), np.float32) if eps is None else eps
    base = dict(name="t", nx=nx, ny=ny, nz=nz, dx=20e-9, dt=I.cfl_dt(20e-9), n_steps=n_steps,
                pml_thickness=P, eps=eps, design_lo=(P, P, P), design_hi=(nx - P, ny - P, nz - P),
                src_kind=I.SRC_NONE, det_kind=0)
    base.update(kw)
    return I.Workload(**base)


# ------------------------------------------------------------ Eq. 1 -------

def test_eq1_numbers_from_the_paper():
    g = golden("paper_numbers.txt")
    assert I.COURANT == g["courant_factor"][0]
    assert I.C0 == g["speed_of_light_m_s"][0]
    dt = I.cfl_dt(20e-9)
    v, tol = g["dt_at_dx20nm_s"]
    assert abs(dt - v) / v < tol
    v, tol = g["period_1550nm_s"]
    period = 1550e-9 / C0
    assert abs(period - v) / v < tol
    v, tol = g["steps_per_period_1550nm"]
    assert abs(period / dt - v) / v < tol


def test_waveform_carrier_period_matches_paper():
    """Zero crossings of the oracle's source waveform at dx = 20 nm are spaced
    by half of ~136 steps (Sec. 2: 1550 nm ~ 136 time steps)."""
    w = box(8, 8, 8, n_steps=4000, src_kind=I.SRC_POINT, src_pos=(4, 4, 4), t0_over_tau=3.0)
    g = O.waveform(w)
    s = np.sign(g)
    idx = np.nonzero((s[:-1] * s[1:]) < 0)[0]
    # keep crossings where the envelope is well above rounding
    env = np.abs(g).max()
    good = [i for i in idx if max(abs(g[i - 30:i + 30]).max(), 0) > 1e-3 * env]
    # sub-step crossing positions by linear interpolation
    xs = np.array([i + g[i] / (g[i] - g[i + 1]) for i in good])
    half = np.diff(xs).mean()
    steps_per_period = golden("paper_numbers.txt")["steps_per_period_1550nm"][0]
    assert abs(2 * half - steps_per_period) / steps_per_period < 1e-2
    # closed form lambda0 / (S dx) with S = 0.99/sqrt(3)
    S = C0 * w.dt / w.dx
    assert abs(2 * half - 1550e-9 / (S * 20e-9)) < 0.05


def test_waveform_bandwidth_is_30_percent_fwhm():
    """Power-spectrum FWHM of the pulse equals rel_bandwidth * w0."""
    w = box(8, 8, 8, n_steps=20000, src_kind=I.SRC_POINT, src_pos=(4, 4, 4), t0_over_tau=6.0)
    g = O.waveform(w)
    n = 1 << 18
    spec = np.abs(np.fft.rfft(g, n)) ** 2
    f = np.fft.rfftfreq(n)               # cycles per step
    k = spec.argmax()
    half = spec[k] / 2
    lo = np.nonzero(spec[:k] < half)[0][-1]
    hi = k + np.nonzero(spec[k:] < half)[0][0]
    fwhm = f[hi] - f[lo]
    S = C0 * w.dt / w.dx
    f0 = S * w.dx / w.lambda0            # cycles per step
    assert abs(f[k] - f0) / f0 < 2e-3
    assert abs(fwhm / f0 - 0.3) < 5e-3


# ------------------------------------------------ Yee dispersion ----------

@pytest.mark.parametrize("mode", ["Ez_xy", "Ex_yz", "Ey_zx"])
@pytest.mark.parametrize("eps_r", [1.0, 2.25])
def test_yee_dispersion_closed_form(mode, eps_r):
    """A transverse standing mode cos(k.r) on a periodic grid obeys
    E^{n+1} + E^{n-1} = (2 - 4 (S^2/eps) sum_i sin^2(k_i/2)) E^n exactly
    (discrete curl-curl eigenvalue); a sign or index error in any of the
    curl terms used by the mode breaks it."""
    nx, ny, nz = 16, 12, 10
    eps = np.full((nz, ny, nx), eps_r, np.float32)
    w = box(nx, ny, nz, eps=eps, n_steps=60)
    kx, ky, kz = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny, 2 * np.pi * 1 / nz
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    st = O.zero_state(w)
    comp, ks = {"Ez_xy": (2, (kx, ky)), "Ex_yz": (0, (ky, kz)), "Ey_zx": (1, (kz, kx))}[mode]
    phase = {"Ez_xy": kx * x + ky * y, "Ex_yz": ky * y + kz * z, "Ey_zx": kz * z + kx * x}[mode]
    st[comp] = np.cos(phase)
    S = C0 * w.dt / w.dx
    coef = 2 - 4 * S * S / eps_r * sum(math.sin(kk / 2) ** 2 for kk in ks)
    hist = [st[comp].copy()]
    for n in range(40):
        O.step(w, st, n, periodic=1)
        hist.append(st[comp].copy())
        others = [c for c in range(3) if c != comp]
        assert np.abs(st[others]).max() < 1e-12
    for n in range(1, 40):
        np.testing.assert_allclose(hist[n + 1] + hist[n - 1], coef * hist[n], atol=1e-12, rtol=0)


# ------------------------------------------------------ energy -------------

def test_leapfrog_energy_is_conserved_in_a_zero_padded_box():
    """W^n = sum eps E^n.E^n + sum Ht^{n-1/2}.Ht^{n+1/2} is invariant for the
    lossless update when curlH is the transpose of curlE (zero padding)."""
    nx, ny, nz = 10, 9, 8
    rng = np.random.default_rng(1)
    eps = rng.uniform(1.0, 12.25, (nz, ny, nx)).astype(np.float32)
    w = box(nx, ny, nz, eps=eps, n_steps=2000)
    st = O.zero_state(w)
    st[:6] = I.random_state((nz, ny, nx), 7, 6)
    e64 = eps.astype(np.float64)
    W = []
    for n in range(2000):
        E = st[:3].copy()
        Hm = st[3:6].copy()
        O.step(w, st, n)
        W.append(np.sum(e64 * E * E) + np.sum(Hm * st[3:6]))
    W = np.array(W)
    assert W[0] > 0
    assert np.abs(W / W[0] - 1).max() < 1e-12


# ----------------------------------------------------- reversal -----------

def test_exact_time_reversal_without_pml():
    """N steps forward then N inverse steps recover (E^0, Ht^{-1/2}) to FP64
    rounding (the premise of time-reversible gradients, Sec. 1)."""
    nx, ny, nz = 12, 11, 9
    rng = np.random.default_rng(2)
    eps = rng.uniform(1.0, 12.25, (nz, ny, nx)).astype(np.float32)
    w = box(nx, ny, nz, eps=eps, n_steps=300, src_kind=I.SRC_POINT, src_component=1,
            src_pos=(5, 4, 3), t0_over_tau=0.3)
    st = O.zero_state(w)
    st[:6] = I.random_state((nz, ny, nx), 3, 6)
    init = st[:6].copy()
    O.run(w, st, 0, 300)
    assert np.abs(st[:6] - init).max() > 0.1
    for n in range(299, -1, -1):
        O.unstep(w, st, n)
    assert np.abs(st[:6] - init).max() < 1e-11 * np.abs(init).max()


# -------------------------------------------------- CPML structure ---------

def test_cpml_profiles_vanish_exactly_on_the_lossless_interior():
    """Interior cells [P, N-P) must see b = a = 0 and 1/kappa = 1 at both the
    E and H positions, and every PML cell must be lossy, so the interior
    update is exactly invertible and the layer absorbs."""
    w = I.small_dipole()
    P = w.pml_thickness
    for ax, n in enumerate((w.nx, w.ny, w.nz)):
        pr = O.profiles(w, ax)
        inner = slice(P, n - P)
        for key in ("b_e", "a_e", "b_h", "a_h"):
            assert np.all(pr[key][inner] == 0.0)
        assert np.all(pr["kinv_e"] == 1.0) and np.all(pr["kinv_h"] == 1.0)
        for key in ("a_e", "a_h"):
            assert np.all(pr[key][:P] < 0) and np.all(pr[key][n - P:] < 0)
        for key in ("b_e", "b_h"):
            assert np.all((pr[key][:P] > 0) & (pr[key][:P] < 1))
        # grading deepens toward the outer faces on both sides
        assert np.all(np.diff(pr["b_e"][:P]) > 0) and np.all(np.diff(pr["b_h"][n - P:]) < 0)
        # mirror symmetry of the Yee grid: E positions on the low side match
        # H positions on the high side
        np.testing.assert_allclose(pr["b_e"][:P], pr["b_h"][n - P:][::-1], rtol=1e-15)
        np.testing.assert_allclose(pr["b_h"][:P], pr["b_e"][n - P:][::-1], rtol=1e-15)


def test_cpml_absorbs_an_outgoing_pulse():
    """A dipole pulse radiating in vacuum leaves the box through the CPML: the
    field energy left in the interior long after the pulse is below 1e-9 of
    its peak, while with the absorbing profiles switched off the radiated
    share (~1e-4 of the peak) stays in the box."""
    n, P, T = 40, 10, 1500
    # t0 = 4 tau: the pulse starts from ~0 and carries no DC current, which
    # would otherwise leave a static dipole field behind.
    w = box(n, n, n, P=P, n_steps=T, src_kind=I.SRC_POINT, src_component=2,
            src_pos=(20, 20, 20), t0_over_tau=4.0, dx=25e-9, dt=I.cfl_dt(25e-9))
    inner = (slice(P, n - P),) * 3

    def energy_trace(wl):
        st = O.zero_state(wl)
        out = []
        for s in range(0, T, 100):
            O.run(wl, st, s, 100)
            out.append(sum(np.sum(st[c][inner] ** 2) for c in range(6)))
        return np.array(out)

    e_pml = energy_trace(w)
    e_off = energy_trace(w.replace(pml_sigma_factor=0.0, pml_alpha_factor=0.0))
    # The peak is dominated by the dipole's reactive near field; what radiates
    # is ~1e-4 of it.  Lossless layers keep that share, the CPML removes it.
    assert e_pml[-1] < 1e-9 * e_pml.max()
    assert e_off[-1] > 1e-5 * e_off.max()


# -------------------------------------------------- transpose ---------------

@pytest.mark.parametrize("kappa", [1.0, 3.0])
def test_adjoint_step_is_the_transpose(kappa):
    """<v, F u> = <F^T v, u> for one step on the full state (fields and all 12
    psi arrays) with CPML on every face, random eps and kappa grading."""
    nx, ny, nz, P = 14, 12, 11, 3
    rng = np.random.default_rng(4)
    eps = rng.uniform(1.0, 12.25, (nz, ny, nx)).astype(np.float32)
    w = box(nx, ny, nz, P=P, eps=eps, pml_kappa_max=kappa)
    u = I.random_state((nz, ny, nx), 11, O.NF)
    v = I.random_state((nz, ny, nx), 12, O.NF)
    Fu = u.copy()
    O.step(w, Fu, 0)
    Ftv = v.copy()
    O.step_adjoint(w, Ftv)
    lhs, rhs = np.sum(v * Fu), np.sum(Ftv * u)
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(v * Fu).sum())


def test_adjoint_of_three_steps_composes():
    nx, ny, nz, P = 11, 10, 9, 2
    rng = np.random.default_rng(5)
    eps = rng.uniform(1.0, 12.25, (nz, ny, nx)).astype(np.float32)
    w = box(nx, ny, nz, P=P, eps=eps)
    u = I.random_state((nz, ny, nx), 21, O.NF)
    v = I.random_state((nz, ny, nx), 22, O.NF)
    Fu = u.copy()
    for n in range(3):
        O.step(w, Fu, n)
    Ftv = v.copy()
    for n in range(3):
        O.step_adjoint(w, Ftv)
    assert abs(np.sum(v * Fu) - np.sum(Ftv * u)) <= 1e-13 * np.abs(v * Fu).sum()


# ------------------------------------------------ finite differences --------

def _fd_check(w, cells, h, rtol):
    L0, g = O.gradient(w)
    gmax = np.abs(g).max()
    for (z, y, x) in cells:
        e = w.eps.astype(np.float64)
        c = (z + w.design_lo[2], y + w.design_lo[1], x + w.design_lo[0])
        ep, em = e.copy(), e.copy()
        ep[c] += h
        em[c] -= h
        Lp = O.forward(w.replace(eps=ep))[1].sum()
        Lm = O.forward(w.replace(eps=em))[1].sum()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[z, y, x]) <= rtol * gmax, (c, fd, g[z, y, x])
    return L0, g


def test_gradient_matches_central_differences_on_every_design_cell():
    """Brute force on an 8^3 grid (2-cell CPML, 4^3 design = interior,
    |E|^2 objective, point source): all 64 cells."""
    w = I.fd_cube()
    cells = [(z, y, x) for z in range(4) for y in range(4) for x in range(4)]
    L0, g = _fd_check(w, cells, 1e-5, 1e-7)
    assert L0 > 0 and np.abs(g).max() > 0


def test_gradient_matches_central_differences_poynting_plane_source():
    """Poynting objective and Gaussian plane source on an odd-sized grid."""
    w = I.ragged_box(nx=13, ny=11, nz=10, P=2, n_steps=50)
    rng = np.random.default_rng(6)
    shp = w.design_shape
    cells = [tuple(int(rng.integers(0, s)) for s in shp) for _ in range(12)]
    L0, g = _fd_check(w, cells, 1e-5, 1e-7)
    assert np.abs(g).max() > 0


def _swap_detectors(w):
    """The workload with its second detector as the objective detector."""
    return w.replace(det_kind=w.det2_kind, det_axis=w.det2_axis, det_index=w.det2_index,
                     det_lo=w.det2_lo, det_hi=w.det2_hi, det2_kind=0)


def test_two_detector_gradient_matches_central_differences():
    """Transmission-ratio ingredients (Sec. 4): the stored-history gradient of
    s L + s2 M (L through the output waveguide, M above the coupler, plane-wave
    source) against central differences of the same combination."""
    w = I.coupler_small(n_steps=70)
    s1, s2 = 0.7, -1.3
    L, M, g = O.gradient2(w, s1, s2)
    assert L != 0.0 and M != 0.0
    # each objective on its own equals the single-detector path
    L1, g1 = O.gradient(w)
    M1, gm = O.gradient(_swap_detectors(w))
    assert L1 == pytest.approx(L, rel=1e-14) and M1 == pytest.approx(M, rel=1e-14)
    np.testing.assert_allclose(g, s1 * g1 + s2 * gm, rtol=0, atol=1e-12 * np.abs(g).max())
    gmax = np.abs(g).max()
    rng = np.random.default_rng(9)
    h = 1e-3   # |M| >> |dM/d eps| here: smaller steps are dominated by the rounding of M
    for _ in range(10):
        z, y, x = (int(rng.integers(0, n)) for n in w.design_shape)
        c = (z + w.design_lo[2], y + w.design_lo[1], x + w.design_lo[0])
        ep, em = w.eps.astype(np.float64), w.eps.astype(np.float64)
        ep[c] += h
        em[c] -= h
        f = []
        for e in (ep, em):
            we = w.replace(eps=e)
            f.append(s1 * O.forward(we)[1].sum() + s2 * O.forward(_swap_detectors(we))[1].sum())
        fd = (f[0] - f[1]) / (2 * h)
        assert abs(fd - g[z, y, x]) <= 1e-7 * gmax, (c, fd, g[z, y, x])


def test_plane_wave_source_is_transversely_uniform():
    """A uniform sheet source (normally incident plane wave) on a periodic
    grid without CPML drives fields that do not vary across the sheet's plane,
    only along its normal, and only the source's component and the matching
    magnetic component are excited."""
    w = I.coupler_small(n_steps=40).replace(pml_thickness=0, eps=np.ones((26, 28, 36), np.float32))
    st = O.zero_state(w)
    O.run(w, st, periodic=1, pml=0, count=40)
    Ey, Hx = st[1], st[3]
    assert np.abs(Ey).max() > 0
    for f in (Ey, Hx):
        assert np.abs(f - f[:, :1, :1]).max() <= 1e-14 * np.abs(f).max()
    for c in (0, 2, 4, 5):
        assert np.abs(st[c]).max() == 0.0


# ----------------------------------------- the method vs the definition -----

@pytest.mark.parametrize("maker", [I.fd_cube, lambda: I.ragged_box(nx=15, ny=12, nz=11, P=3, n_steps=70)])
def test_time_reversed_gradient_with_exact_samples_equals_stored_history(maker):
    """With unquantised samples at every step (k = 1) the time-reversed
    simulation reproduces the exact discrete gradient (Sec. 1-2): this pins the
    choice of recorded layers and their half-step alignment.  The oracle sets
    every value outside the interior and the recorded layers to NaN first."""
    w = maker()
    L, g = O.gradient(w)
    L2, g2 = O.reverse(w, "none", k=1)
    assert L2 == pytest.approx(L, rel=1e-14)
    assert np.isfinite(g2).all()
    assert np.linalg.norm(g2 - g) <= 1e-11 * np.linalg.norm(g)


def test_subsampled_exact_samples_converge_with_k():
    """Linear interpolation of exact samples: the gradient error shrinks as k
    decreases (Sec. 2, Fig. 1b)."""
    w = I.ragged_box(nx=15, ny=12, nz=11, P=3, n_steps=120)
    _, g = O.gradient(w)
    errs = []
    for k in (8, 4, 2):
        _, gk = O.reverse(w, "none", k=k)
        errs.append(np.linalg.norm(gk - g) / np.linalg.norm(g))
    assert errs[0] > errs[1] > errs[2] > 0


# --------------------------------------------------------- codecs ------------

TORCH_DT = {"bf16": "bfloat16", "f16": "float16", "e4m3": "float8_e4m3fn"}


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
def test_quantizer_matches_library_casts(fmt):
    """RNE onto bf16 / fp16 / e4m3fn equals torch's float32 casts bit for bit
    on float32 inputs spanning normals, subnormals and exact ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    fmax = O.format_max(fmt)
    mags = np.exp(rng.uniform(np.log(fmax) - 40, np.log(fmax), 20000))
    x = (mags * rng.choice([-1, 1], mags.size)).astype(np.float32)
    # exact ties halfway between neighbours of the target format
    t = torch.from_numpy(x).to(getattr(torch, TORCH_DT[fmt])).to(torch.float64).numpy()
    up = np.nextafter(np.abs(t).astype(np.float32), np.float32(np.inf))
    nxt = torch.from_numpy(up).to(getattr(torch, TORCH_DT[fmt])).to(torch.float64).numpy()
    ties = (np.abs(t) + (np.abs(nxt) - np.abs(t)) / 2).astype(np.float32)
    ties = ties[np.abs(ties) <= fmax]
    xs = np.concatenate([x, ties, -ties, np.float32([0.0, fmax, -fmax])])
    ref = torch.from_numpy(xs).to(getattr(torch, TORCH_DT[fmt])).to(torch.float64).numpy()
    got = O.quantize(fmt, xs.astype(np.float64))
    np.testing.assert_array_equal(got, ref)


def test_quantizer_fp32_and_saturation():
    rng = np.random.default_rng(8)
    x = rng.standard_normal(5000) * 10.0 ** rng.uniform(-40, 30, 5000)
    np.testing.assert_array_equal(O.quantize("f32", x), x.astype(np.float32).astype(np.float64))
    assert O.quantize("e4m3", [1e6])[0] == 448.0 and O.quantize("e4m3", [-1e6])[0] == -448.0
    assert O.quantize("f16", [1e9])[0] == 65504.0


# The 8-bit formats of Sec. 4 (Fig. 3), defined by their bit layout: E
# exponent bits, M mantissa bits, exponent bias, and whether the all-ones
# exponent is reserved (IEEE-like: infinities and NaNs) or finite ("fnuz": one
# NaN code 0x80, no negative zero, no infinities).
FP8_LAYOUT = {"e4m3b11fnuz": (4, 3, 11, "fnuz"), "e5m2fnuz": (5, 2, 16, "fnuz"),
              "e4m3fnuz": (4, 3, 8, "fnuz"), "e4m3ieee": (4, 3, 7, "ieee"),
              "e3m4": (3, 4, 3, "ieee")}


def fp8_codes(layout):
    """All finite non-negative values with their codes, by brute force over
    the 128 non-negative bit patterns."""
    E, M, bias, kind = layout
    out = []
    for code in range(128):
        ef, mf = code >> M, code & ((1 << M) - 1)
        if kind == "ieee" and ef == (1 << E) - 1:
            continue                       # infinities and NaNs
        if ef == 0:
            v = mf * 2.0 ** (1 - bias - M)
        else:
            v = (1 + mf / 2.0 ** M) * 2.0 ** (ef - bias)
        out.append((v, code))
    return sorted(out)


def fp8_round_brute(layout, x):
    """Nearest representable value, ties to the even code, saturating at the
    largest finite value."""
    table = fp8_codes(layout)
    vals = np.array([v for v, _ in table])
    codes = np.array([c for _, c in table])
    out = np.empty_like(x)
    for i, xi in enumerate(x):
        a = abs(xi)
        if a >= vals[-1]:
            out[i] = np.copysign(vals[-1], xi)
            continue
        j = np.searchsorted(vals, a)       # vals[j-1] < a <= vals[j]
        if vals[j] == a:
            q = a
        else:
            lo, hi = vals[j - 1], vals[j]
            if a - lo < hi - a:
                q = lo
            elif hi - a < a - lo:
                q = hi
            else:
                q = lo if codes[j - 1] % 2 == 0 else hi
        out[i] = np.copysign(q, xi)
    return out


@pytest.mark.parametrize("fmt", sorted(FP8_LAYOUT))
def test_paper_fp8_formats_against_brute_force(fmt):
    """RNE with saturation onto the paper's 8-bit formats (Sec. 4) equals the
    nearest value among all codes of the bit layout, ties to the even code, on
    random magnitudes over the whole range, exact midpoints and out-of-range
    values; the largest finite value is the layout's."""
    layout = FP8_LAYOUT[fmt]
    table = fp8_codes(layout)
    vals = np.array([v for v, _ in table])
    assert O.format_max(fmt) == vals[-1]
    rng = np.random.default_rng(11)
    mags = np.exp(rng.uniform(np.log(vals[1]) - 3, np.log(vals[-1]) + 2, 4000))
    mids = (vals[:-1] + vals[1:]) / 2
    x = np.concatenate([mags * rng.choice([-1, 1], mags.size), mids, -mids, vals, [0.0]])
    np.testing.assert_array_equal(O.quantize(fmt, x), fp8_round_brute(layout, x))


@pytest.mark.parametrize("fmt,tname", [("e4m3fnuz", "float8_e4m3fnuz"),
                                       ("e5m2fnuz", "float8_e5m2fnuz")])
def test_paper_fp8_formats_match_torch_casts_in_range(fmt, tname):
    """Inside the finite range the fnuz quantisers equal torch's casts of the
    same float32 values (torch does not saturate, so the range is clipped)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    fmax = O.format_max(fmt)
    x = (np.exp(rng.uniform(np.log(fmax) - 25, np.log(fmax), 20000)) *
         rng.choice([-1, 1], 20000)).astype(np.float32)
    ref = torch.from_numpy(x).to(getattr(torch, tname)).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.quantize(fmt, x.astype(np.float64)), ref)


def test_compression_factor_of_the_paper():
    """(32 / bits) x k: float8 with k = 16 gives the paper's 64x."""
    v = golden("paper_numbers.txt")["compression_e4m3b11fnuz_k16"][0]
    assert (32 // 8) * 16 == v


# --------------------------------------------------- interpolation -----------

def test_linear_interpolation_is_exact_on_affine_series():
    t = np.array([-1.0, 2, 6, 10, 14])
    p = 0.25 - 1.5 * t
    q = np.linspace(-1, 14, 61)
    np.testing.assert_allclose(O.interp_series("linear", t, p, q), 0.25 - 1.5 * q, atol=1e-13)


def test_cubic_interpolation_is_exact_on_quadratics_with_uneven_knots():
    t = np.array([-1.0, 3, 7, 11, 15, 19])           # first gap 4, like the zero knot
    t2 = np.array([0.0, 2, 7, 12, 17])               # first gap 2
    for tt in (t, t2):
        p = 0.5 + 0.3 * tt - 0.07 * tt * tt
        q = np.linspace(tt[0], tt[-1], 97)
        np.testing.assert_allclose(O.interp_series("cubic", tt, p, q),
                                   0.5 + 0.3 * q - 0.07 * q * q, atol=1e-12)


def test_cubic_on_uniform_knots_is_catmull_rom():
    t = np.arange(0.0, 40.0, 4.0)
    rng = np.random.default_rng(9)
    p = rng.standard_normal(t.size)
    q = 13.0                      # between t[3] = 12 and t[4] = 16
    s = 0.25
    cr = 0.5 * ((2 * p[4 - 1]) + (-p[2] + p[4]) * s + (2 * p[2] - 5 * p[3] + 4 * p[4] - p[5]) * s * s
                + (-p[2] + 3 * p[3] - 3 * p[4] + p[5]) * s ** 3)
    assert O.interp_series("cubic", t, p, [q])[0] == pytest.approx(cr, rel=1e-13)


@pytest.mark.parametrize("k", [2, 4, 8, 16, 32])
def test_sine_at_136_steps_per_period(k):
    """Fig. 1b analogue: a sine at 136 steps per period sampled every k steps.
    Linear interpolation error is at most h^2 w^2 / 8 (h = k steps) and
    reaches at least 70% of it; cubic is well below linear."""
    w = 2 * np.pi / 136.0
    t = np.arange(0.0, 1000.0, k)
    p = np.sin(w * t)
    q = np.arange(0.0, t[-1] + 1, 1.0)
    lin = np.abs(O.interp_series("linear", t, p, q) - np.sin(w * q)).max()
    bound = (k * w) ** 2 / 8
    assert lin <= bound * (1 + 1e-9)
    if k >= 4:
        assert lin >= 0.7 * bound
    inner = (q > t[1]) & (q < t[-2])
    cub = np.abs(O.interp_series("cubic", t, p, q) - np.sin(w * q))[inner].max()
    # cubic's edge shrinks as sampling approaches Nyquist (4.25 samples/period at k = 32)
    assert cub < (0.2 if k <= 16 else 0.5) * lin


# ------------------------------------------------ block-transform codec ---
# The tape codec beyond the paper (Sec. 4 names JPEG-like tape compression as
# future work): 8 x 8 orthonormal DCT-II, first K coefficients in diagonal
# order, int8 codes with one float32 scale per block.

def _dct_order():
    return [(d - v, v) for d in range(15) for v in range(d + 1) if d - v <= 7 and v <= 7]


def test_bdct_basis_is_the_orthonormal_dct_in_diagonal_order():
    """Rows of the basis are orthonormal (to float32 rounding) and row i is
    the outer product of the 1D DCT-II vectors of (u_i, v_i), the diagonal
    order u + v ascending then v ascending; checked against scipy's DCT."""
    from scipy.fft import dct
    b = O.bdct_basis().astype(np.float64)
    m = b.reshape(64, 64)
    assert np.abs(m @ m.T - np.eye(64)).max() < 2e-7
    d = dct(np.eye(8), type=2, norm="ortho", axis=0)      # d[u, x]
    order = _dct_order()
    assert order[:10] == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2),
                          (0, 3)]
    for i, (u, v) in enumerate(order):
        np.testing.assert_allclose(b[i], np.outer(d[v], d[u]), rtol=0, atol=1e-7)


def test_bdct_coefficients_match_scipy_dctn():
    """All 64 coefficients kept: codes * scale are the 2D DCT-II coefficients
    of the block (scipy.fft.dctn, orthonormal, FP64) to within half a code
    step, the largest code is +-127, and decoding reproduces the block to
    within the accumulated half steps."""
    from scipy.fft import dctn
    rng = np.random.default_rng(4)
    order = _dct_order()
    for trial in range(20):
        x = (rng.standard_normal((8, 8)) * 10.0 ** rng.uniform(-6, 3)).astype(np.float32)
        codes, s = O.bdct_encode(x, 64)
        C = dctn(x.astype(np.float64), type=2, norm="ortho")   # C[v, u]
        ref = np.array([C[v, u] for (u, v) in order])
        got = codes[0].astype(np.float64) * s[0]
        assert np.abs(got - ref).max() <= 0.5 * s[0] * (1 + 1e-5) + 1e-6 * np.abs(ref).max()
        assert np.abs(codes[0]).max() == 127
        assert s[0] == np.float32(np.float32(np.abs(ref).max()) / np.float32(127.0)) or \
            abs(s[0] - np.abs(ref).max() / 127) <= 1e-6 * s[0]
        y = O.bdct_decode(codes, s, 8, 8)
        # each decoded cell carries at most 64 half-step errors, each weighted
        # by |B_i(cell)| <= 1/4
        assert np.abs(y - x).max() <= 64 * 0.25 * 0.5 * s[0] * 1.01


def test_bdct_single_basis_function_and_constant_blocks():
    """A block equal to a * B_j (j < K) codes to +-127 at j and 0 elsewhere;
    a constant block c has the single coefficient 8c (DC) and decodes to c to
    within one code step; an all-zero block has scale 1 and zero codes."""
    b = O.bdct_basis()
    for j in (0, 1, 2, 4, 9):
        for a in (3.5, -0.02):
            codes, s = O.bdct_encode(a * b[j], 10)
            assert codes[0, j] == (127 if a > 0 else -127)
            assert np.abs(np.delete(codes[0], j)).max() == 0
            assert s[0] == pytest.approx(abs(a) / 127, rel=1e-6)
    x = np.full((8, 8), 0.7, np.float32)
    codes, s = O.bdct_encode(x, 6)
    assert codes[0, 0] == 127 and np.abs(codes[0, 1:]).max() == 0
    assert s[0] == pytest.approx(8 * 0.7 / 127, rel=1e-6)
    np.testing.assert_allclose(O.bdct_decode(codes, s, 8, 8), x, rtol=0, atol=s[0] / 8)
    codes, s = O.bdct_encode(np.zeros((8, 8), np.float32), 10)
    assert s[0] == 1.0 and not codes.any()


def test_bdct_ragged_faces_repeat_the_edge():
    """Cells past the face edge repeat the last row / column: an 11 x 5 face
    codes exactly like the 16 x 8 face padded by edge replication, and the
    decoded face is the padded one's decode, cropped."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((5, 11)).astype(np.float32)
    xp = np.pad(x, ((0, 3), (0, 5)), mode="edge")
    for K in (1, 10, 64):
        c, s = O.bdct_encode(x, K)
        cp, sp = O.bdct_encode(xp, K)
        np.testing.assert_array_equal(c, cp)
        np.testing.assert_array_equal(s, sp)
        np.testing.assert_array_equal(O.bdct_decode(c, s, 11, 5),
                                      O.bdct_decode(cp, sp, 16, 8)[:5, :11])


def test_bdct_keeps_smooth_fields_and_drops_fine_detail():
    """Zonal truncation: a long-wavelength field (period 40 cells, as the
    boundary fields of the 20 nm waveguide) keeps its shape when only the
    first K coefficients are kept (FP64 with scipy's DCT: max error 5 % of the
    amplitude at K = 10, < 2 % at K = 21); the codec's error stays within that
    truncation error plus the quantisation bound 0.5 s sum_i |B_i(cell)| per
    cell.  A block of the highest frequency (u = v = 7) alone is removed
    (down to the float32 rounding of the kept coefficients)."""
    from scipy.fft import dctn, idctn
    yy, xx = np.mgrid[0:32, 0:48]
    smooth = np.sin(2 * np.pi * (xx / 40.0 + yy / 55.0)).astype(np.float32)
    errs = {}
    for K in (10, 21):
        keep = np.zeros((8, 8), bool)
        for (u, v) in _dct_order()[:K]:
            keep[v, u] = True
        trunc = np.zeros((32, 48))
        for by in range(4):
            for bx in range(6):
                blk = smooth[8 * by:8 * by + 8, 8 * bx:8 * bx + 8].astype(np.float64)
                C = dctn(blk, type=2, norm="ortho")
                trunc[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] = idctn(np.where(keep, C, 0.0),
                                                                    type=2, norm="ortho")
        terr = np.abs(trunc - smooth)
        errs[K] = terr.max()
        c, s = O.bdct_encode(smooth, K)
        y = O.bdct_decode(c, s, 48, 32)
        wsum = np.abs(O.bdct_basis()[:K]).sum(axis=0)            # [8 y][8 x]
        bound = (0.5 * s.reshape(4, 6)[:, None, :, None] * wsum[None, :, None, :]).reshape(32, 48)
        assert np.all(np.abs(y - smooth) <= terr + bound * 1.001 + 1e-6)
    assert errs[21] < 0.02 < errs[10] < 0.06
    hf = np.tile(5.0 * O.bdct_basis()[63], (4, 6))
    c, s = O.bdct_encode(hf, 10)
    # what is left is the float32 rounding of the kept coefficients (~1e-7)
    assert np.abs(O.bdct_decode(c, s, 48, 32)).max() < 1e-5


def test_bdct_single_coefficient_is_the_block_mean():
    """K = 1 keeps the DC term only: C_0 = 8 mean(block), coded as +-127 with
    s = |C_0| / 127, so every decoded cell is C_0 / 8 = the block mean (to
    float32 rounding); on a ragged plane the mean is over the block with its
    edge cells repeated."""
    rng = np.random.default_rng(11)
    x = rng.standard_normal((13, 21)).astype(np.float32)
    codes, s = O.bdct_encode(x, 1)
    y = O.bdct_decode(codes, s, 21, 13)
    xp = np.pad(x.astype(np.float64), ((0, 3), (0, 3)), mode="edge")
    for bv in range(2):
        for bu in range(3):
            m = xp[8 * bv:8 * bv + 8, 8 * bu:8 * bu + 8].mean()
            blk = y[8 * bv:min(8 * bv + 8, 13), 8 * bu:min(8 * bu + 8, 21)]
            np.testing.assert_allclose(blk, m, rtol=1e-5, atol=1e-6)
            assert abs(codes[bv * 3 + bu, 0]) == 127


# -------------------------------------- per-face scaled tape encoder ---------

MANT = {"e4m3": 3, "f16": 10}
MIN_SUB = {"e4m3": 2.0 ** -9, "f16": 2.0 ** -24}


@pytest.mark.parametrize("fmt", ["e4m3", "f16"])
def test_scaled_face_encoder_properties(fmt):
    """The per-face scale of the reduced bit-width tape (Sec. 2; the scale
    reading of the benchmark's FP8 tape): the face's largest magnitude maps onto the
    format's largest finite value and comes back exactly; every value is
    within half a step of the format at the face's scale; scaling a face by a
    power of two scales its code values by the same power (the scale absorbs
    the exponent, where the unscaled format would flush or saturate); an
    all-zero face keeps scale 1; the scale never drops below 2^-126."""
    rng = np.random.default_rng(31)
    fmax = O.format_max(fmt)
    v = rng.standard_normal(3000) * 10.0 ** rng.uniform(-6, 0, 3000) * 3.7e-2
    q, s = O.encode_face(fmt, v)
    amax = np.abs(v).max()
    assert np.abs(q).max() == pytest.approx(amax, rel=1e-15)
    assert s == pytest.approx(amax / fmax, rel=1e-15)
    bound = amax * 2.0 ** -(MANT[fmt] + 1) + s * MIN_SUB[fmt] / 2
    assert np.all(np.abs(q - v) <= bound * (1 + 1e-12))
    # relative precision of the format for values near the face's maximum
    big = np.abs(v) > amax / 2
    assert np.all(np.abs(q - v)[big] <= np.abs(v[big]) * 2.0 ** -MANT[fmt] * (1 + 1e-12))
    for e in (-100, -20, 30):
        q2, s2 = O.encode_face(fmt, v * 2.0 ** e)
        np.testing.assert_array_equal(q2, q * 2.0 ** e)
        assert s2 == s * 2.0 ** e
    # far below the format's range: the unscaled format loses the face, the
    # scaled one keeps what it kept at the original scale
    qu, su = O.encode_face(fmt, v * 2.0 ** -40, scaled=False)
    assert su == 1.0 and np.count_nonzero(qu) < np.count_nonzero(q) // 10
    z, sz = O.encode_face(fmt, np.zeros(64))
    assert sz == 1.0 and not z.any()
    # a face whose absmax / fmax is below 2^-126 gets the floor scale
    _, sf = O.encode_face(fmt, np.full(8, fmax * 2.0 ** -140))
    assert sf == 2.0 ** -126


def _face_slices(w):
    """Offsets of the six faces in one tape sample: face f = 2 axis + high,
    two tangential components of the interior cross-section each."""
    P = w.pml_thickness
    dims = (w.nx, w.ny, w.nz)
    out, off = [], 0
    for f in range(6):
        a = f // 2
        ua, va = (1 if a == 0 else 0), (1 if a == 2 else 2)
        n = 2 * (dims[ua] - 2 * P) * (dims[va] - 2 * P)
        out.append(slice(off, off + n))
        off += n
    return out


@pytest.mark.parametrize("fmt", ["e4m3", "f16"])
def test_method_tape_is_scaled_per_face_and_sample(fmt):
    """The method's recorded tape with a scaled format equals, face by face and
    sample by sample, the exact samples divided by that face's own scale
    max(absmax / format_max, 2^-126) (1 for an all-zero face), quantised and
    multiplied back.  The faces of one sample have very different magnitudes
    here, so a scale shared across a sample, a missing floor or a multiply in
    place of the divide would change the codes."""
    w = I.ragged_box(nx=16, ny=13, nz=12, P=3, n_steps=60)
    _, _, raw = O.reverse(w, "none", k=1, want_tape=True)
    _, _, tq = O.reverse(w, fmt, scaled=True, k=1, want_tape=True)
    fmax = O.format_max(fmt)
    faces = _face_slices(w)
    spread, zero_faces = 0.0, 0
    for j in range(raw.shape[0]):
        amaxes = []
        for sl in faces:
            r = raw[j, sl]
            amax = np.abs(r).max()
            amaxes.append(amax)
            s = max(amax / fmax, 2.0 ** -126) if amax > 0 else 1.0
            zero_faces += amax == 0
            np.testing.assert_array_equal(tq[j, sl], O.quantize(fmt, r / s) * s)
        nz = [a for a in amaxes if a > 0]
        if len(nz) > 1:
            spread = max(spread, max(nz) / min(nz))
    assert spread > 100 and zero_faces > 0


# ------------------------------------------ two detectors in the method -----

def test_two_detector_method_with_exact_samples_equals_stored_history():
    """Both detectors seeded in the same time-reversed run (the transmission
    ratio of Sec. 4): with exact samples at every step it reproduces the
    stored-history gradient of s L + s2 M, and L, M themselves."""
    w = I.coupler_small(n_steps=70)
    s1, s2 = 0.7, -1.3
    L, M, g = O.gradient2(w, s1, s2)
    L2, M2, g2 = O.reverse2(w, "none", k=1, seed=s1, seed2=s2)
    assert L2 == pytest.approx(L, rel=1e-14) and M2 == pytest.approx(M, rel=1e-14)
    assert np.isfinite(g2).all()
    assert np.linalg.norm(g2 - g) <= 1e-11 * np.linalg.norm(g)


def test_two_detector_method_is_linear_in_the_seeds_for_a_compressed_tape():
    """The tape does not depend on the seeds and the adjoint is linear: the
    method's gradient of s L + s2 M with a compressed tape equals s times its
    gradient of L plus s2 times its gradient of M (the second detector made
    the only one) from the same tape."""
    w = I.coupler_small(n_steps=70)
    s1, s2 = 0.7, -1.3
    _, _, g = O.reverse2(w, "e4m3", scaled=True, k=2, interp="cubic", seed=s1, seed2=s2)
    _, g1 = O.reverse(w, "e4m3", scaled=True, k=2, interp="cubic")
    _, gm = O.reverse(_swap_detectors(w), "e4m3", scaled=True, k=2, interp="cubic")
    np.testing.assert_allclose(g, s1 * g1 + s2 * gm, rtol=0, atol=1e-12 * np.abs(g).max())
    assert np.abs(gm).max() > 1e-3 * np.abs(g1).max()
