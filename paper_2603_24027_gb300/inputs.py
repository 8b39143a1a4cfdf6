"""Seeded synthetic workloads shared by the CUDA path, its tests and the oracle.

This module only builds inputs: grid sizes, the Courant time step of Eq. 1,
material maps eps_r, and the source / detector / design-box geometry.  It holds
none of the method's arithmetic (no curl, CPML profile, waveform, codec or
interpolation); each side of the parity check computes those itself.

Workload shapes follow the paper's setting (Sec. 2-3): Si (eps 12.25) and
SiO2 (eps 2.085) at a 220 nm layer, a 60 nm Gaussian smoothing of the design
variables, 1550 nm light at ~136 steps per period for dx = 20 nm, and a
Poynting-flux detector behind the device.  The paper's grating-coupler
geometry is not reproduced; a straight Si strip through a random smoothed
design box stands in for it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C0 = 299792458.0          # speed of light in vacuum, m/s (Eq. 1)
COURANT = 0.99            # Courant factor C of Eq. 1
EPS_SIO2 = 2.085
EPS_SI = 12.25

SRC_NONE, SRC_POINT, SRC_PLANE_GAUSS, SRC_PLANE_UNIFORM = 0, 1, 2, 3
OBJ_E2_PLANE, OBJ_POYNTING_PLANE = 1, 2


def cfl_dt(dx: float, courant: float = COURANT) -> float:
    """Time step of Eq. 1: dt = C dx / (c sqrt(3))."""
    return courant * dx / (C0 * math.sqrt(3.0))


@dataclasses.dataclass
class Workload:
    """One FDTD gradient problem.

    eps is float32 [nz][ny][nx] (x fastest).  Boxes are half-open cell ranges.
    Detector/source plane coordinates (u, v) are the two axes other than the
    plane's normal, in increasing axis order: x-normal -> (y, z),
    y-normal -> (x, z), z-normal -> (x, y).
    """
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    n_steps: int
    pml_thickness: int
    eps: np.ndarray
    design_lo: tuple
    design_hi: tuple
    src_kind: int = SRC_POINT
    src_component: int = 2
    src_pos: tuple = (0, 0, 0)
    src_axis: int = 0
    src_sigma_uv: tuple = (1.0, 1.0)
    lambda0: float = 1550e-9
    rel_bandwidth: float = 0.3
    t0_over_tau: float = 3.0
    amplitude: float = 1.0
    det_kind: int = OBJ_E2_PLANE
    det_axis: int = 2
    det_index: int = 0
    det_lo: tuple = (0, 0)
    det_hi: tuple = (0, 0)
    # optional second detector (kind 0 = none): its objective M sits beside L
    det2_kind: int = 0
    det2_axis: int = 2
    det2_index: int = 0
    det2_lo: tuple = (0, 0)
    det2_hi: tuple = (0, 0)
    pml_order: int = 3
    pml_sigma_factor: float = 0.8
    pml_kappa_max: float = 1.0
    pml_alpha_factor: float = 0.05

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def design_shape(self):
        lo, hi = self.design_lo, self.design_hi
        return (hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])

    def design_slice(self):
        lo, hi = self.design_lo, self.design_hi
        return (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _uniform_f32(rng, shape, lo, hi):
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def _gaussian_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(4.0 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _smooth_axis(a: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    r = (len(w) - 1) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad, mode="symmetric")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for t, wt in enumerate(w):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(t, t + n)
        out += wt * ap[tuple(sl)]
    return out


def smoothed_design(rng, shape, sigma_cells: float) -> np.ndarray:
    """eps = 2.085 + 10.165 * sigmoid(G_sigma * N(0,1)), the Gaussian-filtered
    density of Sec. 3 (60 nm filter).  The filtered noise is rescaled to unit
    standard deviation before the sigmoid so the box spans SiO2..Si rather than
    collapsing to the mid value."""
    noise = rng.standard_normal(shape)
    w = _gaussian_kernel(sigma_cells)
    s = noise
    for ax in range(3):
        s = _smooth_axis(s, w, ax)
    s = (s - s.mean()) / max(s.std(), 1e-30)
    rho = 1.0 / (1.0 + np.exp(-s))
    return (EPS_SIO2 + (EPS_SI - EPS_SIO2) * rho).astype(np.float32)


# ---------------------------------------------------------------- configs ----

def small_dipole(seed: int = 0) -> Workload:
    """48^3 cells at 25 nm, 8-cell CPML, 400 steps, Ez point dipole, |E|^2 on a
    32x32 plane, random eps ~ U[1, 12.25] in the central 16^3 box, vacuum
    elsewhere."""
    n, P = 48, 8
    dx = 25e-9
    eps = np.ones((n, n, n), np.float32)
    lo, hi = (16, 16, 16), (32, 32, 32)
    rng = _rng(seed)
    eps[16:32, 16:32, 16:32] = _uniform_f32(rng, (16, 16, 16), 1.0, EPS_SI)
    return Workload(
        name="dipole48", nx=n, ny=n, nz=n, dx=dx, dt=cfl_dt(dx), n_steps=400,
        pml_thickness=P, eps=eps, design_lo=lo, design_hi=hi,
        src_kind=SRC_POINT, src_component=2, src_pos=(24, 24, 12),
        t0_over_tau=2.0,
        det_kind=OBJ_E2_PLANE, det_axis=2, det_index=36, det_lo=(8, 8), det_hi=(40, 40))


def waveguide(nx=200, ny=200, nz=100, P=12, n_steps=2000, design_xy=100,
              dx=20e-9, seed: int = 0, sigma_cells: float = 3.0) -> Workload:
    """Si strip (eps 12.25, 25 x 11 cells) along x in SiO2 (eps 2.085, PML
    included), a design box design_xy x design_xy x 11 centred on the strip
    with smoothed random eps, a Gaussian-profile Ey plane source at x = P+4
    and a Poynting-flux detector on x = nx-P-4 over the interior (y, z)."""
    eps = np.full((nz, ny, nx), EPS_SIO2, np.float32)
    yc, zc = ny // 2, nz // 2
    strip_w, strip_h = 25, 11
    y0, z0 = yc - strip_w // 2, zc - strip_h // 2
    eps[z0:z0 + strip_h, y0:y0 + strip_w, :] = EPS_SI
    dlo = (nx // 2 - design_xy // 2, ny // 2 - design_xy // 2, z0)
    dhi = (dlo[0] + design_xy, dlo[1] + design_xy, z0 + strip_h)
    rng = _rng(seed)
    box = (dhi[2] - dlo[2], dhi[1] - dlo[1], dhi[0] - dlo[0])
    eps[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = smoothed_design(rng, box, sigma_cells)
    return Workload(
        name=f"waveguide{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=cfl_dt(dx),
        n_steps=n_steps, pml_thickness=P, eps=eps, design_lo=dlo, design_hi=dhi,
        src_kind=SRC_PLANE_GAUSS, src_component=1, src_axis=0,
        src_pos=(P + 4, yc, zc), src_sigma_uv=(8.0, 4.0), t0_over_tau=3.0,
        det_kind=OBJ_POYNTING_PLANE, det_axis=0, det_index=nx - P - 4,
        det_lo=(P, P), det_hi=(ny - P, nz - P))


def waveguide_mid(seed: int = 0) -> Workload:
    """200 x 200 x 100 cells at 20 nm, 12-cell CPML, 2000 steps, 100x100x11 design."""
    return waveguide(seed=seed)


def waveguide_sweep(seed: int = 0, n_steps: int = 2000) -> Workload:
    """The waveguide device at 100 x 100 x 50 (50 x 50 x 11 design), the size
    the FP64 oracle finishes in about a minute."""
    return waveguide(nx=100, ny=100, nz=50, P=12, n_steps=n_steps, design_xy=50, seed=seed)


def waveguide_large(seed: int = 0, n_steps: int = 10000) -> Workload:
    """600 x 600 x 300 cells at 10 nm (22 cells = 220 nm), 16-cell CPML,
    400 x 400 x 22 design smoothed at 6 cells (60 nm)."""
    nx, ny, nz, P = 600, 600, 300, 16
    w = waveguide(nx=nx, ny=ny, nz=nz, P=P, n_steps=n_steps, design_xy=400,
                  dx=10e-9, seed=seed, sigma_cells=6.0)
    # 50 x 22 strip for the finer grid.
    eps = np.full((nz, ny, nx), EPS_SIO2, np.float32)
    yc, zc = ny // 2, nz // 2
    y0, z0 = yc - 25, zc - 11
    eps[z0:z0 + 22, y0:y0 + 50, :] = EPS_SI
    dlo = (100, 100, z0)
    dhi = (500, 500, z0 + 22)
    eps[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]] = smoothed_design(
        _rng(seed), (22, 400, 400), 6.0)
    return w.replace(name="waveguide600x600x300", eps=eps, design_lo=dlo, design_hi=dhi,
                     src_pos=(P + 4, yc, zc), src_sigma_uv=(16.0, 8.0))


def batched_cubes(n_sims: int = 64, seed: int = 0, sizes=(32, 48, 64, 96, 128),
                  steps=(600, 1500)) -> list:
    """Independent cubic vacuum grids n^3 (n drawn from `sizes`), 8-cell CPML,
    25 nm cells, random eps ~ U[1, 12.25] in the central cube of half-width n/4,
    Ez point source at (n/2, n/2, P+4), |E|^2 plane at z = n-P-4."""
    rng = _rng(seed)
    out = []
    P = 8
    dx = 25e-9
    for s in range(n_sims):
        n = int(rng.choice(sizes))
        ns = int(rng.integers(steps[0], steps[1] + 1))
        eps = np.ones((n, n, n), np.float32)
        lo = (n // 4,) * 3
        hi = (n // 4 + n // 2,) * 3
        eps[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = _uniform_f32(rng, (n // 2,) * 3, 1.0, EPS_SI)
        out.append(Workload(
            name=f"cube{n}_{s}", nx=n, ny=n, nz=n, dx=dx, dt=cfl_dt(dx), n_steps=ns,
            pml_thickness=P, eps=eps, design_lo=lo, design_hi=hi,
            src_kind=SRC_POINT, src_component=2, src_pos=(n // 2, n // 2, P + 4),
            t0_over_tau=2.0, det_kind=OBJ_E2_PLANE, det_axis=2, det_index=n - P - 4,
            det_lo=(P, P), det_hi=(n - P, n - P)))
    return out


def ragged_box(nx=70, ny=21, nz=19, P=6, n_steps=80, seed: int = 0,
               det_kind=OBJ_POYNTING_PLANE, src_kind=SRC_PLANE_GAUSS) -> Workload:
    """Odd-sized grid that spans several 32 x 8 tiles with ragged tails, random
    eps ~ U[1, 12.25] over the whole interior box (design = interior)."""
    rng = _rng(seed)
    eps = np.ones((nz, ny, nx), np.float32)
    lo, hi = (P, P, P), (nx - P, ny - P, nz - P)
    eps[P:nz - P, P:ny - P, P:nx - P] = _uniform_f32(rng, (nz - 2 * P, ny - 2 * P, nx - 2 * P), 1.0, EPS_SI)
    dx = 25e-9
    kw = dict(det_kind=det_kind)
    if det_kind == OBJ_POYNTING_PLANE:
        kw.update(det_axis=0, det_index=min(nx - P - 2, P + 11), det_lo=(P, P),
                  det_hi=(ny - P, nz - P))
    else:
        kw.update(det_axis=2, det_index=min(nz - P - 2, P + 9), det_lo=(P + 1, P + 1),
                  det_hi=(nx - P - 1, ny - P - 1))
    if src_kind == SRC_PLANE_GAUSS:
        kw.update(src_kind=src_kind, src_component=1, src_axis=0, src_pos=(P + 1, ny // 2, nz // 2),
                  src_sigma_uv=(2.5, 2.0))
    else:
        kw.update(src_kind=src_kind, src_component=2, src_pos=(nx // 3, ny // 2, P + 1))
    # broadband pulse (rel. bandwidth 1, ~41-step envelope) so that it reaches
    # the detector within a short run
    return Workload(name=f"ragged{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=cfl_dt(dx),
                    n_steps=n_steps, pml_thickness=P, eps=eps, design_lo=lo, design_hi=hi,
                    rel_bandwidth=1.0, t0_over_tau=1.2, **kw)


def fd_cube(seed: int = 0, n_steps: int = 60) -> Workload:
    """8^3 cells, 2-cell CPML, 4^3 interior = design box, for brute-force
    central finite differences of the gradient."""
    n, P = 8, 2
    rng = _rng(seed)
    eps = np.ones((n, n, n), np.float32)
    eps[P:n - P, P:n - P, P:n - P] = _uniform_f32(rng, (4, 4, 4), 1.0, EPS_SI)
    dx = 25e-9
    return Workload(name="fd8", nx=n, ny=n, nz=n, dx=dx, dt=cfl_dt(dx), n_steps=n_steps,
                    pml_thickness=P, eps=eps, design_lo=(P,) * 3, design_hi=(n - P,) * 3,
                    src_kind=SRC_POINT, src_component=2, src_pos=(3, 3, 3), t0_over_tau=0.5,
                    det_kind=OBJ_E2_PLANE, det_axis=2, det_index=4, det_lo=(2, 2), det_hi=(6, 6))


def coupler(nx: int = 150, ny: int = 110, nz: int = 70, P: int = 12, n_steps: int = 2000,
            dx: float = 20e-9, dev: int = 80, wg_w: int = 20, layer: int = 11,
            src_dz: int = 14, det_dz: int = 8, rho=None, seed: int = 0) -> Workload:
    """Grating-coupler analogue of the paper's optimisation benchmark (Sec. 4):
    a dev x dev x layer design region (1.6 um x 1.6 um x 220 nm at 20 nm) in
    SiO2 cladding feeding a wg_w-wide Si waveguide that runs along +x into the
    CPML; a normally incident Ey plane wave from a z-plane src_dz cells above
    the layer.  Objective L: Poynting flux along +x through the waveguide
    cross-section near the far end; second detector M: Poynting flux along +z
    through the plane det_dz cells above the device (the incident side).  The
    transmission is -L/M (the incident flux points down).  rho (dev x dev in
    [0, 1], or None for a seeded smooth random start) maps to eps = SiO2 +
    (Si - SiO2) rho, extruded over the layer."""
    eps = np.full((nz, ny, nx), EPS_SIO2, np.float32)
    z0 = nz // 2 - layer // 2
    z1 = z0 + layer
    x0 = P + 6
    x1 = x0 + dev
    y0 = (ny - dev) // 2
    y1 = y0 + dev
    yw0 = (ny - wg_w) // 2
    yw1 = yw0 + wg_w
    eps[z0:z1, yw0:yw1, x1:] = EPS_SI
    if rho is None:
        rng = _rng(seed)
        noise = rng.standard_normal((dev, dev))
        k = _gaussian_kernel(3.0)
        c = (len(k) - 1) // 2

        def conv(r):   # zero-padded, centred, also for rows shorter than k
            return np.convolve(r, k, mode="full")[c:c + len(r)]
        sm = np.apply_along_axis(conv, 0, noise)
        sm = np.apply_along_axis(conv, 1, sm)
        sm = (sm - sm.mean()) / (sm.std() + 1e-12)
        rho = 1.0 / (1.0 + np.exp(-sm))
    rho = np.asarray(rho, np.float64)
    eps[z0:z1, y0:y1, x0:x1] = (EPS_SIO2 + (EPS_SI - EPS_SIO2) * rho)[None].astype(np.float32)
    m = 6 if wg_w >= 12 else 2
    return Workload(
        name=f"coupler{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=cfl_dt(dx),
        n_steps=n_steps, pml_thickness=P, eps=eps, design_lo=(x0, y0, z0),
        design_hi=(x1, y1, z1), src_kind=SRC_PLANE_UNIFORM, src_component=1, src_axis=2,
        src_pos=(nx // 2, ny // 2, z1 + src_dz), t0_over_tau=3.0,
        det_kind=OBJ_POYNTING_PLANE, det_axis=0, det_index=nx - P - 4,
        det_lo=(max(P, yw0 - m), max(P, z0 - m)), det_hi=(min(ny - P, yw1 + m), min(nz - P, z1 + m)),
        det2_kind=OBJ_POYNTING_PLANE, det2_axis=2, det2_index=z1 + det_dz,
        det2_lo=(x0, y0), det2_hi=(x1, y1))


def coupler_small(n_steps: int = 90, seed: int = 0) -> Workload:
    """The coupler layout at oracle-test size: 36 x 28 x 26 cells, 5-cell CPML."""
    return coupler(nx=36, ny=28, nz=26, P=5, n_steps=n_steps, dx=25e-9, dev=10, wg_w=4,
                   layer=3, src_dz=4, det_dz=2, seed=seed)


def random_state(shape, seed: int, n_arrays: int, scale: float = 1.0) -> np.ndarray:
    """Seeded float64 state block [n_arrays][nz][ny][nx] for operator tests."""
    return _rng(seed).standard_normal((n_arrays,) + tuple(shape)) * scale


CONFIGS = {
    "coupler150": coupler,
    "dipole48": small_dipole,
    "waveguide200": waveguide_mid,
    "waveguide100": waveguide_sweep,
    "waveguide600": waveguide_large,
}
