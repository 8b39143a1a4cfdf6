"""The benchmark's algorithmic-byte accounting (the numerator of every
roofline fraction it reports), checked on the host.

Per cell and time step (FP32 = 4 B), the two phases of the gradient:
  forward: read E, Ht, cb and write E, Ht (52 B), and every CPML axis the
    cell lies in adds its four auxiliaries read and written (32 B);
  reverse: an interior cell reads E, Ht, lamE, lamH, cb and writes the four
    fields (100 B); a cell in the CPML runs the adjoint only (52 B); every
    CPML axis adds 32 B of adjoint auxiliaries; a design cell adds its FP64
    accumulator read and written (16 B).
The tape adds one sample's codes every k-th forward step and, per reverse
step, the codes of the samples the interpolation reads plus the restored
FP32 value of every face value.  A tape sample holds the two tangential
components on each of the six interface faces.

The per-kernel breakdown (what each split half-step launch moves itself) is
checked by the same per-cell loop.
"""
import itertools

import numpy as np
import pytest

import bench
from paper_2603_24027_gb300 import inputs as I


def per_cell(w):
    """Per-cell loop over the grid with the rules above (tape excluded)."""
    P = w.pml_thickness
    lo = [s.start for s in w.design_slice()][::-1]   # (x, y, z)
    hi = [s.stop for s in w.design_slice()][::-1]
    tot = dict(forward=0, reverse=0, fwd_h=0, fwd_e=0, rev_e=0, rev_h=0)
    for z, y, x in itertools.product(range(w.nz), range(w.ny), range(w.nx)):
        slabs = sum(int(c < P or c >= n - P) for c, n in ((x, w.nx), (y, w.ny), (z, w.nz)))
        inside = slabs == 0
        design = all(lo[a] <= c < hi[a] for a, c in enumerate((x, y, z)))
        tot["forward"] += 52 + 32 * slabs
        tot["reverse"] += (100 if inside else 52) + 32 * slabs + 16 * design
        tot["fwd_h"] += 36 + 16 * slabs
        tot["fwd_e"] += 40 + 16 * slabs
        tot["rev_e"] += (76 if inside else 40) + 16 * design + 16 * slabs
        tot["rev_h"] += (72 if inside else 36) + 16 * slabs
    return tot


@pytest.mark.parametrize("tape,cbytes,terms", [("f32:1:linear", 4, 2), ("e4m3:8:linear", 1, 2),
                                               ("bf16:4:cubic", 2, 4)])
def test_phase_bytes_match_a_per_cell_loop(tape, cbytes, terms):
    w = I.ragged_box()
    pb = bench.phase_bytes(w, tape)
    ref = per_cell(w)
    tv = bench.tape_values(w)
    k = int(tape.split(":")[1])
    assert pb["forward"] == pytest.approx(ref["forward"] + tv * (4 + cbytes) / k, rel=1e-15)
    assert pb["reverse"] == pytest.approx(ref["reverse"] + tv * (terms * cbytes + 4), rel=1e-15)


def test_kernel_breakdown_matches_a_per_cell_loop():
    w = I.ragged_box()
    kb = bench.kernel_bytes(w)
    ref = per_cell(w)
    for k in ("fwd_h", "fwd_e", "rev_e", "rev_h"):
        assert kb[k] == ref[k], k
    # the split reverse moves more than the reverse phase's algorithmic bytes
    assert kb["rev_e"] + kb["rev_h"] > bench.phase_bytes(w, "f32:1:linear")["reverse"]


def test_waveguide_phase_bytes_by_hand():
    """200 x 200 x 100 cells, 12-cell CPML, 100 x 100 x 11 design box, by hand:
    interior 176 x 176 x 76 = 2 354 176 cells; slab-axis memberships
    2 * 12 * (200*100 + 200*100 + 200*200) = 1 920 000; a tape sample holds
    4 (176*76 + 176*76 + 176*176) = 230 912 values."""
    w = I.waveguide()
    assert w.shape == (100, 200, 200) and w.pml_thickness == 12
    n, ni, nd, sa, tv = 4_000_000, 2_354_176, 110_000, 1_920_000, 230_912
    assert bench.tape_values(w) == tv
    pb = bench.phase_bytes(w, "e4m3:8:linear")
    assert pb["forward"] == pytest.approx(52 * n + 32 * sa + tv * 5 / 8)
    assert pb["reverse"] == pytest.approx(100 * ni + 52 * (n - ni) + 32 * sa + 16 * nd + tv * 6)
    assert 52 * n + 32 * sa == 269_440_000
    assert 100 * ni + 52 * (n - ni) + 32 * sa + 16 * nd == 384_200_448


def test_large_waveguide_cell_classes():
    """600 x 600 x 300 cells, 16-cell CPML: interior 568 x 568 x 268, slab-axis
    memberships 2 * 16 * (600*300 + 600*300 + 600*600) = 23 040 000, design
    box 400 x 400 x 22."""
    w = I.waveguide_large(n_steps=10)
    c = bench.cell_classes(w)
    assert c["cells"] == 108_000_000
    assert c["interior"] == 568 * 568 * 268
    assert c["slab_axes"] == 23_040_000
    assert c["design"] == 400 * 400 * 22


@pytest.mark.parametrize("make", [I.ragged_box, I.small_dipole, I.waveguide])
def test_tape_sample_values(make):
    """Two tangential components on every interface face, each face spanning
    the interior cross-section."""
    w = make()
    P = w.pml_thickness
    mask = np.zeros((3, w.nz, w.ny, w.nx), bool)   # face planes, one per normal axis
    mask[0, P:w.nz - P, P:w.ny - P, [P - 1, w.nx - P]] = True
    mask[1, P:w.nz - P, [P - 1, w.ny - P], P:w.nx - P] = True
    mask[2, [P - 1, w.nz - P], P:w.ny - P, P:w.nx - P] = True
    assert bench.tape_values(w) == 2 * int(mask.sum())


def test_default_line_is_the_large_waveguide_with_a_16x_tape():
    """The default bench line runs the largest single-GPU workload (600 x 600
    x 300, 10 000 steps) with an FP8 tape every 8th step: 32x smaller than
    the FP32 tape of every step (per-face scales included)."""
    a = bench.parse([])
    assert a.workload == "waveguide600" and a.tape == "e4m3:8:linear"
    w = bench.workload(0, name=a.workload)
    assert (w.nx, w.ny, w.nz, w.n_steps) == (600, 600, 300, 10000)
    tv = bench.tape_values(w)
    J = -(-w.n_steps // 8)
    f32 = w.n_steps * tv * 4
    e4m3 = J * (tv * 1 + 6 * 4)
    assert f32 / e4m3 >= 16
