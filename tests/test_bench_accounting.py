"""The benchmark's algorithmic-byte accounting (the numerator of every
roofline fraction it reports), checked on the host.

Per cell and launch (FP32 = 4 B): the forward H half-step reads E and Ht and
writes Ht (36 B), the forward E half-step reads Ht, E and cb and writes E
(40 B); the reverse E phase moves 76 B in the interior (primal and adjoint)
and 40 B elsewhere, plus 16 B of FP64 accumulator in the design box; the
reverse H phase 72 B / 36 B; every CPML slab axis a cell lies in adds two
auxiliaries read and written (16 B).  A tape sample holds the two tangential
components on each of the six interface faces.
"""
import itertools

import numpy as np
import pytest

import bench
from paper_2603_24027_gb300 import inputs as I


def brute_force_bytes(w):
    """Per-cell loop over the grid with the rules above."""
    P = w.pml_thickness
    lo = [s.start for s in w.design_slice()][::-1]   # (x, y, z)
    hi = [s.stop for s in w.design_slice()][::-1]
    tot = dict(fwd_h=0, fwd_e=0, rev_e=0, rev_h=0)
    for z, y, x in itertools.product(range(w.nz), range(w.ny), range(w.nx)):
        slabs = sum(int(c < P or c >= n - P) for c, n in ((x, w.nx), (y, w.ny), (z, w.nz)))
        inside = slabs == 0
        design = all(lo[a] <= c < hi[a] for a, c in enumerate((x, y, z)))
        tot["fwd_h"] += 36 + 16 * slabs
        tot["fwd_e"] += 40 + 16 * slabs
        tot["rev_e"] += (76 if inside else 40) + 16 * design + 16 * slabs
        tot["rev_h"] += (72 if inside else 36) + 16 * slabs
    return tot


def test_counts_match_a_per_cell_loop():
    w = I.ragged_box()
    ab = bench.algorithmic_bytes(w)
    for k, v in brute_force_bytes(w).items():
        assert ab[k] == v, k


def test_waveguide_launch_bytes():
    """200 x 200 x 100 cells, 12-cell CPML, 100 x 100 x 11 design box, by hand:
    interior 176 x 176 x 76 = 2 354 176 cells; slab-axis memberships
    2 * 12 * (200*100 + 200*100 + 200*200) = 1 920 000."""
    w = I.waveguide()
    assert w.shape == (100, 200, 200) and w.pml_thickness == 12
    ab = bench.algorithmic_bytes(w)
    n, ni, nd, sa = 4_000_000, 2_354_176, 110_000, 1_920_000
    assert ab["fwd_h"] == 36 * n + 16 * sa == 174_720_000
    assert ab["fwd_e"] == 40 * n + 16 * sa == 190_720_000
    assert ab["rev_e"] == 76 * ni + 40 * (n - ni) + 16 * nd + 16 * sa == 277_230_336
    assert ab["rev_h"] == 72 * ni + 36 * (n - ni) + 16 * sa == 259_470_336


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
