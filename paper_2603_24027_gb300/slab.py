"""Slab decomposition of one gradient over z: one rank per GPU.

The paper motivates its tape compression by the memory of large 3D
simulations (Sec. 1, Sec. 4); a grid too large for one GPU is cut into z
slabs, one per rank.  Every update of the Yee scheme reads neighbours one
cell away, and across a cut only the z-differences of the curls reach the
other side.  Those read the two tangential components (x, y) of the other
field one plane away, so per half-step a rank needs exactly one plane of two
components from one neighbour:

  half-step                     reads across the cut         ghost plane
  forward H (curl E, +z diff.)  E_x, E_y at z1               above (hi)
  forward E (curl Ht, -z diff.) Ht_x, Ht_y at z0 - 1         below (lo)
  inverse E (reverse, r2)       Ht_x, Ht_y at z0 - 1         lo
  inverse H (reverse, r6)       E_x, E_y at z1               hi
  adjoint of the E half-step    lamE_x, lamE_y at z1 (and cb) hi
  adjoint of the H half-step    lamHt_x, lamHt_y at z0 - 1   lo

The adjoint rows hold because the transpose of a forward difference is a
backward one and vice versa.  The z-CPML slabs are never cut: rank 0 owns
[0, P] and the last rank [N_z - P - 1, N_z), so every ghost plane lies in
the z-lossless region, where the z auxiliaries have zero coefficients and
are never exchanged (the x / y auxiliaries of a cell are read only by that
cell).  Only the ranks holding a part of an interface face record and
restore it: each rank its z rows of the four x / y faces, rank 0 the low
z face and the last rank the high one.  A per-face tape scale is the
maximum over the ranks of their shares' absmax (one reduction of six values
per sample), so the partitioned tape equals the single-rank one value for
value.  The objective is one scalar sum over ranks, and the gradient rows
of the design box are disjoint.

This module holds the host side: the cost-balanced partition, each rank's
ownership (planes, tape rows, design rows, detector rows), the ordered
schedule of half-steps and exchanges of one forward and one reverse step,
and the exchange itself over torch.distributed point-to-point messages
(NCCL for CUDA tensors, gloo for CPU tensors).  The per-rank device engine
(the staged kernels on a slab with two ghost planes and a z-CPML on the
owned global faces only) is not part of the library, which drives one GPU
per process and no device-side halo path.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

# Bytes per cell and time step (FP32 = 4 B) of the two phases: forward 52,
# reverse 100 in the interior and 52 in the CPML, 32 more per CPML axis the
# cell lies in (forward and reverse each).
_FWD, _REV_IN, _REV_PML, _PER_AXIS = 52, 100, 52, 32


def plane_cost(nx: int, ny: int, nz: int, P: int) -> np.ndarray:
    """Bytes moved per time step (forward + reverse) by each z plane."""
    full = nx * ny
    inner = max(nx - 2 * P, 0) * max(ny - 2 * P, 0)
    xy_axes = 2 * P * ny + 2 * P * nx          # x-slab cells + y-slab cells of a plane
    cost = np.zeros(nz)
    for z in range(nz):
        zpml = z < P or z >= nz - P
        interior = 0 if zpml else inner
        axes = xy_axes + (full if zpml else 0)
        cost[z] = (_FWD * full + _REV_IN * interior + _REV_PML * (full - interior)
                   + 2 * _PER_AXIS * axes)
    return cost


@dataclasses.dataclass(frozen=True)
class Slab:
    """The z planes [z0, z1) of an nx x ny x nz grid with a P-cell CPML,
    owned by `rank` of `world`."""
    rank: int
    world: int
    nx: int
    ny: int
    nz: int
    P: int
    z0: int
    z1: int

    @property
    def has_lo(self) -> bool:
        """A rank below: the ghost plane z0 - 1 exists."""
        return self.rank > 0

    @property
    def has_hi(self) -> bool:
        """A rank above: the ghost plane z1 exists."""
        return self.rank < self.world - 1

    @property
    def z_lo(self) -> int:
        """First stored plane (the low ghost plane if there is one)."""
        return self.z0 - int(self.has_lo)

    @property
    def z_hi(self) -> int:
        """End of the stored planes (one past the high ghost plane if any)."""
        return self.z1 + int(self.has_hi)

    @property
    def cpml_lo(self) -> bool:
        """This rank runs the low z-CPML slab [0, P)."""
        return self.rank == 0

    @property
    def cpml_hi(self) -> bool:
        """This rank runs the high z-CPML slab [nz - P, nz)."""
        return self.rank == self.world - 1

    def rows(self, lo: int, hi: int):
        """The owned part [a, b) of the global z range [lo, hi) (a == b: none)."""
        a, b = max(lo, self.z0), min(hi, self.z1)
        return (a, b) if a < b else (a, a)

    def face_rows(self, f: int) -> Optional[tuple]:
        """This rank's rows [v0, v1) of tape face f (f = 2 * axis + high), in
        the face's own v coordinate, or None if it holds none of it.  x and y
        faces span z over the interior [P, nz - P) (v = z - P); the low z face
        (layer P - 1) belongs to rank 0, the high one (layer nz - P) to the
        last rank, whole (v = y - P)."""
        axis, high = divmod(f, 2)
        if axis == 2:
            layer = self.nz - self.P if high else self.P - 1
            return (0, self.ny - 2 * self.P) if self.z0 <= layer < self.z1 else None
        a, b = self.rows(self.P, self.nz - self.P)
        return (a - self.P, b - self.P) if a < b else None


def partition(nx: int, ny: int, nz: int, P: int, world: int) -> list:
    """Cut the z axis into `world` slabs of about equal cost (bytes per time
    step, forward + reverse).  The cuts lie in [P + 1, nz - P - 1], so the
    z-CPML slabs stay whole and every ghost plane is z-lossless; each rank
    owns at least one plane.  Raises ValueError if the grid is too thin."""
    if world < 1:
        raise ValueError("world must be >= 1")
    lo_cut, hi_cut = P + 1, nz - P - 1
    if world > 1 and hi_cut - lo_cut + 1 < world - 1:
        raise ValueError(f"{nz} planes with a {P}-cell CPML cannot be cut into {world} slabs")
    cum = np.concatenate([[0.0], np.cumsum(plane_cost(nx, ny, nz, P))])
    cuts = []
    prev = 0
    for r in range(1, world):
        target = cum[-1] * r / world
        b = int(np.searchsorted(cum, target))          # first plane boundary at or past target
        if b > 0 and target - cum[b - 1] < cum[b] - target:
            b -= 1                                      # nearer boundary
        b = min(max(b, lo_cut, prev + 1), hi_cut - (world - 1 - r))
        cuts.append(b)
        prev = b
    edges = [0] + cuts + [nz]
    return [Slab(r, world, nx, ny, nz, P, edges[r], edges[r + 1]) for r in range(world)]


@dataclasses.dataclass(frozen=True)
class Halo:
    """One exchange: components [c0, c1] of a 6-component field block (E or
    lamE x, y: 0, 1; Ht or lamHt x, y: 3, 4) of the plane next to the cut;
    side "hi" fills the ghost plane z1 from the rank above, "lo" the ghost
    plane z0 - 1 from the rank below.  `block` names the field block:
    "state" (E, Ht) or "adjoint" (lamE, lamHt)."""
    block: str
    c0: int
    c1: int
    side: str


HALO = {
    "forward_h": Halo("state", 0, 1, "hi"),
    "forward_e": Halo("state", 3, 4, "lo"),
    "inverse_e": Halo("state", 3, 4, "lo"),
    "adjoint_e": Halo("adjoint", 0, 1, "hi"),
    "inverse_h": Halo("state", 0, 1, "hi"),
    "adjoint_h": Halo("adjoint", 3, 4, "lo"),
}

# One forward step n: (kind, name) in order.  "record_e": E^n on the high
# faces (sample steps), "record_h": Ht^{n+1/2} on the low faces, "objective":
# the rank's detector rows of l_n.
FORWARD_STEP = (
    ("record", "record_e"),
    ("exchange", "forward_h"),
    ("op", "forward_h"),
    ("record", "record_h"),
    ("exchange", "forward_e"),
    ("op", "forward_e"),
    ("objective", "objective"),
)

# One reverse step n (Sec. 2: the time-reversed run with the recorded slices
# injected, together with the adjoint).
REVERSE_STEP = (
    ("restore", "restore_h"),          # Ht^{n+1/2} on the low interface layers
    ("seed", "seed"),                  # lam += seed * dl_n on the rank's detector rows
    ("exchange", "inverse_e"),
    ("op", "inverse_e"),               # E^n on the interior, dE = E^{n+1} - E^n
    ("grad", "grad"),                  # rank's design rows: -lamE . dE / eps
    ("exchange", "adjoint_e"),
    ("op", "adjoint_e"),
    ("restore", "restore_e"),          # E^n on the high interface layers
    ("exchange", "inverse_h"),
    ("op", "inverse_h"),               # Ht^{n-1/2} on the interior
    ("exchange", "adjoint_h"),
    ("op", "adjoint_h"),
)


def exchange(slab: Slab, fields, halo: Halo, group=None, z_offset: Optional[int] = None):
    """Fill this rank's ghost plane of `halo` from its neighbour and send the
    neighbour the plane it needs, in place.  `fields` is a torch tensor
    [6][planes][ny][nx] whose plane 0 is the global plane `z_offset`
    (default: slab.z_lo, the rank's own storage).  Point-to-point messages of
    the default process group; every rank of the slab group must call it
    with the same halo."""
    import torch
    import torch.distributed as dist

    off = slab.z_lo if z_offset is None else z_offset
    comps = slice(halo.c0, halo.c1 + 1)
    if halo.side == "hi":
        send_to, send_plane = (slab.rank - 1, slab.z0) if slab.has_lo else (None, None)
        recv_from, ghost = (slab.rank + 1, slab.z1) if slab.has_hi else (None, None)
    else:
        send_to, send_plane = (slab.rank + 1, slab.z1 - 1) if slab.has_hi else (None, None)
        recv_from, ghost = (slab.rank - 1, slab.z0 - 1) if slab.has_lo else (None, None)
    reqs, buf = [], None
    if send_to is not None:
        out = fields[comps, send_plane - off].contiguous()
        reqs.append(dist.isend(out, send_to, group=group))
    if recv_from is not None:
        buf = torch.empty_like(fields[comps, ghost - off])
        reqs.append(dist.irecv(buf, recv_from, group=group))
    for r in reqs:
        r.wait()
    if buf is not None:
        fields[comps, ghost - off].copy_(buf)


def reduce_sum(value: float, group=None) -> float:
    """Sum of a per-rank FP64 scalar (the objective's partial sums)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t[0])


def reduce_absmax(amax: Sequence[float], group=None) -> np.ndarray:
    """Elementwise maximum over ranks (the per-face absmax of one tape sample)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(amax, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.numpy()


def gather_rows(slab: Slab, rows: np.ndarray, lo: int, hi: int, group=None) -> np.ndarray:
    """Assemble a z-sliced array (the design box [lo, hi) along z, leading
    axis) from every rank's owned rows; every rank gets the whole array."""
    import torch
    import torch.distributed as dist
    n = hi - lo
    tail = rows.shape[1:]
    a, b = slab.rows(lo, hi)
    full = torch.zeros((n,) + tuple(tail), dtype=torch.float64)
    if b > a:
        full[a - lo:b - lo] = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.float64))
    dist.all_reduce(full, op=dist.ReduceOp.SUM, group=group)   # disjoint rows: a sum places them
    return full.numpy()
