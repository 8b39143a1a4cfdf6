"""The z-group schedule's ordering argument, checked on the host.

Every half-step (forward H or E, reverse E or H phase) reads the state at
most one plane beyond the cells it writes, and writes only its own cells.
The library splits each half-step into groups of consecutive z chunks
(`fdtd_zgroup_ranges`); group g waits for groups g - 1 and g + 1 of the
half-step before and follows its own group in stream order, and launches
that touch whole faces (tape record / restore) join every group and fork
again.  These tests build that dependency graph over the library's own
ranges and check that every pair of conflicting accesses (read-after-write,
write-after-read, write-after-write on a shared plane) is ordered, for
every chunk count and group count the option allows; a schedule that drops
the neighbour waits must fail the same check.
"""
import ctypes as C
import itertools

import pytest

from paper_2603_24027_gb300 import _capi as A


def ranges(nch, G):
    lo = (C.c_int * 16)()
    hi = (C.c_int * 16)()
    n = A.lib().fdtd_zgroup_ranges(nch, G, lo, hi)
    assert n == min(G, nch)
    return [(lo[g], hi[g]) for g in range(n)]


@pytest.mark.parametrize("nch", range(1, 41))
def test_ranges_cover_the_chunks_once(nch):
    for G in range(1, 17):
        r = ranges(nch, G)
        assert r[0][0] == 0 and r[-1][1] == nch
        for (a0, a1), (b0, b1) in zip(r, r[1:]):
            assert a1 == b0
        sizes = [b - a for a, b in r]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_ranges_reject_bad_arguments():
    lo = (C.c_int * 4)()
    hi = (C.c_int * 4)()
    assert A.lib().fdtd_zgroup_ranges(0, 2, lo, hi) == A.FDTD_EINVAL
    assert A.lib().fdtd_zgroup_ranges(5, 0, lo, hi) == A.FDTD_EINVAL
    assert A.lib().fdtd_zgroup_ranges(5, 2, None, hi) == A.FDTD_EINVAL


def schedule(nz, zc, G, n_phases, join_every, neighbour_waits=True):
    """Nodes (name, planes written, planes read, half-step) in issue order
    and the predecessor sets of the library's launch order.  Conservatively,
    a half-step reads every field on its planes and one plane to each side
    and writes every field on its own planes."""
    nch = -(-nz // zc)
    r = ranges(nch, G)
    planes = [set(range(a * zc, min(b * zc, nz))) for a, b in r]
    halo = [set(range(max(min(p) - 1, 0), min(max(p) + 2, nz))) for p in planes]
    everything = set(range(nz))
    nodes, preds = [], []
    last = [None] * len(r)        # last node on each group's stream
    prev = None                   # the previous grouped phase's nodes
    fork = None                   # the join launch the groups forked after
    for p in range(n_phases):
        if join_every and p % join_every == 0:
            deps = set(x for x in last if x is not None)
            if fork is not None:
                deps.add(fork)
            nodes.append(("join", everything, everything, f"join{p}"))
            preds.append(deps)
            fork = len(nodes) - 1
            last = [None] * len(r)
            prev = None
        cur = []
        for g in range(len(r)):
            deps = set()
            if last[g] is not None:
                deps.add(last[g])
            elif fork is not None:
                deps.add(fork)
            if prev is not None and neighbour_waits:
                for n in (g - 1, g + 1):
                    if 0 <= n < len(r):
                        deps.add(prev[n])
            nodes.append((f"phase{p}.g{g}", planes[g], halo[g], p))
            preds.append(deps)
            cur.append(len(nodes) - 1)
        last = list(cur)
        prev = cur
    return nodes, preds


def unordered_conflicts(nodes, preds):
    """Pairs of conflicting launches of different half-steps with no path
    between them.  (Groups of one half-step never conflict: the fields a
    half-step reads beyond its own planes are not the ones it writes, which
    is what lets all z chunks of a single launch run at once.)"""
    reach = []
    for i, ps in enumerate(preds):
        s = set(ps)
        for q in ps:
            s |= reach[q]
        reach.append(s)
    bad = []
    for j in range(len(nodes)):
        for i in range(j):
            if nodes[i][3] == nodes[j][3]:
                continue
            wi, ri = nodes[i][1], nodes[i][2]
            wj, rj = nodes[j][1], nodes[j][2]
            conflict = (wi & rj) or (ri & wj) or (wi & wj)
            if conflict and i not in reach[j]:
                bad.append((nodes[i][0], nodes[j][0]))
    return bad


@pytest.mark.parametrize("nz,zc", [(100, 8), (100, 16), (23, 4), (23, 1), (300, 8), (9, 8),
                                   (17, 3)])
@pytest.mark.parametrize("join_every", [0, 2, 3])
def test_neighbour_waits_order_every_conflict(nz, zc, join_every):
    for G in range(1, 17):
        nodes, preds = schedule(nz, zc, G, n_phases=7, join_every=join_every)
        assert unordered_conflicts(nodes, preds) == [], (nz, zc, G)


def test_dropping_the_neighbour_waits_is_caught():
    """Negative control: waiting only on the own group's stream leaves the
    halo planes unordered, and the check reports it."""
    for nz, zc, G in itertools.product([100, 23], [4, 8], [3, 4, 6]):
        nodes, preds = schedule(nz, zc, G, n_phases=4, join_every=0, neighbour_waits=False)
        assert unordered_conflicts(nodes, preds), (nz, zc, G)
