"""Pins of the oracle's local-recount runs (run_local, xy_run_local).

run_local keeps E_bond and M by recounting, before and after each flip, only
the terms of the bonds and sites the flip touches.  It is pinned against
run(), which recounts both observables from their definitions after every
update (itself pinned by closed forms and exact enumeration): every record
and the final lattice must be equal.  The cases cover both dimensions, L = 2
(double bonds: the forward and backward neighbour along an axis coincide),
odd and even sides, temperatures from always-bonding to never-bonding, and
random and ordered starts, so a dropped or doubled bond term, a wrong
neighbour orientation or a sign slip in either observable changes a record.
"""
import math

import numpy as np
import pytest

import oracle

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


@pytest.mark.parametrize("dim,L", [(2, 2), (2, 3), (2, 4), (2, 7), (2, 16), (2, 33),
                                   (3, 2), (3, 3), (3, 4), (3, 7), (3, 10)])
@pytest.mark.parametrize("T", [0.05, 1.5, TC2, 4.5115, 9.0, float("inf")])
@pytest.mark.parametrize("start", ["random", "ordered"])
def test_run_local_equals_full_recount(dim, L, T, start):
    seed = 5000 + 10 * L + dim
    thr = oracle.bond_threshold(1.0, T)
    s = oracle.init_lattice(dim, L, seed)
    if start == "ordered":
        s[:] = -1
    a, b = s.copy(), s.copy()
    n = 300 if L ** dim <= 400 else 120
    ref = oracle.run(dim, L, thr, seed, 7, n, a)
    got = oracle.run_local(dim, L, thr, seed, 7, n, b)
    assert np.array_equal(got, ref), (dim, L, T, start)
    assert np.array_equal(a, b)
    # in two pieces, the second given the first's E_bond and M
    c = s.copy()
    em = np.array([oracle.energy_bond(dim, L, c), oracle.magnetisation(dim, L, c)], np.int64)
    g1 = oracle.run_local(dim, L, thr, seed, 7, n // 3, c, em)
    assert list(em) == [oracle.energy_bond(dim, L, c), oracle.magnetisation(dim, L, c)]
    g2 = oracle.run_local(dim, L, thr, seed, 7 + n // 3, n - n // 3, c, em)
    assert np.array_equal(np.concatenate([g1, g2]), ref)


def test_run_local_detects_a_dropped_bond_term():
    """The comparison above has teeth: the energy change of a flip that
    forgets the bonds ending at a member (only forward bonds recounted) is
    wrong on a typical update, so such a mistake would fail it."""
    dim, L, seed = 2, 8, 3
    thr = oracle.bond_threshold(1.0, TC2)
    s = oracle.init_lattice(dim, L, seed)
    member, lst, _ = oracle.cluster(dim, L, thr, seed, 0, s)
    after = s.copy()
    after[member] = -after[member]
    full = oracle.energy_bond(dim, L, after) - oracle.energy_bond(dim, L, s)

    def forward_only(x):
        tot = 0
        for i in (int(v) for v in lst):
            for d in range(dim):
                stride = L ** d
                c = (i // stride) % L
                j = i + (((c + 1) % L) - c) * stride
                tot += int(x[i]) * int(x[j])
        return tot
    assert forward_only(after) - forward_only(s) != full or len(lst) == 0
    rec = oracle.run_local(dim, L, thr, seed, 0, 1, s.copy())
    assert int(rec["E"][0]) == oracle.energy_bond(dim, L, after)


@pytest.mark.parametrize("dim,L,bits", [(2, 2, 15), (2, 5, 15), (2, 8, 3), (3, 2, 15),
                                        (3, 4, 15), (3, 5, 2)])
@pytest.mark.parametrize("T", [0.3, 0.9, 2.2, float("inf")])
def test_xy_run_local_equals_full_recount(dim, L, bits, T):
    seed = 7000 + L + bits
    kk = oracle.xy_coupling(1.0, T)
    th = oracle.xy_init(dim, L, bits, seed)
    a, b = th.copy(), th.copy()
    ref = oracle.xy_run(dim, L, bits, kk, seed, 3, 200, a)
    got = oracle.xy_run_local(dim, L, bits, kk, seed, 3, 200, b)
    assert np.array_equal(got, ref), (dim, L, bits, T)
    assert np.array_equal(a, b)
