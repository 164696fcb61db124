"""Pins of the oracle's lattice, observables and cluster construction.

The cluster of one update has a plain definition (section 2, steps (i)-(iv)):
the connected component of the seed site in the graph whose edges are the
active bonds (both ends parallel to the seed spin, bond random number below
the threshold).  The graph is rebuilt here from lattice coordinates with
numpy and handed to scipy's connected-component and breadth-first routines,
so the oracle's neighbour indexing, bond ownership, threshold test, ic/in
list and generation count are all checked against library code.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import breadth_first_order, connected_components, shortest_path

import oracle

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


def coords(dim, L):
    idx = np.arange(L ** dim)
    return [(idx // L ** d) % L for d in range(dim)]


def forward(dim, L, d):
    """Index of the forward neighbour along axis d, from coordinates."""
    c = coords(dim, L)
    c[d] = (c[d] + 1) % L
    return sum(c[k] * L ** k for k in range(dim))


def bond_randoms(dim, L, seed, t):
    """r[o, d] for every bond (o, d) from the oracle's Philox (pinned separately)."""
    n = L ** dim
    r = np.zeros((n, dim), dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for o in range(n):
        out = oracle.philox4x32_10(key, [o, t & 0xFFFFFFFF, t >> 32, 0])
        r[o, :] = out[:dim]
    return r


def reference_cluster(dim, L, thr, seed, t, s):
    n = L ** dim
    i0 = oracle.seed_site(seed, t, n)
    sigma0 = s[i0]
    r = bond_randoms(dim, L, seed, t)
    rows, cols = [], []
    for d in range(dim):
        j = forward(dim, L, d)
        o = np.arange(n)
        active = (s[o] == sigma0) & (s[j] == sigma0) & (r[o, d] < thr)
        rows.append(o[active])
        cols.append(j[active])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    A = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    _, labels = connected_components(A, directed=False)
    member = labels == labels[i0]
    dist = shortest_path(A, unweighted=True, directed=False, indices=i0)
    levels = int(dist[member].max()) + 1
    order = breadth_first_order(A, i0, directed=False, return_predecessors=False)
    return member, i0, levels, order


CASES = [(2, 2, 1.0), (2, 3, TC2), (2, 4, TC2), (2, 5, 1.5), (2, 16, TC2),
         (2, 16, 3.5), (2, 37, TC2), (3, 2, 4.5115), (3, 3, 4.5115),
         (3, 5, 4.5115), (3, 8, 3.0), (3, 7, 6.0)]


@pytest.mark.parametrize("dim,L,T", CASES)
def test_cluster_is_connected_component(dim, L, T):
    thr = oracle.bond_threshold(1.0, T)
    for seed in (1, 77):
        s = oracle.init_lattice(dim, L, seed)
        for t in (0, 1, 5, 2**32 + 3):
            member, lst, levels = oracle.cluster(dim, L, thr, seed, t, s)
            ref_member, i0, ref_levels, order = reference_cluster(dim, L, thr, seed, t, s)
            assert lst[0] == i0
            assert np.array_equal(member, ref_member)
            assert len(lst) == member.sum() == len(set(lst.tolist()))
            assert levels == ref_levels
            assert set(order.tolist()) == set(lst.tolist())
            assert np.all(s[lst] == s[i0])          # every member aligned


def test_seed_site_definition():
    for seed in (1, 2, 3):
        for t in (0, 1, 12345, 2**33 + 1):
            x = oracle.philox4x32_10((seed & 0xFFFFFFFF, seed >> 32),
                                     [0, t & 0xFFFFFFFF, t >> 32, 1])[0]
            for n in (4, 256, 16777216, 27):
                assert oracle.seed_site(seed, t, n) == (int(x) * n) >> 32


def test_init_lattice_draws():
    s = oracle.init_lattice(2, 64, 5)
    assert set(np.unique(s).tolist()) <= {-1, 1}
    for i in (0, 1, 4095, 1234):
        top = oracle.philox4x32_10((5, 0), [i, 0, 0, 2])[0] >> 31
        assert s[i] == (-1 if top else 1)
    big = oracle.init_lattice(2, 512, 2)
    assert abs(int(big.sum())) < 5 * 512     # +-1 fair coin: sd = 512


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("L", [2, 3, 4, 6])
def test_observable_closed_forms(dim, L):
    n = L ** dim
    up = np.ones(n, dtype=np.int8)
    assert oracle.energy_bond(dim, L, up) == dim * n
    assert oracle.magnetisation(dim, L, up) == n
    one = up.copy()
    one[n // 2] = -1
    # one reversed spin breaks its 2D bonds (two of them double at L = 2)
    assert oracle.energy_bond(dim, L, one) == dim * n - 4 * dim
    assert oracle.magnetisation(dim, L, one) == n - 2
    c = coords(dim, L)
    parity = sum(c) % 2
    if L % 2 == 0:
        board = np.where(parity == 0, 1, -1).astype(np.int8)
        assert oracle.energy_bond(dim, L, board) == -dim * n
        assert oracle.magnetisation(dim, L, board) == 0
    for axis in range(dim):
        if L % 2 == 0:
            slab = np.where(c[axis] < L // 2, 1, -1).astype(np.int8)
            # two domain walls, each cutting n/L bonds along the axis
            assert oracle.energy_bond(dim, L, slab) == dim * n - 4 * (n // L)


def test_threshold_exact_values():
    # At T_c of the square lattice p = 1 - exp(-ln(1 + sqrt 2)) = 2 - sqrt 2,
    # so floor(p 2^32) = 2^33 - ceil(sqrt(2^65)) exactly.
    exact = 2**33 - math.isqrt(2**65) - 1
    assert oracle.bond_threshold(1.0, TC2) == exact == 2515933592
    assert oracle.bond_threshold(0.0, 1.0) == 0
    assert oracle.bond_threshold(1.0, float("inf")) == 0
    assert oracle.bond_threshold(1.0, 1e-3) == 2**32
    ts = [0.5, 1.0, 2.0, TC2, 3.0, 4.5115, 10.0]
    thr = [oracle.bond_threshold(1.0, T) for T in ts]
    assert all(a >= b for a, b in zip(thr, thr[1:]))
    for T in ts:
        p = -math.expm1(-2.0 / T)
        assert abs(oracle.bond_threshold(1.0, T) - p * 2**32) <= 1.0


def test_special_cases():
    # thr = 0: no bond is ever active, every cluster is the seed alone
    s = oracle.init_lattice(2, 8, 3)
    rec = oracle.run(2, 8, 0, 3, 0, 50, s)
    assert np.all(rec["C"] == 1) and np.all(rec["levels"] == 1)
    # thr = 2^32 from the all-up state: the whole lattice flips
    for dim, L in ((2, 8), (3, 4), (2, 5)):
        n = L ** dim
        s = np.ones(n, dtype=np.int8)
        rec = oracle.run(dim, L, 2**32, 9, 0, 3, s)
        assert list(rec["C"]) == [n] * 3
        assert list(rec["M"]) == [-n, n, -n]
        assert list(rec["E"]) == [dim * n] * 3
    # checkerboard start: all neighbours anti-parallel, first cluster is one site
    for dim, L in ((2, 8), (3, 4)):
        c = coords(dim, L)
        board = np.where(sum(c) % 2 == 0, 1, -1).astype(np.int8)
        rec = oracle.run(dim, L, 2**32, 4, 0, 1, board)
        assert rec["C"][0] == 1


def test_run_records_match_definitions():
    dim, L, seed = 2, 12, 8
    thr = oracle.bond_threshold(1.0, TC2)
    s = oracle.init_lattice(dim, L, seed)
    s0 = s.copy()
    rec = oracle.run(dim, L, thr, seed, 0, 30, s)
    s1 = s0.copy()
    for t in range(30):
        member, lst, levels = oracle.cluster(dim, L, thr, seed, t, s1)
        s1[member] = -s1[member]
        assert rec["C"][t] == member.sum() and rec["levels"][t] == levels
        assert rec["M"][t] == int(s1.astype(np.int64).sum())
        assert rec["E"][t] == oracle.energy_bond(dim, L, s1)
    assert np.array_equal(s, s1)
    # segments compose: 30 updates == 12 + 18 from the intermediate state
    s2 = s0.copy()
    r1 = oracle.run(dim, L, thr, seed, 0, 12, s2)
    r2 = oracle.run(dim, L, thr, seed, 12, 18, s2)
    assert np.array_equal(np.concatenate([r1, r2]), rec)
    assert np.array_equal(s2, s)
