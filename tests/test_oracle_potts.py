"""Pins of the oracle's q-state Potts update (section 6 of the paper names the
Potts model as the straightforward extension).

- q = 2 reduces exactly to the Ising update of coupling J/2 (colour 1 <-> spin
  -1): the whole trajectory must equal the already pinned Ising oracle's.
- The cluster is the connected component of the seed among neighbours of the
  seed's colour joined by active bonds (scipy, from coordinates).
- The new colour is never the old one and is uniform over the q-1 others.
- The enumeration has the closed-form counts of the lowest excitations, and
  the chain reproduces its Boltzmann averages within 3 sigma.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
from _stats import z_score


def coords(dim, L):
    idx = np.arange(L ** dim)
    return [(idx // L ** d) % L for d in range(dim)]


def forward(dim, L, d):
    c = coords(dim, L)
    c[d] = (c[d] + 1) % L
    return sum(c[k] * L ** k for k in range(dim))


@pytest.mark.parametrize("dim,L,T", [(2, 8, 2.0), (2, 16, 2.2691853142130221), (3, 6, 4.5115),
                                     (2, 2, 1.5), (3, 3, 3.0)])
def test_q2_is_ising_at_half_coupling(dim, L, T):
    J = 1.0
    assert oracle.potts_threshold(J, T) == oracle.bond_threshold(J / 2, T)
    seed = 40 + L
    c = oracle.potts_init(dim, L, 2, seed)
    s = oracle.init_lattice(dim, L, seed)
    assert np.array_equal(s, (1 - 2 * c.astype(np.int64)).astype(np.int8))
    thr = oracle.potts_threshold(J, T)
    rp = oracle.potts_run(dim, L, 2, thr, seed, 0, 400, c)
    ri = oracle.run(dim, L, thr, seed, 0, 400, s)
    N = L ** dim
    assert np.array_equal(rp["C"], ri["C"]) and np.array_equal(rp["levels"], ri["levels"])
    assert np.array_equal(2 * rp["E"] - dim * N, ri["E"])
    assert np.array_equal(2 * rp["M"] - N, ri["M"])
    assert np.array_equal(s, (1 - 2 * c.astype(np.int64)).astype(np.int8))


@pytest.mark.parametrize("dim,L,q,T", [(2, 9, 3, 1.0), (2, 16, 4, 0.9), (3, 5, 3, 1.6),
                                       (2, 3, 5, 0.7)])
def test_potts_cluster_is_connected_component(dim, L, q, T):
    thr = oracle.potts_threshold(1.0, T)
    n = L ** dim
    for seed in (3, 11):
        c = oracle.potts_init(dim, L, q, seed)
        for t in (0, 1, 7, 2**32 + 5):
            member, lst, levels, nc = oracle.potts_cluster(dim, L, q, thr, seed, t, c)
            x = oracle.philox4x32_10((seed & 0xFFFFFFFF, seed >> 32), [0, t & 0xFFFFFFFF, t >> 32, 1])
            i0 = (int(x[0]) * n) >> 32
            c0 = int(c[i0])
            assert lst[0] == i0
            assert nc != c0 and nc == (c0 + 1 + ((int(x[1]) * (q - 1)) >> 32)) % q
            rows, cols = [], []
            key = (seed & 0xFFFFFFFF, seed >> 32)
            for d in range(dim):
                j = forward(dim, L, d)
                for o in range(n):
                    r = int(oracle.philox4x32_10(key, [o, t & 0xFFFFFFFF, t >> 32, 0])[d])
                    if c[o] == c0 and c[j[o]] == c0 and r < thr:
                        rows.append(o)
                        cols.append(int(j[o]))
            A = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
            _, lab = connected_components(A, directed=False)
            assert np.array_equal(member, lab == lab[i0])


def test_new_colour_uniform_over_the_others():
    q, dim, L, seed = 5, 2, 10, 2
    c = oracle.potts_init(dim, L, q, seed)
    thr = oracle.potts_threshold(1.0, 50.0)   # tiny clusters, we only look at colours
    counts = np.zeros((q, q))
    for t in range(3000):
        _, lst, _, nc = oracle.potts_cluster(dim, L, q, thr, seed, t, c)
        counts[c[lst[0]], nc] += 1
    assert np.all(np.diag(counts) == 0)
    for a in range(q):
        row = counts[a][np.arange(q) != a]
        expect = row.sum() / (q - 1)
        assert np.all(np.abs(row - expect) < 5 * math.sqrt(expect) + 1)


@pytest.mark.parametrize("dim,L,q", [(2, 3, 3), (3, 2, 3), (2, 3, 4)])
def test_potts_enumeration_counts(dim, L, q):
    g, E, Z0 = oracle.potts_density_of_states(dim, L, q)
    n = L ** dim
    assert int(g.sum()) == q ** n
    ge = g.sum(axis=1)
    top = dim * n
    assert ge[top] == q                            # uniform colourings
    if L >= 3:
        assert ge[top - 2 * dim] == q * (q - 1) * n    # one site recoloured
    else:
        # at L = 2 each neighbour pair carries two bonds: one recoloured site
        # breaks 2D bonds all the same (D neighbours, two bonds each)
        assert ge[top - 2 * dim] == q * (q - 1) * n
    gz = g.sum(axis=0)
    for k in range(n + 1):   # N0 is binomial(n, 1/q) over all colourings
        assert gz[k] == math.comb(n, k) * (q - 1) ** (n - k)


@pytest.mark.parametrize("dim,L,q,T", [(2, 3, 3, 0.8), (2, 3, 3, 1.0), (2, 3, 3, 1.6),
                                       (3, 2, 3, 1.5)])
def test_potts_chain_matches_enumeration(dim, L, q, T):
    thr = oracle.potts_threshold(1.0, T)
    c = oracle.potts_init(dim, L, q, 77)
    rec = oracle.potts_run(dim, L, q, thr, 77, 0, 300_200, c)[200:]
    ex = oracle.potts_exact_moments(dim, L, q, 1.0, T)
    E = rec["E"].astype(np.float64)
    N0 = rec["M"].astype(np.float64)
    for x, exact, name in ((E, ex["E"], "E"), (N0, ex["N0"], "N0"), (N0 ** 2, ex["N0_2"], "N0^2")):
        z = z_score(x, exact)
        assert abs(z) < 3.0, (dim, L, q, T, name, z)
