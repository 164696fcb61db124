"""Pins of the oracle's XY embedded-cluster update (Wolff 1989; section 6 of
the paper names the XY model as the next extension of its cluster growth).

- The fixed-point cosine table is the rounded cosine (Python's math.cos), and
  its symmetry extension is exact: cos(-a) = cos(a), cos(a + pi) = -cos(a).
- The e^-y of the bond test is within 2 ulp of math.exp and decreasing; the
  threshold is floor(2^32 (1 - e^-y)) within one unit.
- The reflection theta -> pi + 2 phi - theta reverses the projection on r
  and keeps the perpendicular one, exactly.
- At infinite temperature every cluster is the seed alone.
- The cluster is the seed's connected component of the bonds active by the
  embedded Ising rule (scipy, from coordinates and the pinned bond words).
- With angle_bits = 2 (3) the model is the 4 (8)-state clock model, whose
  Boltzmann averages of the energy and |M|^2 are enumerated here from
  cos(k pi / 2) and cos(k pi / 4) over all 4^9, 4^8 and 8^4 states; the chain
  reproduces them within 3.5 sigma (and the 4-state energy histogram passes
  a chi-squared test).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components, shortest_path
from scipy.stats import chi2

import oracle
from _stats import z_score


def coords(dim, L):
    idx = np.arange(L ** dim)
    return [(idx // L ** d) % L for d in range(dim)]


def forward(dim, L, d):
    c = coords(dim, L)
    c[d] = (c[d] + 1) % L
    return sum(c[k] * L ** k for k in range(dim))


def test_table_is_rounded_cosine():
    t = oracle.xy_table()
    ref = np.array([round(math.cos(math.pi * k / 32768.0) * 2 ** 30) for k in range(16385)])
    assert np.array_equal(t.astype(np.int64), ref)
    assert t[0] == 2 ** 30 and t[16384] == 0


def test_cosine_symmetries_are_exact():
    rng = np.random.default_rng(3)
    for a in list(rng.integers(0, 65536, 3000)) + [0, 16384, 32768, 49152, 1, 65535]:
        a = int(a)
        c = oracle.xy_cos(a)
        assert oracle.xy_cos(-a) == c
        assert oracle.xy_cos(a + 32768) == -c
        assert abs(c - 2 ** 30 * math.cos(2 * math.pi * a / 65536)) <= 1.0


def test_exp_neg_within_two_ulp():
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.uniform(0, 3, 4000), rng.uniform(0, 60, 2000), [0.0, 1e-300, 0.5]])
    for y in ys:
        got, ref = oracle.xy_exp_neg(float(y)), math.exp(-float(y))
        assert abs(got - ref) <= 2 * math.ulp(ref), (y, got, ref)
    grid = np.linspace(0, 5, 20001)
    vals = [oracle.xy_exp_neg(float(y)) for y in grid]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
    assert oracle.xy_exp_neg(2000.0) == 0.0


def test_threshold_is_floor_of_probability():
    kk = oracle.xy_coupling(1.0, 0.9)
    assert kk == math.ldexp(2.0 / 0.9, -60)
    assert oracle.xy_threshold(0, kk) == 0 and oracle.xy_threshold(-5, kk) == 0
    rng = np.random.default_rng(7)
    prev = 0
    for prod in sorted(int(x) for x in rng.integers(1, 2 ** 60, 3000)):
        thr = oracle.xy_threshold(prod, kk)
        ref = math.floor((1.0 - math.exp(-kk * float(prod))) * 2 ** 32)
        assert abs(thr - ref) <= 1
        assert thr >= prev
        prev = thr
    assert oracle.xy_threshold(2 ** 60, math.ldexp(2000.0, -60)) == 2 ** 32


def test_reflection_reverses_the_projection_only():
    for phi in (0, 1, 8192, 12345, 40000, 65535):
        for theta in range(0, 65536, 97):
            new = (32768 + 2 * phi - theta) & 0xFFFF
            assert oracle.xy_cos(new - phi) == -oracle.xy_cos(theta - phi)
            assert oracle.xy_cos(new - phi - 16384) == oracle.xy_cos(theta - phi - 16384)
            assert (32768 + 2 * phi - new) & 0xFFFF == theta


@pytest.mark.parametrize("dim,L", [(2, 9), (3, 5)])
def test_infinite_temperature_flips_one_site(dim, L):
    th = oracle.xy_init(dim, L, 15, 11)
    before = th.copy()
    rec = oracle.xy_run(dim, L, 15, 0.0, 11, 0, 50, th)
    assert (rec["C"] == 1).all() and (rec["levels"] == 1).all()
    assert int((th != before).sum()) <= 50


@pytest.mark.parametrize("dim,L,T,bits", [(2, 6, 0.7, 15), (2, 7, 1.2, 15), (3, 4, 1.5, 15),
                                          (2, 6, 0.5, 3)])
def test_cluster_is_connected_component(dim, L, T, bits):
    seed = 300 + L
    kk = oracle.xy_coupling(1.0, T)
    th = oracle.xy_init(dim, L, bits, seed)
    oracle.xy_run(dim, L, bits, kk, seed, 0, 20, th, records=False)
    n = L ** dim
    for t in range(20, 40):
        member, lst, levels, phi = oracle.xy_cluster(dim, L, bits, kk, seed, t, th)
        proj = np.array([oracle.xy_cos(int(a) - phi) for a in th], dtype=np.int64)
        rows, cols = [], []
        for d in range(dim):
            nb = forward(dim, L, d)
            for i in range(n):
                w = oracle.philox4x32_10((seed & 0xFFFFFFFF, seed >> 32),
                                         [i, t & 0xFFFFFFFF, t >> 32, 0])[d]
                prod = int(proj[i]) * int(proj[nb[i]])
                if int(w) < oracle.xy_threshold(prod, kk):
                    rows.append(i)
                    cols.append(int(nb[i]))
        g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n)).tocsr()
        _, lab = connected_components(g, directed=False)
        i0 = int(lst[0])
        assert np.array_equal(member, lab == lab[i0])
        dist = shortest_path(g, directed=False, unweighted=True, indices=i0)
        assert levels == int(dist[member].max()) + 1
        # apply the update as the run does
        th[member] = ((32768 + 2 * phi - th[member].astype(np.int64)) & 0xFFFF).astype(np.uint16)


def clock_exact(dim, L, q, K):
    """<E>/bond-sum and <|M|^2> of the q-state clock model by enumeration,
    energies from cos(2 pi k / q); bonds are the D*N forward bonds."""
    n = L ** dim
    cosk = np.cos(2 * np.pi * np.arange(q) / q)
    sink = np.sin(2 * np.pi * np.arange(q) / q)
    nbs = [forward(dim, L, d) for d in range(dim)]
    states = np.array(list(itertools.product(range(q), repeat=n)), dtype=np.int64)
    E = np.zeros(len(states))
    for d in range(dim):
        E += cosk[(states - states[:, nbs[d]]) % q].sum(axis=1)
    M2 = cosk[states].sum(axis=1) ** 2 + sink[states].sum(axis=1) ** 2
    w = np.exp(K * (E - E.max()))
    w /= w.sum()
    return float((w * E).sum()), float((w * M2).sum()), E, w


@pytest.mark.parametrize("dim,L,bits,T", [(2, 3, 2, 1.0), (2, 3, 2, 0.6), (3, 2, 2, 1.3),
                                          (2, 2, 3, 0.8)])
def test_clock_limit_matches_enumeration(dim, L, bits, T):
    q = 2 ** bits
    K = 1.0 / T
    e_ex, m2_ex, E_all, w = clock_exact(dim, L, q, K)
    seed = 77 + 10 * dim + L + bits
    th = oracle.xy_init(dim, L, bits, seed)
    kk = oracle.xy_coupling(1.0, T)
    oracle.xy_run(dim, L, bits, kk, seed, 0, 2000, th, records=False)
    rec = oracle.xy_run(dim, L, bits, kk, seed, 2000, 200000, th)
    E = rec["E"] / 2.0 ** 30
    M2 = (rec["Mx"] / 2.0 ** 30) ** 2 + (rec["My"] / 2.0 ** 30) ** 2
    assert abs(z_score(E, e_ex)) < 3.5
    assert abs(z_score(M2, m2_ex)) < 3.5
    if q == 4:
        # integer energies: compare the histogram (every 20th update, nearly independent)
        vals = np.round(E[::20]).astype(int)
        levels = np.unique(np.round(E_all).astype(int))
        exp_p = np.array([w[np.round(E_all).astype(int) == v].sum() for v in levels])
        obs = np.array([(vals == v).sum() for v in levels])
        keep = exp_p * len(vals) >= 10
        stat = (((obs - exp_p * len(vals)) ** 2) / (exp_p * len(vals)))[keep].sum()
        assert stat < chi2.ppf(0.999, keep.sum() - 1)
