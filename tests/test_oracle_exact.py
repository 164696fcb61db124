"""Exact results that pin the enumerator and the Kaufman solver.

Two independent exact routes must agree: the oracle's enumeration of all 2^16
states of the 4 x 4 torus and Kaufman's closed form for the periodic square
lattice.  The 3D enumerations are pinned by counting arguments on the lowest
excitations, and the large-L Kaufman energy by Onsager's value at T_c
(section 1 of the paper cites the exact solution and T_c/J = 2.269...).
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
from oracle import kaufman


@pytest.fixture(scope="module")
def dos_2d4():
    return oracle.density_of_states(2, 4)


def test_enumeration_totals(dos_2d4):
    g, E, M = dos_2d4
    assert int(g.sum()) == 2**16
    assert np.array_equal(g, g[:, ::-1])          # M -> -M symmetry
    ge = g.sum(axis=1)
    assert ge[E == 32][0] == 2                    # two ground states
    assert ge[E == 32 - 8][0] == 2 * 16           # one reversed spin
    assert ge[E == 32 - 12][0] == 2 * 32          # a reversed NN pair
    assert int((ge * E).sum()) == 0               # <E_bond> at infinite T


@pytest.mark.parametrize("K", [0.1, 0.3, 0.44068679350977147, 0.55, 0.9])
def test_kaufman_equals_enumeration(dos_2d4, K):
    g, E, _ = dos_2d4
    ge = g.sum(axis=1)
    with mp.workdps(40):
        Zb = mp.fsum(mp.mpf(int(c)) * mp.exp(mp.mpf(K) * int(e))
                     for c, e in zip(ge, E) if c > 0)
        Eb = mp.fsum(mp.mpf(int(c)) * int(e) * mp.exp(mp.mpf(K) * int(e))
                     for c, e in zip(ge, E) if c > 0) / Zb
        assert abs(kaufman.log_partition(4, K) - mp.log(Zb)) < mp.mpf("1e-25")
        assert abs(kaufman.mean_energy_bond(4, K) - Eb) < mp.mpf("1e-12")
    ex = oracle.exact_moments(2, 4, 1.0, 1.0 / K, g)
    assert abs(ex["E"] - float(Eb)) < 1e-9


def test_kaufman_rectangular_against_enumeration():
    # a 4 x 2 torus (m = 2 rows of n = 4) has its own closed form; enumerate it
    # with plain numpy over 2^8 states
    m, n = 2, 4
    states = ((np.arange(256)[:, None] >> np.arange(8)) & 1) * 2 - 1
    s = states.reshape(256, m, n)
    e = (s * np.roll(s, 1, axis=2)).sum(axis=(1, 2)) + (s * np.roll(s, 1, axis=1)).sum(axis=(1, 2))
    for K in (0.2, 0.6):
        Z = float(np.exp(K * e).sum())
        assert abs(float(kaufman.log_partition(n, K, m=m)) - math.log(Z)) < 1e-12


def test_onsager_energy_at_tc():
    # E/N -> -sqrt(2) J at T_c as L -> infinity; the periodic finite-size
    # correction is O(1/L), so L = 4096 must sit within 1e-3
    Kc = kaufman.critical_coupling()
    e4096 = float(kaufman.mean_energy_bond(4096, Kc)) / 4096**2
    assert abs(e4096 - math.sqrt(2)) < 1e-3
    e512 = float(kaufman.mean_energy_bond(512, Kc)) / 512**2
    # and the deviation shrinks roughly as 1/L
    assert abs(e512 - math.sqrt(2)) > 4 * abs(e4096 - math.sqrt(2))


@pytest.mark.parametrize("L", [2, 3])
def test_enumeration_3d_counts(L):
    g, E, M = oracle.density_of_states(3, L)
    n = L**3
    assert int(g.sum()) == 2**n
    ge = g.sum(axis=1)
    top = 3 * n
    assert ge[E == top][0] == 2
    assert ge[E == top - 12][0] == 2 * n                  # one reversed spin
    if L == 3:
        assert ge[E == top - 20][0] == 2 * 3 * n          # reversed NN pair
    else:
        # at L = 2 every neighbour pair is joined by a double bond: a reversed
        # pair (12 cube edges, times the global flip) and a reversed 2 x 2
        # layer (6 of them) both cut 8 bonds
        assert ge[E == top - 16][0] == 2 * (3 * n // 2) + 6
    assert np.array_equal(g, g[:, ::-1])
    assert int((ge * E).sum()) == 0
