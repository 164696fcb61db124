"""The oracle's Markov chain samples the Boltzmann distribution.

Wolff's update satisfies detailed balance, so long runs of the oracle must
reproduce (within 3 sigma, blocking error bars) the exact averages from the
enumerated density of states (2D L = 4, 3D L = 2 and 3), Kaufman's exact
energy of the 16 x 16 torus at T_c (the small parity workload), and the
improved-estimator identity <|C_t|> = <M_{t-1}^2> / N, which relates each
cluster to the configuration it grew from.  A wrong bond probability, a
missing direction or a sign slip in the observables biases at least one of
these.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import kaufman
from _stats import mean_and_error, z_score

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))
TC3 = 4.5115
Z_MAX = 3.0


def chain(dim, L, T, seed, n, burn=200):
    thr = oracle.bond_threshold(1.0, T)
    s = oracle.init_lattice(dim, L, seed)
    rec = oracle.run(dim, L, thr, seed, 0, n + burn, s)
    m_before = np.concatenate([[oracle.magnetisation(dim, L, oracle.init_lattice(dim, L, seed))],
                               rec["M"][:-1]])
    return rec[burn:], m_before[burn:]


def check_against_exact(dim, L, T, seed, n, g=None):
    rec, m_before = chain(dim, L, T, seed, n)
    ex = oracle.exact_moments(dim, L, 1.0, T, g)
    E = rec["E"].astype(np.float64)
    M = rec["M"].astype(np.float64)
    N = L ** dim
    zs = {
        "E": z_score(E, ex["E"]),
        "M2": z_score(M ** 2, ex["M2"]),
        "absM": z_score(np.abs(M), ex["absM"]),
        "M4": z_score(M ** 4, ex["M4"]),
        "C": z_score(rec["C"].astype(np.float64), ex["M2"] / N),
        "C_vs_M2": z_score(rec["C"].astype(np.float64)
                           - m_before.astype(np.float64) ** 2 / N, 0.0),
    }
    for k, z in zs.items():
        assert abs(z) < Z_MAX, (dim, L, T, k, z)
    return rec, ex


@pytest.fixture(scope="module")
def dos_2d4():
    return oracle.density_of_states(2, 4)[0]


@pytest.mark.parametrize("T", [1.5, TC2, 3.5])
def test_2d_l4_moments_and_histogram(dos_2d4, T):
    rec, ex = check_against_exact(2, 4, T, seed=11, n=400_000, g=dos_2d4)
    # joint histogram of (E_bond, M): every bin with probability above 0.5%
    P = ex["P"]
    E0, M0 = ex["E_values"][0], ex["M_values"][0]
    e_idx = rec["E"] - E0
    m_idx = rec["M"] - M0
    worst = 0.0
    for a, b in zip(*np.nonzero(P > 5e-3)):
        ind = ((e_idx == a) & (m_idx == b)).astype(np.float64)
        worst = max(worst, abs(z_score(ind, P[a, b])))
    assert worst < 4.0          # ~ tens of bins: Bonferroni-style margin


def test_3d_l2_moments():
    check_against_exact(3, 2, TC3, seed=12, n=300_000)
    check_against_exact(3, 2, 2.0, seed=13, n=300_000)


@pytest.mark.slow
def test_3d_l3_moments():
    g = oracle.density_of_states(3, 3)[0]
    check_against_exact(3, 3, TC3, seed=14, n=300_000, g=g)


def test_2d_l16_energy_against_kaufman():
    # the small parity workload: 2D L = 16, J = 1, T = T_c
    rec, m_before = chain(2, 16, TC2, seed=1, n=200_000)
    Kc = kaufman.critical_coupling()
    exact = float(kaufman.mean_energy_bond(16, Kc))
    assert abs(z_score(rec["E"].astype(np.float64), exact)) < Z_MAX
    z = z_score(rec["C"].astype(np.float64) - m_before.astype(np.float64) ** 2 / 256, 0.0)
    assert abs(z) < Z_MAX


def test_3d_l8_improved_estimator():
    rec, m_before = chain(3, 8, TC3, seed=3, n=60_000)
    z = z_score(rec["C"].astype(np.float64) - m_before.astype(np.float64) ** 2 / 512, 0.0)
    assert abs(z) < Z_MAX


def test_error_bar_helper_on_iid_data():
    rng = np.random.default_rng(0)
    x = rng.normal(size=100_000)
    mean, err = mean_and_error(x)
    assert abs(err - 1 / math.sqrt(len(x))) < 0.25 / math.sqrt(len(x))
