"""Exact partition function of the periodic L x L square-lattice Ising model.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper (section 1) leans on Onsager's exact solution and quotes
T_c/J = 2.269...; the finite periodic lattice has Kaufman's closed form
(B. Kaufman, Phys. Rev. 76, 1232 (1949); in the notation of A. E. Ferdinand
and M. E. Fisher, Phys. Rev. 185, 832 (1969), eqs. (2.1)-(2.6)):

    Z = 1/2 (2 sinh 2K)^(m n / 2) (Z1 + Z2 + Z3 + Z4),
    Z1 = prod_{r=0}^{n-1} 2 cosh(m gamma_{2r+1} / 2),
    Z2 = prod_{r=0}^{n-1} 2 sinh(m gamma_{2r+1} / 2),
    Z3 = prod_{r=0}^{n-1} 2 cosh(m gamma_{2r} / 2),
    Z4 = prod_{r=0}^{n-1} 2 sinh(m gamma_{2r} / 2),
    cosh gamma_l = cosh 2K coth 2K - cos(pi l / n)   (l >= 1, gamma_l > 0),
    gamma_0 = 2K + ln tanh K                          (negative above T_c),

for an m x n torus with K = J/T, where Z = sum over states of exp(K E_bond).
Everything is evaluated in mpmath at 60 significant digits, so rounding does
not limit the derivatives taken below.
"""
import mpmath as mp

_DPS = 60


def log_partition(L, K, m=None):
    """ln Z of the m x L torus (m defaults to L) at coupling K = J/T."""
    with mp.workdps(_DPS):
        K = mp.mpf(K)
        n = int(L)
        m = n if m is None else int(m)
        c = mp.cosh(2 * K) * mp.coth(2 * K)

        def gamma(l):
            if l == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(mp.pi * l / n))

        half = mp.mpf(m) / 2
        log_z1 = log_z2 = log_z3 = mp.mpf(0)
        z4_sign = 1
        log_z4 = mp.mpf(0)
        for r in range(n):
            g_odd = gamma(2 * r + 1)
            g_even = gamma(2 * r)
            log_z1 += mp.log(2 * mp.cosh(half * g_odd))
            log_z2 += mp.log(2 * mp.sinh(half * g_odd))
            log_z3 += mp.log(2 * mp.cosh(half * g_even))
            s4 = 2 * mp.sinh(half * g_even)
            if s4 == 0:
                z4_sign = 0
            else:
                if s4 < 0:
                    z4_sign = -z4_sign
                log_z4 += mp.log(abs(s4))
        top = max(log_z1, log_z2, log_z3, log_z4)
        total = (mp.exp(log_z1 - top) + mp.exp(log_z2 - top)
                 + mp.exp(log_z3 - top) + z4_sign * mp.exp(log_z4 - top))
        prefactor = mp.log(mp.mpf(1) / 2) + (mp.mpf(m * n) / 2) * mp.log(
            2 * mp.sinh(2 * K))
        return prefactor + top + mp.log(total)


def _derivative(L, K, order):
    """Central difference of ln Z in K with step 1e-15 at 60 digits: the
    truncation error (~1e-30 relative) and the cancellation error (~1e-45)
    are both far below double precision."""
    with mp.workdps(_DPS):
        K = mp.mpf(K)
        h = mp.mpf("1e-15")
        if order == 1:
            return (log_partition(L, K + h) - log_partition(L, K - h)) / (2 * h)
        return (log_partition(L, K + h) - 2 * log_partition(L, K)
                + log_partition(L, K - h)) / (h * h)


def mean_energy_bond(L, K):
    """<E_bond> = d ln Z / dK on the L x L torus."""
    return _derivative(L, K, 1)


def energy_bond_variance(L, K):
    """<E_bond^2> - <E_bond>^2 = d^2 ln Z / dK^2."""
    return _derivative(L, K, 2)


def critical_coupling():
    """K_c = ln(1 + sqrt 2) / 2, i.e. T_c/J = 2 / ln(1 + sqrt 2) = 2.2691..."""
    with mp.workdps(_DPS):
        return mp.log(1 + mp.sqrt(2)) / 2
