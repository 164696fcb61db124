"""The premise of window mode's conflict rule, checked on the oracle.

Section 2 grows the cluster of update t from its seed through active bonds:
both ends parallel to the seed spin and the bond's draw below the threshold.
Window mode grows consecutive updates on one lattice and commits an update
whose reads an earlier committed update changed only if the change cannot
matter.  This file checks the two facts that rule rests on, for random
lattices, updates and flip sets, with the oracle's own cluster and chain:

- flipping any set of sites that holds no member and no neighbour reached
  through an open boundary bond leaves the cluster and its level count
  unchanged (such a neighbour is anti-parallel, or it would be a member);
- the energy change of the update then differs from the one on the unflipped
  lattice only through the flipped neighbours across closed boundary bonds,
  each turning its bond's term around: +4 in E_bond if the neighbour was
  parallel to the seed spin, -4 if it was anti-parallel.

A control shows the premise is not vacuous: flipping one member or one
open-bond neighbour does change some clusters.
"""
import math

import numpy as np
import pytest

import oracle

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


def neighbour(dim, L, i, d, sign):
    c = [(i // L ** k) % L for k in range(dim)]
    c[d] = (c[d] + sign) % L
    return sum(c[k] * L ** k for k in range(dim))


def bond_draw(seed, t, owner, d):
    """Draw of bond (owner, d): lane d of Philox(owner, t_lo, t_hi, 0) under the seed key."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    return int(oracle.philox4x32_10(key, (owner, t & 0xFFFFFFFF, t >> 32, 0))[d])


def boundary_pairs(dim, L, seed, t, thr, s, member):
    """(neighbour, open, parallel) for every (member, direction) pair whose
    neighbour is outside the cluster; the seed spin is that of any member."""
    sig = int(s[np.flatnonzero(member)[0]])
    pairs = []
    for m in np.flatnonzero(member):
        for d in range(dim):
            for sign in (1, -1):
                b = neighbour(dim, L, int(m), d, sign)
                owner = int(m) if sign == 1 else b
                if member[b]:
                    continue
                pairs.append((b, bond_draw(seed, t, owner, d) < thr, int(s[b]) == sig))
    return pairs


def energy_change(dim, L, thr, seed, t, s):
    """E_bond after update t minus before, from the oracle's chain."""
    a = np.array(s, dtype=np.int8, copy=True)
    rec = oracle.run(dim, L, thr, seed, t, 1, a)
    return int(rec["E"][0]) - oracle.energy_bond(dim, L, s)


@pytest.mark.parametrize("dim,L,T", [(2, 12, TC2), (2, 10, 2.6), (2, 12, 5.0), (3, 6, 4.5115),
                                     (3, 5, 8.0)])
def test_flips_outside_the_read_set_that_matters(dim, L, T):
    thr = oracle.bond_threshold(1.0, T)
    rng = np.random.default_rng(7000 + 100 * dim + L)
    seed = 31 + L
    n = L ** dim
    changed_by_relevant = 0
    corrections_seen = 0
    for trial in range(80):
        t = int(rng.integers(0, 1 << 40))
        s = rng.choice(np.array([-1, 1], np.int8), size=n)
        member, _, levels = oracle.cluster(dim, L, thr, seed, t, s)
        pairs = boundary_pairs(dim, L, seed, t, thr, s, member)
        # an open boundary bond's neighbour is anti-parallel (else it joins)
        assert not any(op and par for _, op, par in pairs)
        dE = energy_change(dim, L, thr, seed, t, s)
        assert dE == sum(-2 if par else 2 for _, _, par in pairs)
        relevant = member.copy()
        for b, op, _ in pairs:
            if op:
                relevant[b] = True
        # flip a random set of the other sites
        flip = (rng.random(n) < 0.35) & ~relevant
        s2 = s.copy()
        s2[flip] *= -1
        member2, _, levels2 = oracle.cluster(dim, L, thr, seed, t, s2)
        assert np.array_equal(member2, member) and levels2 == levels, trial
        corr = sum((4 if par else -4) for b, op, par in pairs if not op and flip[b])
        corrections_seen += sum(1 for b, op, _ in pairs if not op and flip[b])
        assert energy_change(dim, L, thr, seed, t, s2) == dE + corr, trial
        # control: one relevant site flipped
        k = int(rng.choice(np.flatnonzero(relevant)))
        s3 = s.copy()
        s3[k] *= -1
        member3, _, _ = oracle.cluster(dim, L, thr, seed, t, s3)
        if not np.array_equal(member3, member):
            changed_by_relevant += 1
    assert corrections_seen > 0
    assert changed_by_relevant > 0
