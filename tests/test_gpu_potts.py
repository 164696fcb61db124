"""GPU q-state Potts update vs the CPU oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest

import oracle
from _gpu import assert_records_equal, require_cuda

pytestmark = pytest.mark.gpu


def potts_ref(dim, L, q, T, seed, n, c=None):
    thr = oracle.potts_threshold(1.0, T)
    c = oracle.potts_init(dim, L, q, seed) if c is None else np.array(c, dtype=np.int8)
    rec = oracle.potts_run(dim, L, q, thr, seed, 0, n, c)
    return rec, c


CASES = [(2, 16, 3, 1.0, 600), (2, 37, 4, 0.9, 300), (3, 8, 3, 1.6, 300), (2, 2, 3, 0.8, 200),
         (3, 3, 5, 1.2, 200), (2, 128, 3, 0.99497, 80), (3, 24, 3, 1.8, 40)]


@pytest.mark.parametrize("cluster,threads", [(1, 256), (4, 256), (16, 512)])
@pytest.mark.parametrize("dim,L,q,T,n", CASES)
def test_potts_matches_oracle(dim, L, q, T, n, cluster, threads):
    torch, w = require_cuda()
    seed = 900 + L + q
    ref, c_ref = potts_ref(dim, L, q, T, seed, n)
    lat = w.WolffLattice(dim, L, T, seed=seed, q=q)
    try:
        lat.set_schedule(w.SCHED_CLUSTER, cluster, threads)
    except w.WolffError:
        pytest.skip("cluster size not launchable")
    lat.set_local_thresholds(32, 8)
    rec = lat.step(n)
    cols, t = lat.get_state()
    assert lat.measure()[:2] == lat.measure_full()
    lat.close()
    assert_records_equal(rec, ref, "potts q=%d %dD L=%d" % (q, dim, L))
    assert np.array_equal(cols, c_ref) and t == n


def test_potts_q2_equals_ising_at_half_coupling():
    torch, w = require_cuda()
    dim, L, T, n = 2, 64, 2.1, 300
    potts = w.WolffLattice(dim, L, T, J=1.0, seed=5, q=2)
    ising = w.WolffLattice(dim, L, T, J=0.5, seed=5, schedule=w.SCHED_CLUSTER)
    rp, ri = potts.step(n), ising.step(n)
    N = L * L
    assert np.array_equal(rp["C"], ri["C"]) and np.array_equal(rp["levels"], ri["levels"])
    assert np.array_equal(2 * rp["E"] - dim * N, ri["E"])
    assert np.array_equal(2 * rp["M"] - N, ri["M"])
    potts.close()
    ising.close()


def test_potts_state_roundtrip_and_rejects_bad_colours():
    torch, w = require_cuda()
    dim, L, q, T = 2, 20, 4, 0.9
    lat = w.WolffLattice(dim, L, T, seed=3, q=q)
    start = np.zeros(L * L, np.int8)          # ordered start: big clusters
    lat.set_state(start, 0)
    ref, c_ref = potts_ref(dim, L, q, T, 3, 50, c=start)
    assert_records_equal(lat.step(50), ref, "potts ordered start")
    bad = start.copy()
    bad[5] = q
    with pytest.raises(w.WolffError) as ei:
        lat.set_state(bad, 0)
    assert ei.value.status == w.WOLFF_EINVAL
    with pytest.raises(w.WolffError):
        lat.set_schedule(w.SCHED_PERSISTENT)
    lat.close()
