"""GPU parity of the XY embedded-cluster update: every record (|C|, levels
and the fixed-point E, Mx, My) and every angle must equal the oracle's, on
the production 15-bit angle grid and on clock-model grids, from hot lattices
(single sites) to cold ones whose clusters span the lattice and run on the
whole team, with ragged shapes and every cluster size."""
import numpy as np
import pytest

import oracle
from _gpu import require_cuda

pytestmark = pytest.mark.gpu


def oracle_xy(dim, L, bits, T, seed, n, t0=0, theta=None, J=1.0):
    kk = oracle.xy_coupling(J, T)
    th = oracle.xy_init(dim, L, bits, seed) if theta is None else np.array(theta, np.uint16)
    rec = oracle.xy_run(dim, L, bits, kk, seed, t0, n, th)
    return rec, th


def assert_xy_equal(got, ref, label):
    for f in ("C", "levels", "E", "Mx", "My"):
        if not np.array_equal(got[f], ref[f]):
            bad = int(np.nonzero(got[f] != ref[f])[0][0])
            raise AssertionError("%s: field %s first differs at update %d: gpu %r oracle %r"
                                 % (label, f, bad, got[bad], ref[bad]))


@pytest.mark.parametrize("dim,L,bits,T,n", [
    (2, 16, 15, 0.9, 400),     # near the BKT temperature
    (2, 33, 15, 0.6, 200),     # ragged, ordered: clusters span the lattice
    (2, 24, 15, 3.0, 400),     # hot: small clusters
    (3, 8, 15, 2.2, 300),      # 3D, near its transition
    (3, 11, 15, 1.5, 100),     # 3D ragged, ordered
    (2, 20, 2, 1.0, 400),      # 4-state clock grid
    (2, 18, 3, 0.8, 300),      # 8-state clock grid
])
def test_records_and_lattice_match_oracle(dim, L, bits, T, n):
    torch, w = require_cuda()
    seed = 5000 + L + bits
    ref, th_ref = oracle_xy(dim, L, bits, T, seed, n)
    lat = w.WolffXY(dim, L, T, seed=seed, angle_bits=bits)
    E0 = lat.measure_full()
    assert E0 == oracle.xy_observables(dim, L, oracle.xy_init(dim, L, bits, seed))
    rec = np.concatenate([lat.step(k) for k in (n // 4, n - n // 4)])
    theta, t = lat.get_state()
    assert lat.measure()[:3] == lat.measure_full()
    lat.close()
    assert_xy_equal(rec, ref, "xy %dD L=%d bits=%d T=%g" % (dim, L, bits, T))
    assert t == n and np.array_equal(theta, th_ref)


@pytest.mark.parametrize("cs,threads", [(1, 128), (2, 256), (4, 512), (16, 512)])
def test_team_shapes_give_the_same_chain(cs, threads):
    """Cold 2D lattice: the clusters cover most of the lattice, so fronts go
    to the team (distributed counters, cluster barrier) and back."""
    torch, w = require_cuda()
    dim, L, bits, T, n, seed = 2, 64, 15, 0.5, 60, 77
    start = np.zeros(L * L, np.uint16)   # ordered: the clusters span the lattice
    ref, th_ref = oracle_xy(dim, L, bits, T, seed, n, theta=start)
    lat = w.WolffXY(dim, L, T, seed=seed, grid_blocks=cs, block_threads=threads)
    lat.set_state(start, 0)
    rec = lat.step(n)
    theta, _ = lat.get_state()
    st = lat.stats()
    lat.close()
    assert_xy_equal(rec, ref, "xy team cs=%d threads=%d" % (cs, threads))
    assert np.array_equal(theta, th_ref)
    assert rec["C"].max() > 1000


def test_state_roundtrip_and_rejection():
    torch, w = require_cuda()
    dim, L, bits, T, seed = 2, 20, 4, 1.1, 9
    lat = w.WolffXY(dim, L, T, seed=seed, angle_bits=bits)
    rng = np.random.default_rng(1)
    th = (rng.integers(0, 16, L * L) << 12).astype(np.uint16)
    lat.set_state(th, 1234)
    back, t = lat.get_state()
    assert t == 1234 and np.array_equal(back, th)
    assert lat.measure()[:3] == oracle.xy_observables(dim, L, th)
    ref, th_ref = oracle_xy(dim, L, bits, T, seed, 150, t0=1234, theta=th)
    rec = lat.step(150)
    assert_xy_equal(rec, ref, "xy after set_state")
    assert np.array_equal(lat.get_state()[0], th_ref)
    bad = th.copy()
    bad[7] |= 1                      # off the 4-bit grid
    with pytest.raises(w.WolffError):
        lat.set_state(bad, 0)
    # a valid lattice is left behind, and it keeps working
    assert lat.measure()[:3] == lat.measure_full()
    lat.step(10)
    lat.close()


def test_infinite_temperature_single_sites():
    torch, w = require_cuda()
    lat = w.WolffXY(2, 32, 1e300, seed=3)
    rec = lat.step(200)
    assert (rec["C"] == 1).all() and (rec["levels"] == 1).all()
    ref, _ = oracle_xy(2, 32, 15, 1e300, 3, 200)
    assert_xy_equal(rec, ref, "xy T=inf")
    lat.close()


def test_ising_entry_points_refuse_xy():
    torch, w = require_cuda()
    lat = w.WolffXY(2, 16, 1.0, seed=1)
    lib = w.load_library()
    import ctypes
    assert lib.measure(lat.handle, None, None, None) == w.WOLFF_EUNSUPPORTED
    assert lib.wolff_get_state(lat.handle, None, None) == w.WOLFF_EUNSUPPORTED
    assert lib.wolff_set_schedule(lat.handle, w.SCHED_PERSISTENT, 0, 0) == w.WOLFF_EUNSUPPORTED
    lat.close()


@pytest.mark.parametrize("dim,L,T,seed", [(2, 1024, 0.89, 6), (3, 128, 2.2, 7)])
def test_full_size_bench_step_every_record(dim, L, T, seed):
    """The bench's XY workloads at full size (2D L=1024 near the BKT
    temperature, 3D L=128 near its transition; ordered start, 200
    equilibration updates): the bench's step of 1000 updates in one launch.
    The same 1000 updates also run as ten launches of 100 with a snapshot
    after each; the oracle replays every segment from its snapshot (one host
    thread per segment; the oracle's calls release the interpreter lock), and
    every record and every snapshot must match bit for bit.  The one-launch
    records must equal the segmented ones."""
    from concurrent.futures import ThreadPoolExecutor
    torch, w = require_cuda()
    N = L ** dim
    lat = w.WolffXY(dim, L, T, seed=seed)
    lat.set_state(np.zeros(N, np.uint16), 0)
    lat.step(200, records=False)
    start, t0 = lat.get_state()
    one = lat.step(1000)
    lat.set_state(start, t0)
    snaps, segs = [(start, t0)], []
    for _ in range(10):
        segs.append(lat.step(100))
        snaps.append(lat.get_state())
    assert lat.measure()[:3] == lat.measure_full()
    lat.close()
    assert np.array_equal(np.concatenate(segs), one)
    kk = oracle.xy_coupling(1.0, T)
    oracle.xy_cos(0)   # the oracle's cosine table is built once, before the threads

    def replay(k):
        th = np.array(snaps[k][0], np.uint16)
        rec = oracle.xy_run_local(dim, L, 15, kk, seed, snaps[k][1], 100, th)
        return rec, th
    with ThreadPoolExecutor(max_workers=10) as ex:
        out = list(ex.map(replay, range(10)))
    for k, (rec, th) in enumerate(out):
        assert_xy_equal(segs[k], rec, "xy full size %dD segment %d" % (dim, k))
        assert np.array_equal(th, snaps[k + 1][0]), k
    assert one["C"].mean() > 1000
