"""The tiny schedule (one CTA, the whole lattice in shared memory as bit
planes) against the oracle, bit for bit: every record (|C|, levels, E_bond,
M) and the final lattice, on the small workload, ragged and extreme shapes
(rows of one to six words, partial last words), both regimes (warp 0 alone
with drawing warps beside it / every thread), one and two words per thread,
degenerate thresholds, and chains that move between schedules."""
import math

import numpy as np
import pytest

import oracle
from _gpu import assert_records_equal, oracle_trajectory, require_cuda

pytestmark = pytest.mark.gpu

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


def run_tiny(w, dim, L, T, seed, n, threads=0, s0=None, t0=0):
    lat = w.WolffLattice(dim, L, T, seed=seed)
    lat.set_schedule(w.SCHED_TINY, 0, threads)
    if s0 is not None:
        lat.set_state(s0, t0)
    info = lat.info()
    assert info["schedule"] == w.SCHED_TINY and info["grid_blocks"] == 1
    rec = lat.step(n)
    spins, t = lat.get_state()
    E, M, C = lat.measure()
    Ef, Mf = lat.measure_full()
    st = lat.stats()
    lat.close()
    assert t == t0 + n
    assert (E, M) == (Ef, Mf)
    if n:
        assert (E, M, C) == (rec["E"][-1], rec["M"][-1], rec["C"][-1])
    assert st["updates"] == n and st["levels_local"] == int(rec["levels"].sum())
    return rec, spins


def test_small_workload_is_tiny_by_default():
    """2D L=16, J=1, T=Tc, seed 1, 10^4 updates on the default schedule."""
    torch, w = require_cuda()
    ref, s_ref = oracle_trajectory(2, 16, TC2, 1, 10_000)
    lat = w.WolffLattice(2, 16, TC2, seed=1)
    assert lat.info()["schedule"] == w.SCHED_TINY
    rec = lat.step(10_000)
    spins, t = lat.get_state()
    lat.close()
    assert_records_equal(rec, ref, "2D L=16 tiny")
    assert np.array_equal(spins, s_ref) and t == 10_000


def test_3d_l8():
    torch, w = require_cuda()
    ref, s_ref = oracle_trajectory(3, 8, 4.5115, 3, 2_000)
    rec, spins = run_tiny(w, 3, 8, 4.5115, 3, 2_000)
    assert_records_equal(rec, ref, "3D L=8 tiny")
    assert np.array_equal(spins, s_ref)


# L=2 (double bonds), odd L, non powers of two, rows of one to six words
# with full and one-bit last words (L=32, 33, 64, 65), one drawing warp (64
# threads), a single warp on the all-thread path (32), the most threads (768
# in 2D, 512 in 3D), rows of 2 to 16 sites packed several to a warp's draw, and the
# largest lattices the schedule takes (2D L=181: 32761 sites, 3D L=32: 32768)
SHAPES = [
    (2, 2, 1.0, 300, 64), (2, 3, TC2, 300, 96), (3, 2, 4.5115, 300, 64),
    (3, 3, 3.0, 300, 128), (2, 37, TC2, 400, 96), (2, 100, 2.0, 300, 512),
    (3, 13, 4.5115, 300, 256), (3, 17, 4.0, 200, 512), (2, 64, 2.6, 400, 128),
    (2, 32, TC2, 400, 32), (2, 33, TC2, 300, 0), (2, 65, 2.2, 200, 128),
    (2, 181, TC2, 150, 768), (3, 32, 4.5115, 60, 512), (2, 181, 2.1, 40, 544),
    (3, 16, 4.5115, 200, 128), (3, 5, 4.3, 300, 32), (2, 10, TC2, 300, 64),
]


@pytest.mark.parametrize("dim,L,T,n,threads", SHAPES)
def test_ragged_and_extreme_shapes(dim, L, T, n, threads):
    torch, w = require_cuda()
    seed = 1000 + L
    ref, s_ref = oracle_trajectory(dim, L, T, seed, n)
    rec, spins = run_tiny(w, dim, L, T, seed, n, threads)
    assert_records_equal(rec, ref, "%dD L=%d tiny %d threads" % (dim, L, threads))
    assert np.array_equal(spins, s_ref)


# (dim, L, T, updates, thread counts): warp 0 alone (>= 64 threads, at most
# 64 words) and the all-thread path, with one and two words per thread
REGIMES = [
    (2, 32, TC2, 40, (32, 64, 512)), (3, 8, 4.5115, 40, (32, 64, 512)),
    (2, 100, 2.1, 30, (224, 416)), (3, 24, 4.5115, 30, (288, 512)),
    (2, 181, TC2, 12, (544, 768)), (2, 128, TC2, 30, (256, 512)),
]


@pytest.mark.parametrize("dim,L,T,n,threads", REGIMES)
def test_regimes_from_an_ordered_start(dim, L, T, n, threads):
    """Large clusters from an ordered start (whole-lattice clusters, many
    levels) on every regime and word split."""
    torch, w = require_cuda()
    up = np.ones(L ** dim, dtype=np.int8)
    ref, s_ref = oracle_trajectory(dim, L, T, 31, n, s=up)
    for thr in threads:
        rec, spins = run_tiny(w, dim, L, T, 31, n, thr, s0=up)
        assert_records_equal(rec, ref, "%dD L=%d %d threads" % (dim, L, thr))
        assert np.array_equal(spins, s_ref)


def test_degenerate_thresholds():
    torch, w = require_cuda()
    # T = inf: thr = 0, every cluster is the seed alone
    rec, _ = run_tiny(w, 2, 32, float("inf"), 4, 100)
    assert np.all(rec["C"] == 1) and np.all(rec["levels"] == 1)
    ref, _ = oracle_trajectory(2, 32, float("inf"), 4, 100)
    assert_records_equal(rec, ref, "T=inf")
    # T -> 0: thr = 2^32, clusters are whole aligned domains
    for dim, L in ((2, 48), (3, 10)):
        ref, s_ref = oracle_trajectory(dim, L, 1e-3, 6, 50)
        rec, spins = run_tiny(w, dim, L, 1e-3, 6, 50)
        assert_records_equal(rec, ref, "T=0")
        assert np.array_equal(spins, s_ref)


def test_chain_moves_between_schedules():
    """One context: tiny, cluster, persistent, graph and tiny again, the
    records of the whole chain equal to the oracle's; calls of one update
    and of none; records not kept."""
    torch, w = require_cuda()
    dim, L, T, seed = 2, 40, TC2, 17
    ref, s_ref = oracle_trajectory(dim, L, T, seed, 700)
    lat = w.WolffLattice(dim, L, T, seed=seed)
    parts = []
    for sched, n in ((w.SCHED_TINY, 150), (w.SCHED_CLUSTER, 100), (w.SCHED_TINY, 1),
                     (w.SCHED_PERSISTENT, 100), (w.SCHED_TINY, 0), (w.SCHED_GRAPH, 99),
                     (w.SCHED_TINY, 200)):
        lat.set_schedule(sched)
        if n:
            parts.append(lat.step(n))
    assert_records_equal(np.concatenate(parts), ref[:650], "schedule changes")
    lat.set_schedule(w.SCHED_TINY)
    assert lat.step(50, records=False) is None
    spins, t = lat.get_state()
    E, M, C = lat.measure()
    assert t == 700 and np.array_equal(spins, s_ref)
    assert (E, M, C) == (ref["E"][-1], ref["M"][-1], ref["C"][-1])
    lat.close()


def test_host_buffer_path_on_tiny():
    torch, w = require_cuda()
    for dim, L, T, seed in ((3, 8, 4.5115, 12), (3, 12, 4.5115, 13)):
        s0 = oracle.init_lattice(dim, L, seed)
        ref, s_ref = oracle_trajectory(dim, L, T, seed, 300, t0=40, s=s0)
        lat = w.WolffLattice(dim, L, T, seed=seed)
        lat.set_schedule(w.SCHED_TINY)
        rec, spins = lat.run_host(300, spins_in=s0, t_in=40)
        lat.close()
        assert_records_equal(rec, ref, "run_host tiny %dD L=%d" % (dim, L))
        assert np.array_equal(spins, s_ref)


def test_schedule_choice_and_refusals():
    torch, w = require_cuda()
    big = w.WolffLattice(2, 182, TC2, seed=1)   # 33124 sites
    assert big.info()["schedule"] == w.SCHED_CLUSTER
    with pytest.raises(w.WolffError) as ei:
        big.set_schedule(w.SCHED_TINY)
    assert ei.value.status == w.WOLFF_EUNSUPPORTED
    big.close()
    # AUTO: TINY up to 64 words (2D L <= 32, 3D L <= 8), CLUSTER above
    for dim, L, sched in ((2, 32, w.SCHED_TINY), (2, 33, w.SCHED_CLUSTER),
                          (3, 8, w.SCHED_TINY), (3, 9, w.SCHED_CLUSTER)):
        x = w.WolffLattice(dim, L, TC2 if dim == 2 else 4.5115, seed=1)
        assert x.info()["schedule"] == sched, (dim, L)
        x.close()
    mid = w.WolffLattice(2, 65, TC2, seed=1)
    assert mid.info()["schedule"] == w.SCHED_CLUSTER
    mid.set_schedule(w.SCHED_TINY, 1, 768)
    inf = mid.info()
    assert inf["schedule"] == w.SCHED_TINY and inf["block_threads"] == 768
    with pytest.raises(w.WolffError) as ei:          # 2D CTAs take at most 768 threads
        mid.set_schedule(w.SCHED_TINY, 0, 800)
    assert ei.value.status == w.WOLFF_EINVAL
    mid.close()
    edge = w.WolffLattice(2, 181, TC2, seed=1)  # 1086 words: needs >= 543 threads
    assert edge.info()["schedule"] == w.SCHED_CLUSTER
    edge.set_schedule(w.SCHED_TINY)
    assert edge.info()["block_threads"] == 544
    with pytest.raises(w.WolffError) as ei:
        edge.set_schedule(w.SCHED_TINY, 0, 512)
    assert ei.value.status == w.WOLFF_EINVAL
    edge.set_schedule(w.SCHED_AUTO, 0, 512)     # a shape TINY cannot use: CLUSTER
    assert edge.info()["schedule"] == w.SCHED_CLUSTER
    edge.close()
    cube = w.WolffLattice(3, 16, 4.5115, seed=1)   # 3D CTAs take at most 512 threads
    with pytest.raises(w.WolffError) as ei:
        cube.set_schedule(w.SCHED_TINY, 0, 1024)
    assert ei.value.status == w.WOLFF_EINVAL
    cube.close()
    lat = w.WolffLattice(2, 16, TC2, seed=1)
    for blocks, threads in ((2, 0), (0, 48)):
        with pytest.raises(w.WolffError) as ei:
            lat.set_schedule(w.SCHED_TINY, blocks, threads)
        assert ei.value.status == w.WOLFF_EINVAL
    lat.set_schedule(w.SCHED_AUTO, 8, 256)     # a cluster shape: AUTO means CLUSTER
    assert lat.info()["schedule"] == w.SCHED_CLUSTER
    lat.set_schedule(w.SCHED_AUTO)
    assert lat.info()["schedule"] == w.SCHED_TINY
    lat.close()
    potts = w.WolffLattice(2, 16, 1.0, seed=1, q=3)
    assert potts.info()["schedule"] == w.SCHED_CLUSTER
    with pytest.raises(w.WolffError) as ei:
        potts.set_schedule(w.SCHED_TINY)
    assert ei.value.status == w.WOLFF_EUNSUPPORTED
    potts.close()


# (dim, L, T, seed): 2D and 3D, from L=2 to the largest lattices the engine
# takes, at and around T_c
BATCH = [(2, 2, 1.0, 5), (2, 16, TC2, 6), (2, 33, 2.2, 7), (2, 100, TC2, 8), (2, 181, 2.5, 9),
         (3, 2, 4.0, 10), (3, 8, 4.5115, 11), (3, 13, 4.3, 12), (3, 32, 4.6, 13),
         (2, 64, 2.0, 14), (3, 5, 4.5115, 15)]


def test_tiny_batch_keeps_every_chain():
    """Every lattice of a tiny-engine batch (one CTA each, one launch per
    dimension, mixed sizes) follows the oracle's chain across calls."""
    torch, w = require_cuda()
    lats = [w.WolffLattice(d, L, T, seed=s) for d, L, T, s in BATCH]
    batch = w.WolffBatch(len(lats), schedule=w.SCHED_TINY)
    got = [[] for _ in lats]
    for n in (30, 1, 45):
        bufs = [lat.record_buffer(n) for lat in lats]
        batch.run(lats, n, bufs, cluster_size=1, block_threads=0)
        torch.cuda.synchronize()
        for k, lat in enumerate(lats):
            got[k].append(w.records_to_numpy(bufs[k], n))
    batch.close()
    for k, (d, L, T, s) in enumerate(BATCH):
        ref, s_ref = oracle_trajectory(d, L, T, s, 76)
        assert_records_equal(np.concatenate(got[k]), ref, "tiny batch %dD L=%d" % (d, L))
        spins, t = lats[k].get_state()
        assert t == 76 and np.array_equal(spins, s_ref)
        assert lats[k].measure()[:2] == lats[k].measure_full()
        lats[k].close()


def test_tiny_batch_time_budget_and_refusals():
    torch, w = require_cuda()
    specs = [(2, 96, 2.0, 5), (3, 12, 4.0, 6), (2, 40, 2.3, 7), (2, 20, 2.1, 8)]
    lats = [w.WolffLattice(d, L, T, seed=s) for d, L, T, s in specs]
    for lat in lats:
        lat.set_state(np.ones(lat.N, np.int8), 0)   # ordered: large clusters, slow updates
    batch = w.WolffBatch(len(lats), schedule=w.SCHED_TINY)
    got = [[] for _ in lats]
    seen = [0] * len(lats)
    for call in range(6):
        bufs = [lat.record_buffer(400) for lat in lats]
        batch.run(lats, 400, bufs, cluster_size=1, block_threads=0, budget_ns=20_000)
        torch.cuda.synchronize()
        for k, lat in enumerate(lats):
            ran = lat.stats()["updates"] - seen[k]
            seen[k] += ran
            assert 1 <= ran <= 400
            got[k].append(w.records_to_numpy(bufs[k], ran))
    assert any(sum(len(x) for x in g) < 6 * 400 for g in got)   # the budget did stop some
    for k, (dim, L, T, seed) in enumerate(specs):
        rec = np.concatenate(got[k])
        ref, s_ref = oracle_trajectory(dim, L, T, seed, len(rec), s=np.ones(L ** dim, np.int8))
        assert_records_equal(rec, ref, "budgeted tiny lattice %d" % k)
        spins, t = lats[k].get_state()
        assert t == len(rec) and np.array_equal(spins, s_ref)
    # refusals: a team shape, a CTA too small for the largest lattice, a
    # lattice the engine does not take, a Potts lattice
    for cs, th in ((2, 0), (1, 48)):
        with pytest.raises(w.WolffError) as ei:
            batch.run(lats, 1, None, cluster_size=cs, block_threads=th)
        assert ei.value.status == w.WOLFF_EINVAL
    with pytest.raises(w.WolffError) as ei:
        batch.run(lats[:1], 1, None, cluster_size=1, block_threads=32)   # 2D L=96: 288 words
    assert ei.value.status == w.WOLFF_EINVAL
    big = w.WolffLattice(2, 200, TC2, seed=1)
    potts = w.WolffLattice(2, 16, 1.0, seed=1, q=3)
    for other in (big, potts):
        with pytest.raises(w.WolffError) as ei:
            batch.run([lats[0], other], 1, None, cluster_size=1, block_threads=0)
        assert ei.value.status == w.WOLFF_EUNSUPPORTED
    for x in lats + [big, potts]:
        x.close()
    batch.close()


def test_runner_with_tiny_groups_matches_alone():
    torch, w = require_cuda()
    from paper_1110_0899_gb300 import batched
    specs = [dict(dim=d, L=L, T=T, seed=s) for d, L, T, s in BATCH]
    specs += [dict(dim=2, L=256, T=TC2, seed=40), dict(dim=3, L=40, T=4.5115, seed=41)]
    tw, tl, rest = batched.tiny_split(specs, range(len(specs)))
    assert tw and tl and rest == [len(BATCH), len(BATCH) + 1]
    plan = batched.Plan([batched.Group(tw, th=0, kind=batched.TINY),
                         batched.Group(tl, th=0, kind=batched.TINY),
                         batched.Group(rest, 2, 256)], "tiny groups + team")
    lats = [w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"]) for s in specs]
    r = batched.BatchedRunner(lats, plan)
    bufs = r.run(40)
    torch.cuda.synchronize()
    got = r.records_numpy(bufs, 40)
    r.close()
    for i, s in enumerate(specs):
        alone = w.WolffLattice(s["dim"], s["L"], s["T"], seed=s["seed"])
        alone.set_schedule(w.SCHED_CLUSTER)
        assert_records_equal(got[i], alone.step(40), "runner lattice %d vs alone" % i)
        alone.close()
        lats[i].close()
