"""The allocation-free entry point wolff_step_static.

Callers that cannot call cudaMalloc (a framework's caching allocator owns the
memory, a loop that cannot take cudaMalloc's device-wide synchronisation, a
budget fixed at load time) run updates through wolff_step_static, whose
scratch is a static device array.  Its output must equal the context path's
(ising_init + wolff_step) and the oracle's bit for bit, on two calls in a
row: the second call continues the chain from the first call's lattice and
also checks that the shared scratch left behind by the first call does not
leak into the second.  A lattice entry that is not +-1 must be reported
through wolff_step_static_status.
This file is collected last so that a failure here cannot hide others.
"""
import ctypes
import math

import numpy as np
import pytest

from _gpu import assert_records_equal, oracle_trajectory

pytestmark = pytest.mark.gpu

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


def _static_call(lib, torch, w, dim, L, T, seed, t0, n, d_spins, d_rec):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.wolff_step_static(dim, L, 1.0, T, seed, t0, n, ctypes.c_void_p(d_spins.data_ptr()),
                               ctypes.c_void_p(d_rec.data_ptr()), stream)
    assert st == w.WOLFF_OK
    status, detail, t_next = _status(lib, torch, w)
    assert (status, t_next) == (0, t0 + n), detail
    return d_rec.cpu().numpy().view(w.RECORD_DTYPE)[:n].copy(), d_spins.cpu().numpy().copy()


def _status(lib, torch, w):
    status, detail, t_next = ctypes.c_int(-1), ctypes.c_uint32(0), ctypes.c_uint64(0)
    st = lib.wolff_step_static_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      ctypes.byref(status), ctypes.byref(detail),
                                      ctypes.byref(t_next))
    assert st == w.WOLFF_OK
    return status.value, detail.value, t_next.value


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_0899_gb300 as w
    return torch, w, w.load_library()


@pytest.mark.parametrize("dim,L,T,seed", [(2, 64, TC2, 21), (3, 20, 4.5115, 22), (2, 37, 2.0, 23)])
def test_static_entry_matches_context_path_twice(dim, L, T, seed):
    torch, w, lib = _cuda()
    n1, n2 = 150, 120
    ref = w.WolffLattice(dim, L, T, seed=seed)
    start, _ = ref.get_state()
    r1 = ref.step(n1)
    s1, _ = ref.get_state()
    r2 = ref.step(n2)
    s2, _ = ref.get_state()
    ref.close()
    # the oracle's chain from the same start
    o_rec, o_end = oracle_trajectory(dim, L, T, seed, n1 + n2)

    N = L ** dim
    d_spins = torch.zeros((N + 3) // 4 * 4, dtype=torch.int8, device="cuda")
    d_spins[:N] = torch.from_numpy(start).cuda()
    d_rec = torch.zeros(max(n1, n2) * w.RECORD_BYTES, dtype=torch.uint8, device="cuda")
    g1, sp1 = _static_call(lib, torch, w, dim, L, T, seed, 0, n1, d_spins, d_rec)
    g2, sp2 = _static_call(lib, torch, w, dim, L, T, seed, n1, n2, d_spins, d_rec)
    for f in ("C", "levels", "E", "M"):
        assert np.array_equal(g1[f], r1[f]), f
        assert np.array_equal(g2[f], r2[f]), f
    assert_records_equal(np.concatenate([g1, g2]), o_rec, "static vs oracle %dD L=%d" % (dim, L))
    assert np.array_equal(sp1[:N], s1)
    assert np.array_equal(sp2[:N], s2)
    assert np.array_equal(sp2[:N], o_end)


def test_static_entry_reports_an_invalid_entry():
    """A lattice entry that is 0 latches WOLFF_EINVAL on the device: no update
    runs, no record is written, the entry comes back as -1 and every other
    entry is unchanged; the status query reports it and the next valid call
    starts clean."""
    torch, w, lib = _cuda()
    dim, L, T, seed = 2, 48, TC2, 31
    N = L * L
    lat = w.WolffLattice(dim, L, T, seed=seed)
    start = np.array(lat.get_state()[0])
    lat.close()
    bad = start.copy()
    bad[777] = 0
    d_spins = torch.from_numpy(bad).cuda()
    d_rec = torch.full((40 * w.RECORD_BYTES,), 0x5A, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.wolff_step_static(dim, L, 1.0, T, seed, 5, 40, ctypes.c_void_p(d_spins.data_ptr()),
                               ctypes.c_void_p(d_rec.data_ptr()), stream)
    assert st == w.WOLFF_OK   # launched; the device finds the bad entry
    status, detail, t_next = _status(lib, torch, w)
    assert (status, detail, t_next) == (w.WOLFF_EINVAL, 777, 5)
    after = d_spins.cpu().numpy()
    expect = start.copy()
    expect[777] = -1
    assert np.array_equal(after, expect)
    assert (d_rec.cpu().numpy() == 0x5A).all()
    # a valid call afterwards clears the status and runs normally
    d_spins = torch.from_numpy(start).cuda()
    g, sp = _static_call(lib, torch, w, dim, L, T, seed, 0, 40, d_spins, d_rec)
    o_rec, o_end = oracle_trajectory(dim, L, T, seed, 40)
    assert_records_equal(g, o_rec, "static after a rejected lattice")
    assert np.array_equal(sp[:N], o_end)


def test_static_entry_rejects_oversized_lattice():
    torch, w, lib = _cuda()
    big = 1025   # 1025^2 > 2^20 sites
    st = lib.wolff_step_static(2, big, 1.0, TC2, 1, 0, 1, ctypes.c_void_p(256), None, None)
    assert st == w.WOLFF_EINVAL
