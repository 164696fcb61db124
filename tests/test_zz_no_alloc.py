"""The allocation-free entry point wolff_step_static.

Callers that cannot call cudaMalloc (a framework's caching allocator owns the
memory, a loop that cannot take cudaMalloc's device-wide synchronisation, a
budget fixed at load time) run updates through wolff_step_static, whose
scratch is a static device array.  Its output must equal the context path's
(ising_init + wolff_step) bit for bit, on two calls in a row: the second call
continues the chain from the first call's lattice and also checks that the
shared scratch left behind by the first call does not leak into the second.
This file is collected last so that a failure here cannot hide others.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))


def _static_call(lib, torch, w, dim, L, T, seed, t0, n, d_spins, d_rec):
    lib.wolff_step_static.restype = ctypes.c_int
    lib.wolff_step_static.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
    st = lib.wolff_step_static(dim, L, 1.0, T, seed, t0, n, ctypes.c_void_p(d_spins.data_ptr()),
                               ctypes.c_void_p(d_rec.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == w.WOLFF_OK
    torch.cuda.synchronize()
    return d_rec.cpu().numpy().view(w.RECORD_DTYPE)[:n].copy(), d_spins.cpu().numpy().copy()


@pytest.mark.parametrize("dim,L,T,seed", [(2, 64, TC2, 21), (3, 20, 4.5115, 22), (2, 37, 2.0, 23)])
def test_static_entry_matches_context_path_twice(dim, L, T, seed):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_0899_gb300 as w
    lib = w.load_library()
    n1, n2 = 150, 120
    ref = w.WolffLattice(dim, L, T, seed=seed)
    start, _ = ref.get_state()
    r1 = ref.step(n1)
    s1, _ = ref.get_state()
    r2 = ref.step(n2)
    s2, _ = ref.get_state()
    ref.close()

    N = L ** dim
    d_spins = torch.zeros((N + 3) // 4 * 4, dtype=torch.int8, device="cuda")
    d_spins[:N] = torch.from_numpy(start).cuda()
    d_rec = torch.zeros(max(n1, n2) * w.RECORD_BYTES, dtype=torch.uint8, device="cuda")
    g1, sp1 = _static_call(lib, torch, w, dim, L, T, seed, 0, n1, d_spins, d_rec)
    g2, sp2 = _static_call(lib, torch, w, dim, L, T, seed, n1, n2, d_spins, d_rec)
    for f in ("C", "levels", "E", "M"):
        assert np.array_equal(g1[f], r1[f]), f
        assert np.array_equal(g2[f], r2[f]), f
    assert np.array_equal(sp1[:N], s1)
    assert np.array_equal(sp2[:N], s2)


def test_static_entry_rejects_oversized_lattice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_0899_gb300 as w
    lib = w.load_library()
    lib.wolff_step_static.restype = ctypes.c_int
    big = 1025   # 1025^2 > 2^20 sites
    st = lib.wolff_step_static(2, big, ctypes.c_double(1.0), ctypes.c_double(TC2),
                               ctypes.c_uint64(1), ctypes.c_uint64(0), ctypes.c_uint64(1),
                               ctypes.c_void_p(256), None, None)
    assert st == w.WOLFF_EINVAL
