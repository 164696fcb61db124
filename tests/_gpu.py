"""Shared helpers of the GPU tests."""
import numpy as np
import pytest

import oracle


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_0899_gb300 as w
    w.load_library()
    return torch, w


def oracle_trajectory(dim, L, T, seed, n, t0=0, s=None, J=1.0):
    thr = oracle.bond_threshold(J, T)
    if s is None:
        s = oracle.init_lattice(dim, L, seed)
    else:
        s = np.array(s, dtype=np.int8, copy=True)
    rec = oracle.run(dim, L, thr, seed, t0, n, s)
    return rec, s


def assert_records_equal(got, ref, label=""):
    for f in ("C", "levels", "E", "M"):
        if not np.array_equal(got[f], ref[f]):
            bad = int(np.nonzero(got[f] != ref[f])[0][0])
            raise AssertionError("%s: field %s first differs at update %d: gpu %r oracle %r"
                                 % (label, f, bad, got[bad], ref[bad]))
