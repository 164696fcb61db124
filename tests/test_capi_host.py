"""CPU checks of the C ABI library: it loads, exports every declared entry
point, and its host logic (bond threshold, workspace sizes, argument
validation) agrees with the oracle and the header -- no GPU call is made."""
import ctypes
import math
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_0899_gb300 import build
    build.build()
    import paper_1110_0899_gb300 as w
    return w.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "wolff.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[a-z_][a-z0-9_ \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "return")))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ising_init" in names and "wolff_step" in names and "measure" in names
    for n in names:
        assert hasattr(lib, n), n


def test_threshold_matches_oracle(lib):
    import paper_1110_0899_gb300 as w
    for J in (0.0, 0.5, 1.0, 2.0):
        for T in (1e-3, 0.5, 1.0, w.TC_2D, 3.0, w.TC_3D, 100.0, float("inf")):
            assert w.wolff_bond_threshold(J, T) == oracle.bond_threshold(J, T), (J, T)
    assert w.wolff_bond_threshold(1.0, w.TC_2D) == 2**33 - math.isqrt(2**65) - 1


def test_workspace_bytes(lib):
    import paper_1110_0899_gb300 as w
    n = 4096 * 4096
    ring = 4096 * 1024   # pre-grown updates, lattices of 2^20 sites or more
    b = w.wolff_workspace_bytes(2, 4096)
    assert b >= n + 4 * n + ring and b <= n + 4 * n + ring + 4096
    assert w.wolff_workspace_bytes(3, 256) == w.wolff_workspace_bytes(2, 4096)
    small = 1023 * 1023
    b = w.wolff_workspace_bytes(2, 1023)
    assert small + 4 * small <= b <= small + 4 * small + 4096
    b = w.wolff_workspace_bytes(2, 1024)
    assert b >= 1024 * 1024 * 5 + ring
    for dim, L in ((1, 10), (4, 2), (2, 1), (2, 0), (3, 1025), (2, 40000)):
        assert w.wolff_workspace_bytes(dim, L) == 0
    assert w.wolff_workspace_bytes(2, 16, 7) == 0


def test_init_rejects_bad_arguments_before_touching_the_device(lib):
    import paper_1110_0899_gb300 as w
    h = ctypes.c_void_p()
    bad = [(4, 16, 1.0, 2.0), (2, 1, 1.0, 2.0), (3, 2000, 1.0, 2.0),
           (2, 16, -1.0, 2.0), (2, 16, 1.0, 0.0), (2, 16, 1.0, -1.0),
           (2, 16, float("nan"), 2.0)]
    for dim, L, J, T in bad:
        st = lib.ising_init(ctypes.byref(h), dim, L, J, T, 1, 0, None, 0, None)
        assert st == w.WOLFF_EINVAL, (dim, L, J, T)
    assert lib.ising_init(None, 2, 16, 1.0, 2.0, 1, 0, None, 0, None) == w.WOLFF_EINVAL
    # a caller workspace that is too small or misaligned
    st = lib.ising_init(ctypes.byref(h), 2, 16, 1.0, 2.0, 1, 0, ctypes.c_void_p(256), 16, None)
    assert st == w.WOLFF_ENOMEM
    st = lib.ising_init(ctypes.byref(h), 2, 16, 1.0, 2.0, 1, 0, ctypes.c_void_p(4096 + 8),
                        1 << 20, None)
    assert st == w.WOLFF_EINVAL
    assert lib.wolff_step(None, 1, None) == w.WOLFF_EINVAL
    assert lib.measure(None, None, None, None) == w.WOLFF_EINVAL
    assert lib.wolff_status_string(4) == b"WOLFF_ETIMEOUT"
    assert lib.wolff_last_error(None) == b""


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1110_0899_gb300 as w
    monkeypatch.setattr(w._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(w, "_lib", None)
    with pytest.raises(ImportError):
        w.load_library()


def test_xy_workspace_and_argument_checks(lib):
    import paper_1110_0899_gb300 as w
    n = 1024 * 1024
    b = lib.wolff_xy_workspace_bytes(2, 1024)
    # two 32-bit arrays (site words, cluster list), the cosine table, 1/n!
    assert 8 * n + 16385 * 4 <= b <= 8 * n + 16385 * 4 + 8192
    assert lib.wolff_xy_workspace_bytes(2, 1) == 0 and lib.wolff_xy_workspace_bytes(4, 8) == 0
    h = ctypes.c_void_p()
    for bits in (0, 16, -1):
        assert lib.xy_init(ctypes.byref(h), 2, 16, bits, 1.0, 1.0, 1, None, 0, None) == w.WOLFF_EINVAL
    for dim, L, J, T in [(4, 16, 1.0, 1.0), (2, 1, 1.0, 1.0), (2, 16, 1.0, 0.0), (2, 16, -1.0, 1.0)]:
        assert lib.xy_init(ctypes.byref(h), dim, L, 15, J, T, 1, None, 0, None) == w.WOLFF_EINVAL
    assert lib.xy_init(None, 2, 16, 15, 1.0, 1.0, 1, None, 0, None) == w.WOLFF_EINVAL
    assert lib.xy_measure(None, None, None, None, None) == w.WOLFF_EINVAL
    assert lib.xy_measure_full(None, None, None, None) == w.WOLFF_EINVAL
    assert lib.xy_get_state(None, None, None) == w.WOLFF_EINVAL
    assert lib.xy_set_state(None, None, 0) == w.WOLFF_EINVAL
    assert w.XY_RECORD_DTYPE.itemsize == 32 and w.XY_RECORD_DTYPE == oracle.XY_RECORD_DTYPE


def test_bit_packing_definition(lib):
    """Bit (i mod 32) of word i / 32 is set when site i is +1; unused high
    bits of the last word are zero; unpacking inverts packing."""
    import numpy as np
    import paper_1110_0899_gb300 as w
    rng = np.random.default_rng(4)
    for N in (1, 31, 32, 33, 1331, 4096):
        s = rng.choice(np.array([-1, 1], np.int8), N)
        b = w.pack_spins(s)
        assert b.dtype == np.uint32 and b.size == (N + 31) // 32
        for i in rng.integers(0, N, 50):
            assert ((int(b[i // 32]) >> (i % 32)) & 1) == int(s[i] == 1)
        if N % 32:
            assert int(b[-1]) >> (N % 32) == 0
        assert np.array_equal(w.unpack_bits(b, N), s)


def test_static_entry_checks_before_touching_the_device(lib):
    """wolff_step_static rejects a lattice pointer that is not 16-byte aligned
    (its recount reads 16-byte vectors), a misaligned record buffer, a bad
    shape and an oversized lattice, all on the host: none of these pointers
    is ever dereferenced, and no CUDA call is made."""
    import paper_1110_0899_gb300 as w
    tc = w.TC_2D
    base = 1 << 20   # a stand-in address, never dereferenced
    for off in (4, 8, 12, 1):
        assert lib.wolff_step_static(2, 64, 1.0, tc, 1, 0, 1, ctypes.c_void_p(base + off),
                                     None, None) == w.WOLFF_EINVAL, off
    assert lib.wolff_step_static(2, 64, 1.0, tc, 1, 0, 1, ctypes.c_void_p(base),
                                 ctypes.c_void_p(base + 4), None) == w.WOLFF_EINVAL
    for dim, L in ((2, 1), (4, 8), (3, 1025), (2, 1025), (3, 102)):
        assert lib.wolff_step_static(dim, L, 1.0, tc, 1, 0, 1, ctypes.c_void_p(base),
                                     None, None) == w.WOLFF_EINVAL, (dim, L)
    assert lib.wolff_step_static(2, 64, 1.0, 0.0, 1, 0, 1, ctypes.c_void_p(base),
                                 None, None) == w.WOLFF_EINVAL
    assert lib.wolff_step_static(2, 64, 1.0, tc, 1, 0, 1, None, None, None) == w.WOLFF_EINVAL
