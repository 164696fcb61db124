"""CPU oracle for the Wolff single-cluster update (Komura & Okabe, section 2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's timed CPU-baseline leg may import this package.  It shares no code
with the CUDA library: the arithmetic lives in ``wolff_oracle.c`` (Philox,
bond threshold, breadth-first cluster with the ic/in list, flip, observables by
definition, exact enumeration) and in ``kaufman.py`` (the exact partition
function of the periodic square lattice).  This module only marshals arrays.

Every function here is pinned by a CPU test against something other than
itself: Philox against an independent library implementation, the cluster
against a connected-component routine, the observables against closed forms,
the chain against exact enumeration and the exact finite-lattice solution.
"""
import ctypes

import numpy as np

from . import build as _build

RECORD_DTYPE = np.dtype([("C", "<u4"), ("levels", "<u4"),
                         ("E", "<i8"), ("M", "<i8")])

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(_build.build())
    u32, u64, i64, i32 = (ctypes.c_uint32, ctypes.c_uint64,
                          ctypes.c_int64, ctypes.c_int)
    p = ctypes.c_void_p
    lib.orc_philox4x32_10.argtypes = [u32, u32, p, p]
    lib.orc_philox4x32_10.restype = None
    lib.orc_bond_threshold.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_bond_threshold.restype = u64
    lib.orc_init.argtypes = [i32, u32, u64, p]
    lib.orc_init.restype = None
    lib.orc_energy_bond.argtypes = [i32, u32, p]
    lib.orc_energy_bond.restype = i64
    lib.orc_magnetisation.argtypes = [i32, u32, p]
    lib.orc_magnetisation.restype = i64
    lib.orc_seed_site.argtypes = [u64, u64, u32]
    lib.orc_seed_site.restype = u32
    lib.orc_cluster.argtypes = [i32, u32, u64, u64, u64, p, p, p, p]
    lib.orc_cluster.restype = u32
    lib.orc_run.argtypes = [i32, u32, u64, u64, u64, u64, p, p]
    lib.orc_run_local.restype = ctypes.c_int
    lib.orc_run_local.argtypes = [i32, u32, u64, u64, u64, u64, p, p, p]
    lib.orc_run.restype = i32
    lib.orc_enumerate.argtypes = [i32, u32, p]
    lib.orc_enumerate.restype = i32
    lib.orc_potts_init.argtypes = [i32, u32, u32, u64, p]
    lib.orc_potts_init.restype = None
    lib.orc_potts_energy_bond.argtypes = [i32, u32, p]
    lib.orc_potts_energy_bond.restype = i64
    lib.orc_potts_count0.argtypes = [i32, u32, p]
    lib.orc_potts_count0.restype = i64
    lib.orc_potts_cluster.argtypes = [i32, u32, u32, u64, u64, u64, p, p, p, p, p]
    lib.orc_potts_cluster.restype = u32
    lib.orc_potts_run.argtypes = [i32, u32, u32, u64, u64, u64, u64, p, p]
    lib.orc_potts_run.restype = i32
    lib.orc_potts_enumerate.argtypes = [i32, u32, u32, p]
    lib.orc_potts_enumerate.restype = i32
    lib.orc_potts_threshold.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_potts_threshold.restype = u64
    f64 = ctypes.c_double
    lib.orc_xy_table.argtypes = [p]
    lib.orc_xy_table.restype = None
    lib.orc_xy_cos_at.argtypes = [u32]
    lib.orc_xy_cos_at.restype = ctypes.c_int32
    lib.orc_xy_exp_neg.argtypes = [f64]
    lib.orc_xy_exp_neg.restype = f64
    lib.orc_xy_coupling.argtypes = [f64, f64]
    lib.orc_xy_coupling.restype = f64
    lib.orc_xy_threshold.argtypes = [i64, f64]
    lib.orc_xy_threshold.restype = u64
    lib.orc_xy_init.argtypes = [i32, u32, i32, u64, p]
    lib.orc_xy_init.restype = None
    lib.orc_xy_observables.argtypes = [i32, u32, p, p]
    lib.orc_xy_observables.restype = None
    lib.orc_xy_phi.argtypes = [u64, u64, i32]
    lib.orc_xy_phi.restype = u32
    lib.orc_xy_cluster.argtypes = [i32, u32, i32, f64, u64, u64, p, p, p, p, p]
    lib.orc_xy_cluster.restype = u32
    lib.orc_xy_run.argtypes = [i32, u32, i32, f64, u64, u64, u64, p, p]
    lib.orc_xy_run_local.restype = ctypes.c_int
    lib.orc_xy_run_local.argtypes = [i32, u32, i32, f64, u64, u64, u64, p, p]
    lib.orc_xy_run.restype = i32
    _lib = lib
    return lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(key, ctr):
    """Philox4x32-10 of one 2x32-bit key and 4x32-bit counter -> 4 words."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(int(key[0]) & 0xFFFFFFFF,
                              int(key[1]) & 0xFFFFFFFF, _ptr(c), _ptr(out))
    return out


def bond_threshold(J, T):
    """floor(p * 2^32), p = 1 - exp(-2J/T)  (section 2, step (ii))."""
    return int(_load().orc_bond_threshold(float(J), float(T)))


def n_sites(dim, L):
    return int(L) ** int(dim)


def init_lattice(dim, L, seed):
    """Random +-1 start drawn from Philox (tag 2); int8, site i = x + L*y (+L^2 z)."""
    s = np.zeros(n_sites(dim, L), dtype=np.int8)
    _load().orc_init(dim, L, seed, _ptr(s))
    return s


def energy_bond(dim, L, s):
    """E_bond = sum over sites and axes of s_i s_{nb(i,d)}; energy = -J E_bond."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_energy_bond(dim, L, _ptr(s)))


def magnetisation(dim, L, s):
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_magnetisation(dim, L, _ptr(s)))


def seed_site(seed, t, N):
    return int(_load().orc_seed_site(seed, t, N))


def cluster(dim, L, thr, seed, t, s):
    """Cluster of update t on s (s unchanged).

    Returns (member bool array, list of sites in the order added, levels)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    n = n_sites(dim, L)
    member = np.zeros(n, dtype=np.uint8)
    lst = np.zeros(n, dtype=np.uint32)
    levels = np.zeros(1, dtype=np.uint32)
    c = _load().orc_cluster(dim, L, thr, seed, t, _ptr(s), _ptr(member),
                            _ptr(lst), _ptr(levels))
    return member.astype(bool), lst[:c].copy(), int(levels[0])


def run(dim, L, thr, seed, t0, n, s, records=True):
    """Updates t0..t0+n-1 applied to s (int8, modified in place).

    Returns a structured array of RECORD_DTYPE (|C|, levels, E_bond, M after
    each update), or None when records is False."""
    if s.dtype != np.int8 or not s.flags.c_contiguous:
        raise ValueError("s must be a contiguous int8 array")
    rec = np.zeros(int(n), dtype=RECORD_DTYPE) if records else None
    rc = _load().orc_run(dim, L, thr, seed, t0, n, _ptr(s),
                         _ptr(rec) if rec is not None else None)
    if rc != 0:
        raise MemoryError("oracle could not allocate its scratch arrays")
    return rec


def run_local(dim, L, thr, seed, t0, n, s, em=None):
    """The updates of run() with every record, E_bond and M kept by a local
    recount of the terms each flip changes (O(|C|) per update instead of
    O(N)): the same records as run(), fast enough for whole runs of the
    2^24-site lattices.  em: optional int64 array [E_bond, M] of s on entry
    (else counted from the definitions), updated to the final lattice's."""
    if s.dtype != np.int8 or not s.flags.c_contiguous:
        raise ValueError("s must be a contiguous int8 array")
    if em is not None and (em.dtype != np.int64 or em.size != 2):
        raise ValueError("em must be an int64 array of two entries")
    rec = np.zeros(int(n), dtype=RECORD_DTYPE)
    if _load().orc_run_local(dim, L, thr, seed, t0, n, _ptr(s),
                             _ptr(em) if em is not None else None, _ptr(rec)) != 0:
        raise MemoryError("oracle could not allocate its scratch arrays")
    return rec


def density_of_states(dim, L):
    """g(E_bond, M) by enumerating all 2^N states (N <= 32).

    Returns (g, E values, M values) with g[e_index, m_index] counts."""
    n = n_sites(dim, L)
    width = 2 * n + 1
    hist = np.zeros((2 * dim * n + 1) * width, dtype=np.uint64)
    if _load().orc_enumerate(dim, L, _ptr(hist)) != 0:
        raise ValueError("enumeration needs N <= 32")
    g = hist.reshape(2 * dim * n + 1, width)
    E = np.arange(-dim * n, dim * n + 1)
    M = np.arange(-n, n + 1)
    return g, E, M


def exact_moments(dim, L, J, T, g=None):
    """Boltzmann averages from the enumerated density of states.

    Returns a dict with <E_bond>, <E_bond^2>, <M^2>, <|M|>, <M^4> and the
    normalised joint distribution P(E_bond, M)."""
    if g is None:
        g, E, M = density_of_states(dim, L)
    else:
        n = n_sites(dim, L)
        E = np.arange(-dim * n, dim * n + 1)
        M = np.arange(-n, n + 1)
    K = float(J) / float(T)
    gf = g.astype(np.float64)
    occupied = gf > 0
    logw = np.full(gf.shape, -np.inf)
    logw[occupied] = np.log(gf[occupied]) + K * E[:, None].repeat(
        gf.shape[1], 1)[occupied]
    logw -= logw[occupied].max()
    w = np.exp(logw)
    P = w / w.sum()
    pe = P.sum(axis=1)
    pm = P.sum(axis=0)
    Ef = E.astype(np.float64)
    Mf = M.astype(np.float64)
    return {
        "E": float((pe * Ef).sum()),
        "E2": float((pe * Ef ** 2).sum()),
        "M2": float((pm * Mf ** 2).sum()),
        "absM": float((pm * np.abs(Mf)).sum()),
        "M4": float((pm * Mf ** 4).sum()),
        "P": P, "E_values": E, "M_values": M,
    }


# ---- q-state Potts (section 6 names it as the straightforward extension) ----

def potts_threshold(J, T):
    """floor(p * 2^32), p = 1 - exp(-J/T) (Potts bond probability)."""
    return int(_load().orc_potts_threshold(float(J), float(T)))


def potts_init(dim, L, q, seed):
    c = np.zeros(n_sites(dim, L), dtype=np.int8)
    _load().orc_potts_init(dim, L, q, seed, _ptr(c))
    return c


def potts_energy_bond(dim, L, c):
    c = np.ascontiguousarray(c, dtype=np.int8)
    return int(_load().orc_potts_energy_bond(dim, L, _ptr(c)))


def potts_count0(dim, L, c):
    c = np.ascontiguousarray(c, dtype=np.int8)
    return int(_load().orc_potts_count0(dim, L, _ptr(c)))


def potts_cluster(dim, L, q, thr, seed, t, c):
    """(member bool array, list, levels, new colour) of Potts update t on c."""
    c = np.ascontiguousarray(c, dtype=np.int8)
    n = n_sites(dim, L)
    member = np.zeros(n, dtype=np.uint8)
    lst = np.zeros(n, dtype=np.uint32)
    levels = np.zeros(1, dtype=np.uint32)
    nc = np.zeros(1, dtype=np.int32)
    k = _load().orc_potts_cluster(dim, L, q, thr, seed, t, _ptr(c), _ptr(member), _ptr(lst),
                                  _ptr(levels), _ptr(nc))
    return member.astype(bool), lst[:k].copy(), int(levels[0]), int(nc[0])


def potts_run(dim, L, q, thr, seed, t0, n, c, records=True):
    """Potts updates t0..t0+n-1 on c (int8 colours, in place); records hold
    |C|, levels, E_bond (satisfied bonds) and N0 (in the M field)."""
    if c.dtype != np.int8 or not c.flags.c_contiguous:
        raise ValueError("c must be a contiguous int8 array")
    rec = np.zeros(int(n), dtype=RECORD_DTYPE) if records else None
    rc = _load().orc_potts_run(dim, L, q, thr, seed, t0, n, _ptr(c),
                               _ptr(rec) if rec is not None else None)
    if rc != 0:
        raise MemoryError("oracle could not allocate its scratch arrays (or q < 2)")
    return rec


def potts_density_of_states(dim, L, q):
    """g(E_bond, N0) over all q^N colourings.  Returns (g, E values, N0 values)."""
    n = n_sites(dim, L)
    hist = np.zeros((dim * n + 1) * (n + 1), dtype=np.uint64)
    if _load().orc_potts_enumerate(dim, L, q, _ptr(hist)) != 0:
        raise ValueError("too many states to enumerate")
    return hist.reshape(dim * n + 1, n + 1), np.arange(dim * n + 1), np.arange(n + 1)


def potts_exact_moments(dim, L, q, J, T, g=None):
    """Boltzmann averages <E_bond>, <N0>, <N0^2> from the enumeration."""
    if g is None:
        g, E, Z0 = potts_density_of_states(dim, L, q)
    else:
        n = n_sites(dim, L)
        E, Z0 = np.arange(dim * n + 1), np.arange(n + 1)
    K = float(J) / float(T)
    gf = g.astype(np.float64)
    occ = gf > 0
    logw = np.full(gf.shape, -np.inf)
    logw[occ] = np.log(gf[occ]) + (K * E[:, None].repeat(gf.shape[1], 1))[occ]
    logw -= logw[occ].max()
    w = np.exp(logw)
    P = w / w.sum()
    pe, pz = P.sum(axis=1), P.sum(axis=0)
    Ef, Zf = E.astype(np.float64), Z0.astype(np.float64)
    return {"E": float((pe * Ef).sum()), "N0": float((pz * Zf).sum()),
            "N0_2": float((pz * Zf ** 2).sum()), "P": P}



# ---- XY model (embedded-cluster Wolff update, the extension section 6 names) ----

XY_RECORD_DTYPE = np.dtype([("C", "<u4"), ("levels", "<u4"), ("E", "<i8"),
                            ("Mx", "<i8"), ("My", "<i8")])
XY_ONE = 1 << 30          # fixed-point unit of the cosine table
XY_ANGLE_BITS = 15        # production angle resolution (units of 2 pi / 65536)


def xy_table():
    """I[k] = round(cos(pi k / 32768) 2^30), k = 0..16384."""
    t = np.zeros(16385, dtype=np.int32)
    _load().orc_xy_table(_ptr(t))
    return t


def xy_cos(a):
    """Fixed-point cos of angle a (units of 2 pi / 65536)."""
    return int(_load().orc_xy_cos_at(int(a) & 0xFFFF))


def xy_exp_neg(y):
    return float(_load().orc_xy_exp_neg(float(y)))


def xy_coupling(J, T):
    """2 J / T * 2^-60: y = coupling * (product of two fixed-point projections)."""
    return float(_load().orc_xy_coupling(float(J), float(T)))


def xy_threshold(prod, kk):
    """floor(2^32 (1 - exp(-kk prod))) for prod > 0, else 0."""
    return int(_load().orc_xy_threshold(int(prod), float(kk)))


def xy_init(dim, L, bits, seed):
    th = np.zeros(n_sites(dim, L), dtype=np.uint16)
    _load().orc_xy_init(dim, L, bits, seed, _ptr(th))
    return th


def xy_observables(dim, L, theta):
    """(E_fix, Mx, My) by their definitions."""
    theta = np.ascontiguousarray(theta, dtype=np.uint16)
    out = np.zeros(3, dtype=np.int64)
    _load().orc_xy_observables(dim, L, _ptr(theta), _ptr(out))
    return int(out[0]), int(out[1]), int(out[2])


def xy_phi(seed, t, bits):
    return int(_load().orc_xy_phi(seed, t, bits))


def xy_cluster(dim, L, bits, kk, seed, t, theta):
    """(member bool array, list, levels, phi) of XY update t on theta."""
    theta = np.ascontiguousarray(theta, dtype=np.uint16)
    n = n_sites(dim, L)
    member = np.zeros(n, dtype=np.uint8)
    lst = np.zeros(n, dtype=np.uint32)
    levels = np.zeros(1, dtype=np.uint32)
    phi = np.zeros(1, dtype=np.uint32)
    k = _load().orc_xy_cluster(dim, L, bits, kk, seed, t, _ptr(theta), _ptr(member), _ptr(lst),
                               _ptr(levels), _ptr(phi))
    return member.astype(bool), lst[:k].copy(), int(levels[0]), int(phi[0])


def xy_run(dim, L, bits, kk, seed, t0, n, theta, records=True):
    """XY updates t0..t0+n-1 on theta (uint16 angles, in place)."""
    if theta.dtype != np.uint16 or not theta.flags.c_contiguous:
        raise ValueError("theta must be a contiguous uint16 array")
    rec = np.zeros(int(n), dtype=XY_RECORD_DTYPE) if records else None
    rc = _load().orc_xy_run(dim, L, bits, kk, seed, t0, n, _ptr(theta),
                            _ptr(rec) if rec is not None else None)
    if rc != 0:
        raise MemoryError("oracle could not allocate its scratch arrays (or bad angle bits)")
    return rec


def xy_run_local(dim, L, bits, kk, seed, t0, n, theta):
    """The XY updates of xy_run() with every record kept by a local recount."""
    if theta.dtype != np.uint16 or not theta.flags.c_contiguous:
        raise ValueError("theta must be a contiguous uint16 array")
    rec = np.zeros(int(n), dtype=XY_RECORD_DTYPE)
    if _load().orc_xy_run_local(dim, L, bits, kk, seed, t0, n, _ptr(theta), _ptr(rec)) != 0:
        raise MemoryError("oracle could not allocate its scratch arrays (or bad angle bits)")
    return rec
