"""GB300 Wolff single-cluster library: Python binding of ``include/wolff.h``.

Argument marshalling only.  Every step of an update runs in the CUDA kernels
of ``_build/libwolff.so``; PyTorch provides device memory and the stream.  The
library must be built first (``python -m paper_1110_0899_gb300.build`` or
``__graft_entry__.build()``); importing the binding without it raises.

Names follow the C ABI: ``ising_init``, ``wolff_step``, ``measure``,
``measure_full``, ``wolff_get_state``, ``wolff_set_state``, ``wolff_run_host``,
``ising_free``; :class:`WolffLattice` wraps a context for convenience.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

WOLFF_OK, WOLFF_EINVAL, WOLFF_ENOMEM, WOLFF_ECUDA, WOLFF_ETIMEOUT, WOLFF_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "WOLFF_OK", 1: "WOLFF_EINVAL", 2: "WOLFF_ENOMEM", 3: "WOLFF_ECUDA",
                4: "WOLFF_ETIMEOUT", 5: "WOLFF_EUNSUPPORTED"}
LAYOUT_INT8 = 0
SCHED_AUTO, SCHED_PERSISTENT, SCHED_GRAPH, SCHED_CLUSTER, SCHED_TINY = 0, 1, 2, 3, 4
TINY_MAX_SITES = 32768     # WOLFF_TINY_MAX_SITES

RECORD_DTYPE = np.dtype([("C", "<u4"), ("levels", "<u4"), ("E", "<i8"), ("M", "<i8")])
RECORD_BYTES = RECORD_DTYPE.itemsize  # 24
# XY model records: |C|, levels and the fixed-point E, Mx, My (units 2^-30)
XY_RECORD_DTYPE = np.dtype([("C", "<u4"), ("levels", "<u4"), ("E", "<i8"),
                            ("Mx", "<i8"), ("My", "<i8")])
XY_RECORD_BYTES = XY_RECORD_DTYPE.itemsize  # 32
XY_ANGLE_BITS = 15
XY_ONE = 1 << 30

TC_2D = 2.0 / math.log(1.0 + math.sqrt(2.0))   # Onsager: T_c/J = 2.2691...
TC_3D = 4.5115                                  # simple cubic, J = 1


class WolffError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s%s" % (STATUS_NAMES.get(status, str(status)),
                                   (": " + msg) if msg else ""))


class _Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("L", ctypes.c_int), ("N", ctypes.c_uint32),
                ("thr", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("t", ctypes.c_uint64),
                ("schedule", ctypes.c_int), ("grid_blocks", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("sm_count", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("helper_clusters", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("updates", "levels_local", "levels_grid", "ns_local", "ns_grid", "ns_finish",
                 "handoffs", "grid_finishes", "start_ns", "end_ns", "burst_updates", "bursts",
                 "ns_win_grow", "ns_win_map", "ns_win_check", "ns_win_commit", "win_levels",
                 "pregrown", "ns_win_first_grow", "win_regrown", "win_fresh_grown")]


_lib = None


def library_path():
    return _build.LIB


def load_library():
    """Loads ``libwolff.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libwolff.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    v, i, u32, u64, i64, d, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_size_t)
    P = ctypes.POINTER
    sigs = {
        "wolff_workspace_bytes": (sz, [i, i, i]),
        "ising_init": (i, [P(v), i, i, d, d, u64, i, v, sz, v]),
        "potts_init": (i, [P(v), i, i, i, d, d, u64, v, sz, v]),
        "wolff_xy_workspace_bytes": (sz, [i, i]),
        "xy_init": (i, [P(v), i, i, i, d, d, u64, v, sz, v]),
        "xy_measure": (i, [v, P(i64), P(i64), P(i64), P(u64)]),
        "xy_measure_full": (i, [v, P(i64), P(i64), P(i64)]),
        "xy_get_state": (i, [v, v, P(u64)]),
        "xy_set_state": (i, [v, v, u64]),
        "wolff_step": (i, [v, u64, v]),
        "wolff_run_host": (i, [v, v, u64, u64, v, v]),
        "measure": (i, [v, P(i64), P(i64), P(u64)]),
        "measure_full": (i, [v, P(i64), P(i64)]),
        "wolff_get_state": (i, [v, v, P(u64)]),
        "wolff_set_state": (i, [v, v, u64]),
        "wolff_get_state_bits": (i, [v, v, P(u64)]),
        "wolff_set_state_bits": (i, [v, v, u64]),
        "wolff_run_host_bits": (i, [v, v, u64, u64, v, v]),
        "wolff_set_schedule": (i, [v, i, i, i]),
        "wolff_get_info": (i, [v, P(_Info)]),
        "wolff_set_local_thresholds": (i, [v, u32, u32]),
        "wolff_get_stats": (i, [v, P(_Stats)]),
        "wolff_set_burst": (i, [v, i]),
        "wolff_set_helpers": (i, [v, i]),
        "wolff_batch_create": (i, [P(v), i, v]),
        "wolff_batch_run": (i, [v, v, i, v, v, i, i]),
        "wolff_batch_run_timed": (i, [v, v, i, v, v, i, i, u64]),
        "wolff_batch_free": (i, [v]),
        "wolff_batch_set_window": (i, [v, i]),
        "wolff_batch_set_schedule": (i, [v, i]),
        "wolff_step_static": (i, [i, i, d, d, u64, u64, u64, v, v, v]),
        "wolff_step_static_status": (i, [v, P(i), P(u32), P(u64)]),
        "wolff_l2_probe": (i, [v, sz, i, i, v, v]),
        "wolff_bond_threshold": (u64, [d, d]),
        "wolff_philox": (i, [u32, u32, v, v, u64, v]),
        "wolff_selftest_wait_timeout": (i, [v, u64, P(i)]),
        "ising_free": (i, [v]),
        "wolff_last_error": (ctypes.c_char_p, [v]),
        "wolff_status_string": (ctypes.c_char_p, [i]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != WOLFF_OK:
        msg = ""
        if ctx is not None:
            msg = load_library().wolff_last_error(ctx).decode(errors="replace")
        raise WolffError(status, msg)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---- functions with the C names ---------------------------------------------

def wolff_workspace_bytes(dim, L, layout=LAYOUT_INT8):
    return int(load_library().wolff_workspace_bytes(dim, L, layout))


def wolff_bond_threshold(J, T):
    return int(load_library().wolff_bond_threshold(float(J), float(T)))


def ising_init(dim, L, J, T, seed, layout=LAYOUT_INT8, workspace=None, stream=None):
    """Creates a context; returns (handle, workspace tensor).  The workspace is
    a torch uint8 CUDA tensor that must outlive the handle."""
    torch = _torch()
    lib = load_library()
    nbytes = lib.wolff_workspace_bytes(dim, L, layout)
    if nbytes == 0:
        raise WolffError(WOLFF_EINVAL, "invalid lattice shape dim=%r L=%r" % (dim, L))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    handle = ctypes.c_void_p()
    st = lib.ising_init(ctypes.byref(handle), int(dim), int(L), float(J), float(T),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, int(layout),
                        ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                        _stream_handle(stream))
    _check(st)
    return handle, workspace


def potts_init(dim, L, q, J, T, seed, workspace=None, stream=None):
    """Creates a q-state Potts context; returns (handle, workspace tensor)."""
    torch = _torch()
    lib = load_library()
    nbytes = lib.wolff_workspace_bytes(dim, L, LAYOUT_INT8)
    if nbytes == 0:
        raise WolffError(WOLFF_EINVAL, "invalid lattice shape dim=%r L=%r" % (dim, L))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    handle = ctypes.c_void_p()
    st = lib.potts_init(ctypes.byref(handle), int(dim), int(L), int(q), float(J), float(T),
                        int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.c_void_p(workspace.data_ptr()),
                        workspace.numel(), _stream_handle(stream))
    _check(st)
    return handle, workspace


def wolff_step(handle, n_updates, d_records=None):
    """Enqueues n_updates updates; d_records: torch uint8 CUDA tensor of
    n_updates * 24 bytes (or None)."""
    ptr = ctypes.c_void_p(d_records.data_ptr()) if d_records is not None else None
    _check(load_library().wolff_step(handle, int(n_updates), ptr), handle)


def measure(handle):
    E, M, C = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
    _check(load_library().measure(handle, ctypes.byref(E), ctypes.byref(M), ctypes.byref(C)),
           handle)
    return E.value, M.value, C.value


def measure_full(handle):
    E, M = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().measure_full(handle, ctypes.byref(E), ctypes.byref(M)), handle)
    return E.value, M.value


def wolff_get_state(handle, N):
    s = np.empty(N, dtype=np.int8)
    t = ctypes.c_uint64()
    _check(load_library().wolff_get_state(handle, ctypes.c_void_p(s.ctypes.data),
                                          ctypes.byref(t)), handle)
    return s, t.value


def wolff_set_state(handle, spins, t):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(load_library().wolff_set_state(handle, ctypes.c_void_p(s.ctypes.data), int(t)),
           handle)


def wolff_run_host(handle, N, n_updates, spins_in=None, t_in=0, records=True, spins_out=True,
                   rec_out=None):
    """Host-buffer path: optional upload, n updates, records and lattice back.
    rec_out: optional host array of RECORD_DTYPE (e.g. in pinned memory) that
    receives the records."""
    sin = None if spins_in is None else np.ascontiguousarray(spins_in, dtype=np.int8)
    if records:
        rec = rec_out if rec_out is not None else np.zeros(int(n_updates), dtype=RECORD_DTYPE)
    else:
        rec = None
    sout = np.empty(N, dtype=np.int8) if spins_out else None
    ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    _check(load_library().wolff_run_host(handle, ptr(sin), int(t_in), int(n_updates), ptr(rec),
                                         ptr(sout)), handle)
    return rec, sout


def pack_spins(spins):
    """int8 +-1 lattice -> bit-packed uint32 words (bit i of word i/32 = +1)."""
    b = np.packbits(np.asarray(spins) == 1, bitorder="little")
    words = (len(spins) + 31) // 32
    out = np.zeros(words * 4, dtype=np.uint8)
    out[: len(b)] = b
    return out.view(np.uint32)


def unpack_bits(bits, N):
    """Bit-packed uint32 words -> int8 +-1 lattice of N sites."""
    b = np.unpackbits(np.asarray(bits, dtype=np.uint32).view(np.uint8), bitorder="little")[:N]
    return (2 * b.astype(np.int8) - 1).astype(np.int8)


def ising_free(handle):
    _check(load_library().ising_free(handle))


def wolff_philox(key0, key1, d_ctr, d_out, n, stream=None):
    _check(load_library().wolff_philox(key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF,
                                       ctypes.c_void_p(d_ctr.data_ptr()),
                                       ctypes.c_void_p(d_out.data_ptr()), int(n),
                                       _stream_handle(stream)))


def wolff_l2_probe(d_buf, passes, mode=0, d_sink=None, stream=None):
    """Enqueues the L2 bandwidth probe over the torch CUDA tensor d_buf (its
    whole storage, a multiple of 16 bytes) `passes` times; mode 0 reads, 1
    reads and writes back.  d_sink: a CUDA tensor of at least 4 bytes (made
    here if None; keep it alive until the launch has run)."""
    torch = _torch()
    if d_sink is None:
        d_sink = torch.zeros(1, dtype=torch.int32, device=d_buf.device)
    nbytes = d_buf.numel() * d_buf.element_size()
    _check(load_library().wolff_l2_probe(ctypes.c_void_p(d_buf.data_ptr()), nbytes, int(passes),
                                         int(mode), ctypes.c_void_p(d_sink.data_ptr()),
                                         _stream_handle(stream)))
    return d_sink


def records_to_numpy(d_records, n):
    """Device record buffer -> numpy structured array (synchronises)."""
    host = d_records[: n * RECORD_BYTES].cpu().numpy()
    return host.view(RECORD_DTYPE).copy()


class WolffLattice:
    """One Ising lattice (or, with q, a q-state Potts lattice) and its Wolff
    chain on the current CUDA device."""

    def __init__(self, dim, L, T, J=1.0, seed=0, layout=LAYOUT_INT8, schedule=None,
                 grid_blocks=0, block_threads=0, stream=None, q=None):
        self.dim, self.L, self.J, self.T, self.seed = int(dim), int(L), float(J), float(T), int(seed)
        self.N = self.L ** self.dim
        self.q = q
        # the CUDA stream the context enqueues on (its handle value)
        self.stream = _stream_handle(stream).value
        if q is None:
            self.handle, self.workspace = ising_init(dim, L, J, T, seed, layout, stream=stream)
        else:
            self.handle, self.workspace = potts_init(dim, L, q, J, T, seed, stream=stream)
        self._records = None
        if schedule is not None or grid_blocks or block_threads:
            self.set_schedule(schedule or SCHED_AUTO, grid_blocks, block_threads)

    def set_schedule(self, schedule=SCHED_AUTO, grid_blocks=0, block_threads=0):
        _check(load_library().wolff_set_schedule(self.handle, int(schedule), int(grid_blocks),
                                                 int(block_threads)), self.handle)

    def set_local_thresholds(self, t_up, t_down):
        _check(load_library().wolff_set_local_thresholds(self.handle, int(t_up), int(t_down)),
               self.handle)

    def info(self):
        inf = _Info()
        _check(load_library().wolff_get_info(self.handle, ctypes.byref(inf)), self.handle)
        return {k: getattr(inf, k) for k, _ in _Info._fields_}

    def set_burst(self, enable):
        """Window mode: False/0 off, True/1 on, k >= 2 on with k growth levels
        per commit round."""
        level = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        _check(load_library().wolff_set_burst(self.handle, level), self.handle)

    def set_helpers(self, max_helpers):
        """Helper teams of the cluster schedule: -1 = as many as fit (the
        default), 0 = none, k > 0 = at most k."""
        _check(load_library().wolff_set_helpers(self.handle, int(max_helpers)), self.handle)

    def stats(self):
        st = _Stats()
        _check(load_library().wolff_get_stats(self.handle, ctypes.byref(st)), self.handle)
        return {k: int(getattr(st, k)) for k, _ in _Stats._fields_}

    def record_buffer(self, n):
        torch = _torch()
        need = int(n) * RECORD_BYTES
        if self._records is None or self._records.numel() < need:
            self._records = torch.empty(max(need, RECORD_BYTES), dtype=torch.uint8, device="cuda")
        return self._records

    def step(self, n, records=True):
        """Runs n updates; returns the records as a numpy array (synchronising)
        when records is True, the device buffer when records == "device", else None."""
        buf = self.record_buffer(n) if records else None
        wolff_step(self.handle, n, buf)
        if records == "device":
            return buf
        if records:
            return records_to_numpy(buf, n)
        return None

    def measure(self):
        return measure(self.handle)

    def measure_full(self):
        return measure_full(self.handle)

    def get_state(self):
        return wolff_get_state(self.handle, self.N)

    def set_state(self, spins, t):
        wolff_set_state(self.handle, spins, t)

    def run_host(self, n, spins_in=None, t_in=0, records=True, spins_out=True):
        rec_out = None
        if records:
            # records land in a pinned buffer kept by the lattice (a direct
            # DMA), and the caller gets a copy
            torch = _torch()
            need = int(n) * RECORD_BYTES
            if getattr(self, "_h_records", None) is None or self._h_records.numel() < need:
                self._h_records = torch.empty(max(need, RECORD_BYTES), dtype=torch.uint8,
                                              pin_memory=True)
            rec_out = self._h_records.numpy()[:need].view(RECORD_DTYPE)
        rec, sout = wolff_run_host(self.handle, self.N, n, spins_in, t_in, records, spins_out,
                                   rec_out)
        return (rec.copy() if rec is not None else None), sout

    def get_state_bits(self):
        bits = np.zeros((self.N + 31) // 32, dtype=np.uint32)
        t = ctypes.c_uint64()
        _check(load_library().wolff_get_state_bits(self.handle, ctypes.c_void_p(bits.ctypes.data),
                                                   ctypes.byref(t)), self.handle)
        return bits, t.value

    def set_state_bits(self, bits, t):
        bits = np.ascontiguousarray(bits, dtype=np.uint32)
        if bits.size != (self.N + 31) // 32:
            raise ValueError("need %d words" % ((self.N + 31) // 32))
        _check(load_library().wolff_set_state_bits(self.handle, ctypes.c_void_p(bits.ctypes.data),
                                                   int(t)), self.handle)

    def run_host_bits(self, n, bits_in=None, t_in=0, records=True, bits_out=True,
                      records_out=None):
        """As run_host with bit-packed lattices (see pack_spins).  records_out:
        an optional C-contiguous RECORD_DTYPE array of at least n entries
        (pinned memory for an asynchronous copy) that receives the records
        directly; its first n entries are returned instead of a copy."""
        words = (self.N + 31) // 32
        bin_ = None if bits_in is None else np.ascontiguousarray(bits_in, dtype=np.uint32)
        if bin_ is not None and bin_.size != words:
            raise ValueError("need %d words" % words)
        rec = None
        if records and records_out is not None:
            if (records_out.dtype != RECORD_DTYPE or records_out.size < int(n)
                    or not records_out.flags["C_CONTIGUOUS"]):
                raise ValueError("records_out must be a C-contiguous RECORD_DTYPE array of "
                                 "at least n entries")
            rec = records_out[:int(n)]
        elif records:
            torch = _torch()
            need = int(n) * RECORD_BYTES
            if getattr(self, "_h_records", None) is None or self._h_records.numel() < need:
                self._h_records = torch.empty(max(need, RECORD_BYTES), dtype=torch.uint8,
                                              pin_memory=True)
            rec = self._h_records.numpy()[:need].view(RECORD_DTYPE)
        bout = np.empty(words, dtype=np.uint32) if bits_out else None
        ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        _check(load_library().wolff_run_host_bits(self.handle, ptr(bin_), int(t_in), int(n),
                                                  ptr(rec), ptr(bout)), self.handle)
        if rec is not None and records_out is None:
            rec = rec.copy()
        return rec, bout

    def selftest_wait_timeout(self, wait_ns):
        obs = ctypes.c_int()
        _check(load_library().wolff_selftest_wait_timeout(self.handle, int(wait_ns),
                                                          ctypes.byref(obs)), self.handle)
        return obs.value

    def close(self):
        if self.handle is not None:
            ising_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WolffBatch:
    """Runs the next updates of many WolffLattice objects in one launch (one
    thread-block cluster per lattice, or with schedule=SCHED_TINY one CTA per
    lattice of at most TINY_MAX_SITES sites).  Each lattice's chain is the one
    it would follow alone."""

    def __init__(self, capacity, stream=None, schedule=SCHED_CLUSTER):
        self.handle = ctypes.c_void_p()
        _check(load_library().wolff_batch_create(ctypes.byref(self.handle), int(capacity),
                                                 _stream_handle(stream)))
        self.capacity = int(capacity)
        if schedule != SCHED_CLUSTER:
            self.set_schedule(schedule)

    def set_schedule(self, schedule):
        """SCHED_CLUSTER (teams, the default) or SCHED_TINY (one CTA per
        lattice; run() then takes cluster_size=1 and block_threads=0 for the
        default CTA size)."""
        _check(load_library().wolff_batch_set_schedule(self.handle, int(schedule)))
        self.schedule = int(schedule)

    def run(self, lattices, n_updates, records=None, cluster_size=1, block_threads=256,
            budget_ns=0):
        """lattices: list of WolffLattice; n_updates: int or per-lattice list;
        records: None or a list of device uint8 tensors (or None entries);
        budget_ns: device-time limit per lattice (0 = none; the updates done
        are then read back through each lattice's stats()["updates"])."""
        n = len(lattices)
        if isinstance(n_updates, int):
            n_updates = [n_updates] * n
        ctxs = (ctypes.c_void_p * n)(*[lat.handle.value for lat in lattices])
        nu = (ctypes.c_uint64 * n)(*[int(x) for x in n_updates])
        recs = None
        if records is not None:
            recs = (ctypes.c_void_p * n)(*[None if r is None else r.data_ptr() for r in records])
        _check(load_library().wolff_batch_run_timed(self.handle, ctxs, n, nu, recs,
                                                    int(cluster_size), int(block_threads),
                                                    int(budget_ns)))

    def set_window(self, slots_per_cta):
        """Window slots per CTA of this batch's launches (16, 32, 64, 128; 0 =
        window mode off)."""
        _check(load_library().wolff_batch_set_window(self.handle, int(slots_per_cta)))

    def close(self):
        if self.handle is not None and self.handle.value:
            load_library().wolff_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



def xy_init(dim, L, angle_bits, J, T, seed, workspace=None, stream=None):
    """Creates an XY context; returns (handle, workspace tensor)."""
    torch = _torch()
    lib = load_library()
    nbytes = lib.wolff_xy_workspace_bytes(dim, L)
    if nbytes == 0:
        raise WolffError(WOLFF_EINVAL, "invalid lattice shape dim=%r L=%r" % (dim, L))
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    handle = ctypes.c_void_p()
    st = lib.xy_init(ctypes.byref(handle), int(dim), int(L), int(angle_bits), float(J), float(T),
                     int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.c_void_p(workspace.data_ptr()),
                     workspace.numel(), _stream_handle(stream))
    _check(st)
    return handle, workspace


class WolffXY:
    """One XY lattice (angles in units of 2 pi / 65536 on a grid of
    angle_bits bits) and its embedded-cluster Wolff chain on the current
    CUDA device.  Energies and magnetisations are fixed point (units 2^-30)."""

    def __init__(self, dim, L, T, J=1.0, seed=0, angle_bits=XY_ANGLE_BITS, grid_blocks=0,
                 block_threads=0, stream=None):
        self.dim, self.L, self.J, self.T, self.seed = int(dim), int(L), float(J), float(T), int(seed)
        self.N = self.L ** self.dim
        self.angle_bits = int(angle_bits)
        self.handle, self.workspace = xy_init(dim, L, angle_bits, J, T, seed, stream=stream)
        self._records = None
        if grid_blocks or block_threads:
            self.set_schedule(SCHED_CLUSTER, grid_blocks, block_threads)

    def set_schedule(self, schedule=SCHED_CLUSTER, grid_blocks=0, block_threads=0):
        _check(load_library().wolff_set_schedule(self.handle, int(schedule), int(grid_blocks),
                                                 int(block_threads)), self.handle)

    def record_buffer(self, n):
        torch = _torch()
        need = int(n) * XY_RECORD_BYTES
        if self._records is None or self._records.numel() < need:
            self._records = torch.empty(max(need, XY_RECORD_BYTES), dtype=torch.uint8,
                                        device="cuda")
        return self._records

    def step(self, n, records=True):
        """Runs n updates; returns the records as a numpy array (synchronising)
        when records is True, the device buffer when records == "device", else None."""
        buf = self.record_buffer(n) if records else None
        wolff_step(self.handle, n, buf)
        if records == "device":
            return buf
        if records:
            host = buf[: int(n) * XY_RECORD_BYTES].cpu().numpy()
            return host.view(XY_RECORD_DTYPE).copy()
        return None

    def measure(self):
        E, Mx, My, C = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        _check(load_library().xy_measure(self.handle, ctypes.byref(E), ctypes.byref(Mx),
                                         ctypes.byref(My), ctypes.byref(C)), self.handle)
        return E.value, Mx.value, My.value, C.value

    def measure_full(self):
        E, Mx, My = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load_library().xy_measure_full(self.handle, ctypes.byref(E), ctypes.byref(Mx),
                                              ctypes.byref(My)), self.handle)
        return E.value, Mx.value, My.value

    def get_state(self):
        theta = np.zeros(self.N, dtype=np.uint16)
        t = ctypes.c_uint64()
        _check(load_library().xy_get_state(self.handle, theta.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(t)), self.handle)
        return theta, t.value

    def set_state(self, theta, t):
        theta = np.ascontiguousarray(theta, dtype=np.uint16)
        if theta.size != self.N:
            raise ValueError("need %d angles" % self.N)
        _check(load_library().xy_set_state(self.handle, theta.ctypes.data_as(ctypes.c_void_p),
                                           int(t)), self.handle)

    def set_helpers(self, max_helpers):
        """Helper teams of the cluster schedule: -1 = as many as fit (the
        default), 0 = none, k > 0 = at most k."""
        _check(load_library().wolff_set_helpers(self.handle, int(max_helpers)), self.handle)

    def stats(self):
        st = _Stats()
        _check(load_library().wolff_get_stats(self.handle, ctypes.byref(st)), self.handle)
        return {k: int(getattr(st, k)) for k, _ in _Stats._fields_}

    def info(self):
        inf = _Info()
        _check(load_library().wolff_get_info(self.handle, ctypes.byref(inf)), self.handle)
        return {k: getattr(inf, k) for k, _ in _Info._fields_}

    def close(self):
        if self.handle is not None:
            ising_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
