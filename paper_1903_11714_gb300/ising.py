"""ctypes binding of libising_gb300.so (C ABI in include/ising.h).

Argument marshalling only: every function forwards to the C entry point of the
same name, and every step of the sweep runs in the library's CUDA kernels.  If
the library has not been built, ``lib()`` raises -- there is no fallback.

``Lattice``, ``Lattice3D`` and ``Batch`` are small owners of an ``ising_t`` /
``ising_batch_t`` handle that call the same entry points.  Streams may be given as a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None (the handle then
creates its own stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libising_gb300.so")

ISING_OK, ISING_EINVAL, ISING_ENOMEM, ISING_ECUDA, ISING_ETIMEOUT, ISING_EBUSY = 0, -1, -2, -3, -4, -5
HOT, COLD = 0, 1
PACKED, INT8 = 0, 1
CUBIC = 2  # kernel id recorded in checkpoints of 3D handles

# Entry points declared in include/ising.h: name -> (restype, argtypes)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_d = ctypes.c_double
_P = ctypes.POINTER
_SIGS = {
    "ising_last_error": (ctypes.c_char_p, []),
    "ising_version": (ctypes.c_char_p, []),
    "ising_thresholds": (ctypes.c_int, [_d, _P(_u64)]),
    "ising_init": (ctypes.c_int, [_P(_vp), _i64, _d, _u64]),
    "ising_init_ex": (ctypes.c_int, [_P(_vp), _i64, _d, _u64, ctypes.c_int, ctypes.c_int, _vp]),
    "ising_sweep": (ctypes.c_int, [_vp, _i64]),
    "ising_observables": (ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i64)]),
    "ising_history": (ctypes.c_int, [_vp, _i64, _i64, _P(_i64), _P(_i64)]),
    "ising_moments": (ctypes.c_int, [_vp, _i64, _P(_d), _P(_d), _P(_d), _P(_d), _P(_d)]),
    "ising_moments_ex": (ctypes.c_int, [_vp, _i64, _P(_d), _P(_u64)]),
    "ising_get_lattice": (ctypes.c_int, [_vp, _P(ctypes.c_int8)]),
    "ising_get_rows": (ctypes.c_int, [_vp, _i64, _i64, _P(ctypes.c_int8)]),
    "ising_set_lattice": (ctypes.c_int, [_vp, _P(ctypes.c_int8)]),
    "ising_get_planes": (ctypes.c_int, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_uint32)]),
    "ising_set_planes": (ctypes.c_int, [_vp, _P(ctypes.c_uint32), _P(ctypes.c_uint32)]),
    "ising_state_bytes": (ctypes.c_int, [_vp, _P(_i64)]),
    "ising_save": (ctypes.c_int, [_vp, _vp, _i64]),
    "ising_load": (ctypes.c_int, [_P(_vp), _vp, _i64, _vp]),
    "ising_synchronize": (ctypes.c_int, [_vp]),
    "ising_free": (ctypes.c_int, [_vp]),
    "ising_thresholds3d": (ctypes.c_int, [_d, _P(_u64)]),
    "ising_init3d": (ctypes.c_int, [_P(_vp), _i64, _d, _u64, ctypes.c_int, _vp]),
    "ising_batch_create": (ctypes.c_int, [_P(_vp), _i32, _P(_i64), _P(_d), _P(_u64), _P(_i32)]),
    "ising_batch_create_ex": (ctypes.c_int, [_P(_vp), _i32, _i64, _i64, _i32, _vp]),
    "ising_batch_add": (ctypes.c_int, [_vp, _i64, _d, _u64, _i32, _i64, _i32, _P(_i32)]),
    "ising_batch_add_tiled": (ctypes.c_int, [_vp, _i64, _d, _u64, _i32, _i64, _i32, _i32, _P(_i32)]),
    "ising_batch_remove": (ctypes.c_int, [_vp, _i32]),
    "ising_batch_run": (ctypes.c_int, [_vp, _i64, _i32]),
    "ising_batch_sweeps_done": (ctypes.c_int, [_vp, _i32, _P(_i64)]),
    "ising_batch_progress": (ctypes.c_int, [_vp, _P(_i64), _i32]),
    "ising_batch_observables": (ctypes.c_int, [_vp, _i32, _P(_i64), _P(_i64)]),
    "ising_batch_gather": (ctypes.c_int, [_vp, _i32, _P(_i32), _vp]),
    "ising_batch_specialized": (ctypes.c_int, [_vp, _P(_i32)]),
    "ising_batch_set_cluster": (ctypes.c_int, [_vp, _i32]),
    "ising_batch_cluster_size": (ctypes.c_int, [_vp, _P(_i32)]),
    "ising_batch_observables_ex": (ctypes.c_int, [_vp, _i32, _P(_i64), _P(_i64), _P(_i64)]),
    "ising_batch_history": (ctypes.c_int, [_vp, _i32, _i64, _i64, _P(_i64), _P(_i64)]),
    "ising_batch_moments": (ctypes.c_int, [_vp, _i32, _i64, _P(_d), _P(_u64)]),
    "ising_batch_get_lattice": (ctypes.c_int, [_vp, _i32, _P(ctypes.c_int8)]),
    "ising_batch_usage": (ctypes.c_int, [_vp, _P(_i64), _P(_i32)]),
    "ising_batch_synchronize": (ctypes.c_int, [_vp]),
    "ising_batch_free": (ctypes.c_int, [_vp]),
    "ising_autotune": (ctypes.c_int, [_i64, _P(_i32), _P(_i32), _P(_d)]),
    "ising_dev_philox": (ctypes.c_int, [_u64, _P(ctypes.c_uint32), _i64, _vp, _vp]),
    "ising_probe_int_rates": (ctypes.c_int, [_P(_d)]),
    "ising_selftest_timeout": (ctypes.c_int, [_i64, _P(ctypes.c_int)]),
    "ising_set_specialize": (ctypes.c_int, [_i32]),
    "ising_specialized": (ctypes.c_int, [_vp, _P(_i32), ctypes.c_char_p, _i64]),
    "ising_sweep_packed_noalloc": (ctypes.c_int, [_i32, _P(_vp), _P(_vp), _P(_i64), _P(_d), _P(_u64), _i64, _i64,
                                                  _P(_vp), _vp, _i32]),
}
EXPORTS = tuple(_SIGS)

_lib = None
_lock = threading.Lock()


class IsingError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ising error {code}: {msg}")
        self.code = code


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1903_11714_gb300/build.py "
                                   "(or __graft_entry__.build()); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().ising_last_error().decode()


def _check(rc: int) -> None:
    if rc != ISING_OK:
        raise IsingError(rc, last_error())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# --------------------------------------------------------------- entry points
def ising_thresholds(beta: float) -> tuple[int, int]:
    T = np.zeros(2, dtype=np.uint64)
    _check(lib().ising_thresholds(float(beta), _ptr(T, ctypes.c_uint64)))
    return int(T[0]), int(T[1])


def ising_init_ex(L: int, beta: float, seed: int, start: int = HOT, kernel: int = PACKED, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ising_init_ex(ctypes.byref(h), int(L), float(beta), int(seed), int(start), int(kernel),
                               _stream_ptr(stream)))
    return h.value


def ising_init(L: int, beta: float, seed: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().ising_init(ctypes.byref(h), int(L), float(beta), int(seed)))
    return h.value


def ising_sweep(h: int, n: int) -> None:
    _check(lib().ising_sweep(h, int(n)))


def ising_observables(h: int) -> tuple[int, int, int]:
    M, E, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ising_observables(h, ctypes.byref(M), ctypes.byref(E), ctypes.byref(n)))
    return M.value, E.value, n.value


def ising_history(h: int, first: int, count: int) -> tuple[np.ndarray, np.ndarray]:
    M = np.zeros(count, dtype=np.int64)
    E = np.zeros(count, dtype=np.int64)
    _check(lib().ising_history(h, int(first), int(count), _ptr(M, ctypes.c_int64), _ptr(E, ctypes.c_int64)))
    return M, E


_MOMENT_KEYS = ("abs_m", "m2", "m4", "e", "e2", "binder")


def _moments_dict(out: np.ndarray, sums: np.ndarray) -> dict:
    d = {k: float(v) for k, v in zip(_MOMENT_KEYS, out)}
    s = [int(v) for v in sums]
    d["S1"] = s[0]
    d["S2"] = s[1] | s[2] << 64
    d["S4"] = s[3] | s[4] << 64 | s[5] << 128 | s[6] << 192
    se = s[7] | s[8] << 64
    d["SE"] = se - (1 << 128) if se >> 127 else se
    d["SE2"] = s[9] | s[10] << 64
    return d


def ising_moments(h: int, burn_in: int) -> tuple[float, float, float, float, float]:
    """(<|m|>, <m^2>, <m^4>, <e>, U4) over samples burn_in .. sweeps_done-1."""
    v = [ctypes.c_double() for _ in range(5)]
    _check(lib().ising_moments(h, int(burn_in), *(ctypes.byref(x) for x in v)))
    return tuple(x.value for x in v)


def ising_moments_ex(h: int, burn_in: int) -> dict:
    out = np.zeros(6, dtype=np.float64)
    sums = np.zeros(11, dtype=np.uint64)
    _check(lib().ising_moments_ex(h, int(burn_in), _ptr(out, ctypes.c_double), _ptr(sums, ctypes.c_uint64)))
    return _moments_dict(out, sums)


def ising_batch_create(Ls, betas, seeds, starts) -> int:
    """A batch of len(Ls) packed lattices from per-lattice arrays (slot k = lattice k)."""
    n = len(Ls)
    b = ctypes.c_void_p()
    _check(lib().ising_batch_create(ctypes.byref(b), n, (ctypes.c_int64 * n)(*Ls), (ctypes.c_double * n)(*betas),
                                    (ctypes.c_uint64 * n)(*seeds), (ctypes.c_int32 * n)(*starts)))
    return b.value


def ising_batch_run(b: int, sweeps: int, use_graph: int = 0) -> None:
    _check(lib().ising_batch_run(b, int(sweeps), int(use_graph)))


def ising_batch_observables(b: int, idx: int) -> tuple[int, int]:
    M, E = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ising_batch_observables(b, int(idx), ctypes.byref(M), ctypes.byref(E)))
    return M.value, E.value


SPECIALIZE_OFF, SPECIALIZE_AUTO, SPECIALIZE_ALWAYS = 0, 1, 2
CLUSTER_OFF, CLUSTER_AUTO, CLUSTER_ALWAYS = 0, 1, 2


def ising_set_specialize(mode: int) -> None:
    """Process-wide: whether handles created afterwards sweep with a kernel compiled
    for their thresholds (SPECIALIZE_OFF, _AUTO (default), _ALWAYS)."""
    _check(lib().ising_set_specialize(int(mode)))


def ising_specialized(h: int) -> tuple[bool, str]:
    flag = ctypes.c_int32()
    buf = ctypes.create_string_buffer(256)
    _check(lib().ising_specialized(h, ctypes.byref(flag), buf, len(buf)))
    return bool(flag.value), buf.value.decode()


def ising_thresholds3d(beta: float) -> tuple[int, int, int]:
    T = np.zeros(3, dtype=np.uint64)
    _check(lib().ising_thresholds3d(float(beta), _ptr(T, ctypes.c_uint64)))
    return int(T[0]), int(T[1]), int(T[2])


def ising_init3d(L: int, beta: float, seed: int, start: int = HOT, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().ising_init3d(ctypes.byref(h), int(L), float(beta), int(seed), int(start), _stream_ptr(stream)))
    return h.value


def ising_get_lattice(h: int, L: int, dim: int = 2) -> np.ndarray:
    out = np.empty((L,) * dim, dtype=np.int8)
    _check(lib().ising_get_lattice(h, _ptr(out, ctypes.c_int8)))
    return out


def ising_get_rows(h: int, L: int, row0: int, nrows: int) -> np.ndarray:
    """Rows row0 .. row0+nrows-1 as an (nrows, L) int8 array (a cube's rows are r = i*L + j)."""
    out = np.empty((int(nrows), L), dtype=np.int8)
    _check(lib().ising_get_rows(h, int(row0), int(nrows), _ptr(out, ctypes.c_int8)))
    return out


def ising_set_lattice(h: int, lattice: np.ndarray) -> None:
    a = np.ascontiguousarray(lattice, dtype=np.int8)
    _check(lib().ising_set_lattice(h, _ptr(a, ctypes.c_int8)))


def ising_get_planes(h: int, L: int, black: np.ndarray | None = None,
                     white: np.ndarray | None = None, dim: int = 2) -> tuple[np.ndarray, np.ndarray]:
    n = L ** (dim - 1) * (L // 64)
    b = np.empty(n, dtype=np.uint32) if black is None else black
    w = np.empty(n, dtype=np.uint32) if white is None else white
    assert b.dtype == np.uint32 and w.dtype == np.uint32 and b.flags.c_contiguous and w.flags.c_contiguous
    assert b.size == w.size == n
    _check(lib().ising_get_planes(h, _ptr(b, ctypes.c_uint32), _ptr(w, ctypes.c_uint32)))
    return b, w


def ising_set_planes(h: int, black: np.ndarray, white: np.ndarray) -> None:
    b = np.ascontiguousarray(black, dtype=np.uint32)
    w = np.ascontiguousarray(white, dtype=np.uint32)
    _check(lib().ising_set_planes(h, _ptr(b, ctypes.c_uint32), _ptr(w, ctypes.c_uint32)))


def ising_save(h: int) -> bytes:
    n = ctypes.c_int64()
    _check(lib().ising_state_bytes(h, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().ising_save(h, buf, n.value))
    return buf.raw


def ising_load(blob: bytes, stream=None) -> int:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().ising_load(ctypes.byref(h), buf, len(blob), _stream_ptr(stream)))
    return h.value


def ising_synchronize(h: int) -> None:
    _check(lib().ising_synchronize(h))


def ising_free(h: int) -> None:
    _check(lib().ising_free(h))


def ising_autotune(L: int) -> tuple[int, int, float]:
    tr, th, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(lib().ising_autotune(int(L), ctypes.byref(tr), ctypes.byref(th), ctypes.byref(ms)))
    return tr.value, th.value, ms.value


def ising_dev_philox(key: int, ctr, nblocks: int, out_dev_ptr: int, stream=None) -> None:
    c = np.asarray(ctr, dtype=np.uint32)
    _check(lib().ising_dev_philox(int(key), _ptr(c, ctypes.c_uint32), int(nblocks), out_dev_ptr,
                                  _stream_ptr(stream)))


def ising_probe_int_rates() -> tuple[float, float]:
    out = np.zeros(2, dtype=np.float64)
    _check(lib().ising_probe_int_rates(_ptr(out, ctypes.c_double)))
    return float(out[0]), float(out[1])


def ising_selftest_timeout(wait_cycles: int) -> int:
    """Runs the bounded-wait self-test; returns the status the kernel reported."""
    obs = ctypes.c_int()
    _check(lib().ising_selftest_timeout(int(wait_cycles), ctypes.byref(obs)))
    return obs.value


def ising_sweep_packed_noalloc(black_ptrs, white_ptrs, Ls, betas, seeds, first_sweep: int, nsweeps: int, me_ptrs,
                               stream=None, wait: bool = True) -> None:
    """Sweeps caller-owned device planes without any device allocation (device
    pointers as integers, one entry per lattice)."""
    n = len(Ls)
    vp = ctypes.c_void_p * n
    _check(lib().ising_sweep_packed_noalloc(
        n, vp(*black_ptrs), vp(*white_ptrs), (ctypes.c_int64 * n)(*Ls), (ctypes.c_double * n)(*betas),
        (ctypes.c_uint64 * n)(*seeds), int(first_sweep), int(nsweeps), vp(*me_ptrs), _stream_ptr(stream),
        1 if wait else 0))


# ------------------------------------------------------------------ classes
class Lattice:
    """One lattice (an ``ising_t``)."""

    def __init__(self, L: int, beta: float, seed: int, start: int = HOT, kernel: int = PACKED, stream=None,
                 _handle: int | None = None):
        self.L, self.beta, self.seed, self.start, self.kernel = int(L), float(beta), int(seed), start, kernel
        self.h = _handle if _handle is not None else ising_init_ex(L, beta, seed, start, kernel, stream)

    def sweep(self, n: int) -> "Lattice":
        ising_sweep(self.h, n)
        return self

    def observables(self):
        return ising_observables(self.h)

    def history(self, first: int = 0, count: int | None = None):
        if count is None:
            count = self.observables()[2] - first
        return ising_history(self.h, first, count)

    def moments(self, burn_in: int) -> dict:
        return ising_moments_ex(self.h, burn_in)

    def get_lattice(self) -> np.ndarray:
        return ising_get_lattice(self.h, self.L)

    def get_rows(self, row0: int, nrows: int) -> np.ndarray:
        return ising_get_rows(self.h, self.L, row0, nrows)

    def set_lattice(self, a: np.ndarray) -> None:
        ising_set_lattice(self.h, a)

    def get_planes(self, black=None, white=None):
        return ising_get_planes(self.h, self.L, black, white)

    def set_planes(self, black, white) -> None:
        ising_set_planes(self.h, black, white)

    def save(self) -> bytes:
        return ising_save(self.h)

    @classmethod
    def load(cls, blob: bytes, stream=None):
        """A Lattice (or a Lattice3D for a 3D checkpoint) continuing the saved chain."""
        h = ising_load(blob, stream)
        import struct
        L, kernel, start = struct.unpack_from("<qqq", blob, 16)
        beta, seed = struct.unpack_from("<dQ", blob, 16 + 8 * 5)
        if kernel == CUBIC:
            return Lattice3D(L, beta, seed, start, _handle=h)
        return cls(L, beta, seed, start, kernel, _handle=h)

    def synchronize(self) -> None:
        ising_synchronize(self.h)

    def specialized(self) -> tuple[bool, str]:
        """(True, note) when the sweeps run a kernel compiled for this lattice's thresholds."""
        return ising_specialized(self.h)

    def close(self) -> None:
        if self.h:
            ising_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many packed lattices swept together (an ``ising_batch_t``)."""

    def __init__(self, capacity: int, max_L: int, arena_bytes: int, threads: int = 0, stream=None,
                 _handle: int | None = None, _Ls=None):
        if _handle is not None:
            self.b = _handle
            self.L = {k: int(v) for k, v in enumerate(_Ls)}
            return
        b = ctypes.c_void_p()
        _check(lib().ising_batch_create_ex(ctypes.byref(b), int(capacity), int(max_L), int(arena_bytes),
                                           int(threads), _stream_ptr(stream)))
        self.b = b.value
        self.L = {}

    @classmethod
    def from_arrays(cls, Ls, betas, seeds, starts) -> "Batch":
        """Lattice k of the arrays in slot k, no sweep limit (ising_batch_create)."""
        return cls(0, 0, 0, _handle=ising_batch_create(Ls, betas, seeds, starts), _Ls=Ls)

    def add(self, L: int, beta: float, seed: int, start: int, sweeps: int, tile_rows: int = 0,
            tile_words: int = 0) -> int:
        idx = ctypes.c_int32()
        _check(lib().ising_batch_add_tiled(self.b, int(L), float(beta), int(seed), int(start), int(sweeps),
                                           int(tile_rows), int(tile_words), ctypes.byref(idx)))
        self.L[idx.value] = int(L)
        return idx.value

    def remove(self, idx: int) -> None:
        _check(lib().ising_batch_remove(self.b, int(idx)))
        self.L.pop(idx, None)

    def run(self, sweeps: int, graph_sweeps: int = 0) -> None:
        _check(lib().ising_batch_run(self.b, int(sweeps), int(graph_sweeps)))

    def sweeps_done(self, idx: int) -> int:
        n = ctypes.c_int64()
        _check(lib().ising_batch_sweeps_done(self.b, int(idx), ctypes.byref(n)))
        return n.value

    def progress(self, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=np.int64)
        _check(lib().ising_batch_progress(self.b, _ptr(out, ctypes.c_int64), int(n)))
        return out[:n]

    def observables(self, idx: int):
        M, E, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ising_batch_observables_ex(self.b, int(idx), ctypes.byref(M), ctypes.byref(E),
                                                ctypes.byref(n)))
        return M.value, E.value, n.value

    def history(self, idx: int, first: int = 0, count: int | None = None):
        if count is None:
            count = self.sweeps_done(idx) - first
        M = np.zeros(count, dtype=np.int64)
        E = np.zeros(count, dtype=np.int64)
        _check(lib().ising_batch_history(self.b, int(idx), int(first), int(count), _ptr(M, ctypes.c_int64),
                                         _ptr(E, ctypes.c_int64)))
        return M, E

    def moments(self, idx: int, burn_in: int) -> dict:
        out = np.zeros(6, dtype=np.float64)
        sums = np.zeros(11, dtype=np.uint64)
        _check(lib().ising_batch_moments(self.b, int(idx), int(burn_in), _ptr(out, ctypes.c_double),
                                         _ptr(sums, ctypes.c_uint64)))
        return _moments_dict(out, sums)

    def get_lattice(self, idx: int) -> np.ndarray:
        L = self.L[idx]
        out = np.empty((L, L), dtype=np.int8)
        _check(lib().ising_batch_get_lattice(self.b, int(idx), _ptr(out, ctypes.c_int8)))
        return out

    def specialized(self) -> bool:
        """True while the batch sweeps with a kernel compiled for its one temperature."""
        flag = ctypes.c_int32()
        _check(lib().ising_batch_specialized(self.b, ctypes.byref(flag)))
        return bool(flag.value)

    def set_cluster(self, mode: int) -> None:
        """CLUSTER_OFF, CLUSTER_AUTO (default) or CLUSTER_ALWAYS: when a batch of one
        side L <= 4096 keeps its lattices in thread-block clusters."""
        _check(lib().ising_batch_set_cluster(self.b, int(mode)))

    def cluster_size(self) -> int:
        """CTAs per cluster of the cluster-resident sweep, 0 on the tiled kernel."""
        c = ctypes.c_int32()
        _check(lib().ising_batch_cluster_size(self.b, ctypes.byref(c)))
        return c.value

    def gather(self, idx, out_ptr: int) -> None:
        """Enqueue (sweeps done, M, E) of slots idx into out_ptr (3 int64 each,
        device-accessible memory); returns without waiting."""
        n = len(idx)
        _check(lib().ising_batch_gather(self.b, n, (ctypes.c_int32 * max(n, 1))(*idx), out_ptr))

    def usage(self) -> tuple[int, int]:
        a, s = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().ising_batch_usage(self.b, ctypes.byref(a), ctypes.byref(s)))
        return a.value, s.value

    def synchronize(self) -> None:
        _check(lib().ising_batch_synchronize(self.b))

    def close(self) -> None:
        if self.b:
            _check(lib().ising_batch_free(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice3D(Lattice):
    """One cubic L x L x L lattice (an ``ising_t`` made by ``ising_init3d``)."""

    def __init__(self, L: int, beta: float, seed: int, start: int = HOT, stream=None, _handle: int | None = None):
        self.L, self.beta, self.seed, self.start, self.kernel = int(L), float(beta), int(seed), start, CUBIC
        self.h = _handle if _handle is not None else ising_init3d(L, beta, seed, start, stream)

    def get_lattice(self) -> np.ndarray:
        return ising_get_lattice(self.h, self.L, dim=3)

    def get_rows(self, row0: int, nrows: int) -> np.ndarray:
        return ising_get_rows(self.h, self.L, row0, nrows)

    def set_lattice(self, a: np.ndarray) -> None:
        raise IsingError(ISING_EINVAL, "set_lattice is for 2D lattices; use set_planes")

    def get_planes(self, black=None, white=None):
        return ising_get_planes(self.h, self.L, black, white, dim=3)
