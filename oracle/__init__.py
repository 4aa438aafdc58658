"""CPU oracle for the checkerboard Metropolis sweep of the 2D Ising model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library path
never imports it, and it shares no code with the CUDA path.

The chain itself lives in ``ising_oracle.c`` (plain C, one site at a time, its
own Philox4x32-10) and, for the three-dimensional generalisation the paper's
conclusion names, ``ising3d_oracle.c``; this module builds both with gcc into one
shared object and wraps them with ctypes.
``exact.py`` holds the closed forms and exact enumerations the oracle is pinned
against.

Every function cites the passage it follows: the paper's Sec. 3 (Hamiltonian,
torus, mu = 0, J = 1), Sec. 3.1 (checkerboard kernel and its acceptance rule),
Algorithms 1-2 (the half-sweep), Sec. 4.1 (magnetisation and Binder parameter,
10% burn-in).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

# libgomp reads this when the library loads: threads that wait at the end of a
# parallel region sleep instead of spinning, so a busy host does not stall the
# short per-half-sweep regions of small lattices.
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "ising_oracle.c"), os.path.join(_HERE, "ising3d_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_ising_oracle.so")
_lib = None
_lock = threading.Lock()

HOT, COLD = 0, 1
INIT_SWEEP = 0xFFFFFFFF  # sweep slot (counter word 0) reserved for the hot start


def build(force: bool = False) -> str:
    """Compile ising_oracle.c into a shared object next to it (gcc, OpenMP)."""
    newest = max(os.path.getmtime(p) for p in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, *_SRCS, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i8p = ctypes.POINTER(ctypes.c_int8)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_philox4x32_10.restype = None
            L.oracle_thresholds.argtypes = [ctypes.c_double, u64p]
            L.oracle_thresholds.restype = None
            L.oracle_accept.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_accept.restype = ctypes.c_int
            L.oracle_site_word.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]
            L.oracle_site_word.restype = ctypes.c_uint32
            L.oracle_init.argtypes = [i8p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int]
            L.oracle_init.restype = None
            L.oracle_observe.argtypes = [i8p, ctypes.c_int64, i64p, i64p]
            L.oracle_observe.restype = None
            L.oracle_half_sweep_words.argtypes = [i8p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                                  ctypes.c_uint64, u32p]
            L.oracle_half_sweep_words.restype = ctypes.c_int64
            L.oracle_run.argtypes = [i8p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                     ctypes.c_int64, i64p, i64p, ctypes.c_int]
            L.oracle_run.restype = ctypes.c_int64
            L.oracle_window.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, i8p]
            L.oracle_window.restype = ctypes.c_int
            L.oracle_init_rows.argtypes = [i8p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_int64]
            L.oracle_init_rows.restype = None
            L.oracle_half_sweep_rows.argtypes = [i8p, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64]
            L.oracle_half_sweep_rows.restype = ctypes.c_int64
            dims = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
            L.oracle3d_thresholds.argtypes = [ctypes.c_double, u64p]
            L.oracle3d_thresholds.restype = None
            L.oracle3d_accept.argtypes = [ctypes.c_int, ctypes.c_uint32, u64p]
            L.oracle3d_accept.restype = ctypes.c_int
            L.oracle3d_site_word.argtypes = dims + [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]
            L.oracle3d_site_word.restype = ctypes.c_uint32
            L.oracle3d_init.argtypes = [i8p] + dims + [ctypes.c_uint64, ctypes.c_int]
            L.oracle3d_init.restype = None
            L.oracle3d_observe.argtypes = [i8p] + dims + [i64p, i64p]
            L.oracle3d_observe.restype = None
            L.oracle3d_half_sweep_words.argtypes = [i8p] + dims + [ctypes.c_int, u64p, u32p]
            L.oracle3d_half_sweep_words.restype = ctypes.c_int64
            L.oracle3d_run.argtypes = [i8p] + dims + [ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                                      ctypes.c_int64, i64p, i64p, ctypes.c_int]
            L.oracle3d_run.restype = ctypes.c_int64
            L.oracle3d_window.argtypes = dims + [ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                                 ctypes.c_int64] + [ctypes.c_int64] * 6 + [i8p]
            L.oracle3d_window.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    """Philox4x32-10 (Salmon et al., SC'11) on one 128-bit counter."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return tuple(int(v) for v in out)


def thresholds(beta: float) -> tuple[int, int]:
    """(T_2, T_4): ceil(exp(-2 beta h) 2^32) for h = 2, 4 (Sec. 3.1 acceptance rule)."""
    T = np.zeros(2, dtype=np.uint64)
    lib().oracle_thresholds(float(beta), _ptr(T, ctypes.c_uint64))
    return int(T[0]), int(T[1])


def accept(h: int, x: int, T2: int, T4: int) -> bool:
    return bool(lib().oracle_accept(int(h), int(x), int(T2), int(T4)))


def site_word(L: int, i: int, j: int, seed: int, sweep: int, c: int) -> int:
    return int(lib().oracle_site_word(L, i, j, seed, sweep, c))


def init(L: int, seed: int, start: int = HOT) -> np.ndarray:
    """Start state: hot (iid +-1 from Philox) or cold (all +1); row-major int8."""
    _check_L(L)
    s = np.empty((L, L), dtype=np.int8)
    lib().oracle_init(_ptr(s, ctypes.c_int8), L, int(seed), int(start))
    return s


def observe(s: np.ndarray) -> tuple[int, int]:
    """(M, E) with M = sum sigma and E = H(sigma), mu = 0, J = 1 (Sec. 3)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    M = ctypes.c_int64()
    E = ctypes.c_int64()
    lib().oracle_observe(_ptr(s, ctypes.c_int8), s.shape[0], ctypes.byref(M), ctypes.byref(E))
    return M.value, E.value


def half_sweep_words(s: np.ndarray, c: int, T2: int, T4: int, words: np.ndarray) -> int:
    """One colour-c half-sweep with caller-given uniform words; returns sum of 2h."""
    assert s.flags.c_contiguous and s.dtype == np.int8
    w = np.ascontiguousarray(words, dtype=np.uint32)
    assert w.shape == s.shape
    return int(lib().oracle_half_sweep_words(_ptr(s, ctypes.c_int8), s.shape[0], int(c), int(T2), int(T4),
                                             _ptr(w, ctypes.c_uint32)))


def run(L: int, beta: float, seed: int, start: int = HOT, sweeps: int = 1, sweep0: int = 0,
        state: np.ndarray | None = None, check: bool = False):
    """Checkerboard Metropolis chain (Sec. 3.1, Algorithms 1-2): black then white per sweep.

    Returns (final state, M[sweeps], E[sweeps], incremental-energy mismatches).
    """
    _check_L(L)
    s = init(L, seed, start) if state is None else np.ascontiguousarray(state, dtype=np.int8).copy()
    M = np.zeros(sweeps, dtype=np.int64)
    E = np.zeros(sweeps, dtype=np.int64)
    mism = lib().oracle_run(_ptr(s, ctypes.c_int8), L, float(beta), int(seed), int(sweep0), int(sweeps),
                            _ptr(M, ctypes.c_int64), _ptr(E, ctypes.c_int64), 1 if check else 0)
    return s, M, E, int(mism)


def window(L: int, beta: float, seed: int, start: int, sweeps: int, i0: int, j0: int, h: int, w: int,
           sweep0: int = 0) -> np.ndarray:
    """Exact h x w window (rows i0.., cols j0.., torus-wrapped) after `sweeps` sweeps."""
    _check_L(L)
    out = np.empty((h, w), dtype=np.int8)
    rc = lib().oracle_window(L, float(beta), int(seed), int(start), int(sweep0), int(sweeps), int(i0), int(j0),
                             int(h), int(w), _ptr(out, ctypes.c_int8))
    if rc != 0:
        raise MemoryError("oracle window buffer")
    return out


def init_rows(s: np.ndarray, seed: int, start: int, row0: int, nrows: int) -> None:
    """Start state of rows [row0, row0 + nrows) of the full lattice s (in place)."""
    assert s.flags.c_contiguous and s.dtype == np.int8
    lib().oracle_init_rows(_ptr(s, ctypes.c_int8), s.shape[0], int(seed), int(start), int(row0), int(nrows))


def half_sweep_rows(s: np.ndarray, c: int, beta: float, seed: int, sweep: int, row0: int, nrows: int) -> int:
    """Colour-c half-sweep of rows [row0, row0 + nrows) only (timing samples)."""
    assert s.flags.c_contiguous and s.dtype == np.int8
    return int(lib().oracle_half_sweep_rows(_ptr(s, ctypes.c_int8), s.shape[0], int(c), float(beta), int(seed),
                                            int(sweep), int(row0), int(nrows)))


def lattice_hash(s: np.ndarray) -> str:
    """SHA-256 of the row-major lattice with +1 -> 0x01 and -1 -> 0x00 (2D or 3D),
    fed in slices of the first axis so that large lattices need no full-size copy."""
    a = np.asarray(s)
    h = hashlib.sha256()
    step = max(1, (1 << 28) // max(1, a[0].size))
    for i in range(0, a.shape[0], step):
        h.update((a[i:i + step] > 0).astype(np.uint8).tobytes())
    return h.hexdigest()


def moments_exact(M, E, N: int, burn_in: int) -> dict:
    """Sec. 4.1 observables over samples s >= burn_in, from exact integer sums.

    <|m|> = S1/(n N), <m^2> = S2/(n N^2), <m^4> = S4/(n N^4), <e> = SE/(n N),
    U4 = 1 - <m^4> / (3 <m^2>^2).  Evaluated as exact rationals, then rounded once.
    """
    Ms = [int(v) for v in M[burn_in:]]
    Es = [int(v) for v in E[burn_in:]]
    n = len(Ms)
    if n == 0:
        raise ValueError("no samples after burn-in")
    S1 = sum(abs(v) for v in Ms)
    S2 = sum(v * v for v in Ms)
    S4 = sum(v ** 4 for v in Ms)
    SE = sum(Es)
    SE2 = sum(v * v for v in Es)
    m1 = Fraction(S1, n * N)
    m2 = Fraction(S2, n * N * N)
    m4 = Fraction(S4, n * N ** 4)
    e1 = Fraction(SE, n * N)
    e2 = Fraction(SE2, n * N * N)
    binder = 1 - m4 / (3 * m2 * m2) if m2 != 0 else Fraction(0)
    return {"n": n, "S1": S1, "S2": S2, "S4": S4, "SE": SE, "SE2": SE2,
            "abs_m": float(m1), "m2": float(m2), "m4": float(m4), "e": float(e1), "e2": float(e2),
            "binder": float(binder)}


# ------------------------------------------------- three-dimensional torus
# The Sec. 3 Hamiltonian on the cubic lattice (d = 3) with the same checkerboard
# rules; see the header of ising3d_oracle.c.  Lattices are int8 arrays of shape
# (X, Y, Z), all extents even; the library's lattices are cubic, X = Y = Z = L.

def thresholds3d(beta: float) -> tuple[int, int, int]:
    """(T_2, T_4, T_6): min(2^32, ceil(exp(-2 beta h) 2^32)) for h = 2, 4, 6."""
    T = np.zeros(3, dtype=np.uint64)
    lib().oracle3d_thresholds(float(beta), _ptr(T, ctypes.c_uint64))
    return int(T[0]), int(T[1]), int(T[2])


def accept3d(h: int, x: int, T) -> bool:
    t = np.asarray(T, dtype=np.uint64)
    return bool(lib().oracle3d_accept(int(h), int(x), _ptr(t, ctypes.c_uint64)))


def site_word3d(dims, i: int, j: int, k: int, seed: int, sweep: int, c: int) -> int:
    X, Y, Z = dims
    return int(lib().oracle3d_site_word(X, Y, Z, i, j, k, seed, sweep, c))


def _check_dims(dims) -> tuple[int, int, int]:
    X, Y, Z = (int(v) for v in dims)
    if min(X, Y, Z) < 2 or X % 2 or Y % 2 or Z % 2:
        raise ValueError("the 3D oracle takes even extents >= 2")
    return X, Y, Z


def init3d(dims, seed: int, start: int = HOT) -> np.ndarray:
    X, Y, Z = _check_dims(dims)
    s = np.empty((X, Y, Z), dtype=np.int8)
    lib().oracle3d_init(_ptr(s, ctypes.c_int8), X, Y, Z, int(seed), int(start))
    return s


def observe3d(s: np.ndarray) -> tuple[int, int]:
    """(M, E) with M = sum sigma and E = H(sigma) over the 3N bonds."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    X, Y, Z = _check_dims(s.shape)
    M = ctypes.c_int64()
    E = ctypes.c_int64()
    lib().oracle3d_observe(_ptr(s, ctypes.c_int8), X, Y, Z, ctypes.byref(M), ctypes.byref(E))
    return M.value, E.value


def half_sweep_words3d(s: np.ndarray, c: int, T, words: np.ndarray) -> int:
    """One colour-c half-sweep with caller-given uniform words; returns sum of 2h."""
    assert s.flags.c_contiguous and s.dtype == np.int8
    X, Y, Z = _check_dims(s.shape)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    assert w.shape == s.shape
    t = np.asarray(T, dtype=np.uint64)
    return int(lib().oracle3d_half_sweep_words(_ptr(s, ctypes.c_int8), X, Y, Z, int(c), _ptr(t, ctypes.c_uint64),
                                               _ptr(w, ctypes.c_uint32)))


def run3d(dims, beta: float, seed: int, start: int = HOT, sweeps: int = 1, sweep0: int = 0,
          state: np.ndarray | None = None, check: bool = False):
    """3D checkerboard chain: returns (final state, M[sweeps], E[sweeps], mismatches)."""
    X, Y, Z = _check_dims(dims)
    s = init3d((X, Y, Z), seed, start) if state is None else np.ascontiguousarray(state, dtype=np.int8).copy()
    M = np.zeros(sweeps, dtype=np.int64)
    E = np.zeros(sweeps, dtype=np.int64)
    mism = lib().oracle3d_run(_ptr(s, ctypes.c_int8), X, Y, Z, float(beta), int(seed), int(sweep0), int(sweeps),
                              _ptr(M, ctypes.c_int64), _ptr(E, ctypes.c_int64), 1 if check else 0)
    return s, M, E, int(mism)


def window3d(dims, beta: float, seed: int, start: int, sweeps: int, origin, shape, sweep0: int = 0) -> np.ndarray:
    """Exact box of the 3D state after `sweeps` sweeps: shape (h, w, d) from origin
    (i0, j0, k0), torus-wrapped, index [a, b, c] = site (i0 + a, j0 + b, k0 + c)."""
    X, Y, Z = _check_dims(dims)
    h, w, d = (int(v) for v in shape)
    out = np.empty((h, w, d), dtype=np.int8)
    rc = lib().oracle3d_window(X, Y, Z, float(beta), int(seed), int(start), int(sweep0), int(sweeps),
                               *(int(v) for v in origin), h, w, d, _ptr(out, ctypes.c_int8))
    if rc != 0:
        raise MemoryError("oracle window buffer")
    return out


def _check_L(L: int) -> None:
    if L < 4 or L % 2:
        raise ValueError("the oracle takes even L >= 4")
