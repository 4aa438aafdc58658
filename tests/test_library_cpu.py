"""Host-side checks of the CUDA library that need no GPU.

* The library builds for sm_103a, loads, and exports every function that
  include/ising.h declares (and the binding binds exactly those).
* ising_thresholds (host-only) equals the oracle's independently written
  thresholds bit for bit (the FP64 libm reading of the acceptance rule).
* Argument validation rejects bad input before touching the device, including
  damaged checkpoint headers and ranges whose sums would wrap.
* Without a device the product path reports ISING_ECUDA (there is no CPU
  fallback), and a missing library is an error.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ising.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ising_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ising.lib()


def test_header_declares_the_boundary_entry_points():
    names = header_functions()
    for required in ("ising_init", "ising_sweep", "ising_observables", "ising_history", "ising_moments",
                     "ising_get_lattice", "ising_set_lattice", "ising_thresholds", "ising_free",
                     "ising_last_error", "ising_batch_create", "ising_batch_run", "ising_batch_observables"):
        assert required in names


def test_header_signatures_of_the_boundary_calls():
    """The calls of the hot path's C boundary take exactly these parameters."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"\s+", " ", text)
    want = [
        "int ising_init(ising_t *out, int64_t L, double beta, uint64_t seed);",
        "int ising_init_ex(ising_t *out, int64_t L, double beta, uint64_t seed, int start, int kernel, void *stream);",
        "int ising_sweep(ising_t h, int64_t n);",
        "int ising_observables(ising_t h, int64_t *M, int64_t *E, int64_t *sweeps_done);",
        "int ising_history(ising_t h, int64_t first, int64_t count, int64_t *M, int64_t *E);",
        "int ising_moments(ising_t h, int64_t burn_in, double *abs_m, double *m2, double *m4, double *e, "
        "double *binder);",
        "int ising_get_lattice(ising_t h, int8_t *out);",
        "int ising_set_lattice(ising_t h, const int8_t *in);",
        "int ising_thresholds(double beta, uint64_t T[2]);",
        "int ising_free(ising_t h);",
        "const char *ising_last_error(void);",
        "int ising_batch_create(ising_batch_t *out, int32_t count, const int64_t *L, const double *beta, "
        "const uint64_t *seed, const int32_t *start);",
        "int ising_batch_run(ising_batch_t b, int64_t sweeps, int32_t graph_sweeps);",
        "int ising_batch_observables(ising_batch_t b, int32_t idx, int64_t *M, int64_t *E);",
    ]
    for sig in want:
        assert sig in text, sig


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s(ising_\w+)", out.stdout))
    declared = set(header_functions())
    assert declared <= exported, declared - exported
    assert set(ising.EXPORTS) == declared, set(ising.EXPORTS) ^ declared
    for name in declared:
        assert hasattr(lib, name)


@pytest.mark.parametrize("beta", [0.0, 1e-7, 0.2, 0.35, 0.4406868, 0.44068679350977151, 0.5, 0.6, 1.3, 7.0,
                                  50.0, 200.0])
def test_thresholds_match_oracle(lib, beta):
    assert ising.ising_thresholds(beta) == oracle.thresholds(beta)


def test_thresholds_many_betas_match_oracle(lib):
    rng = np.random.default_rng(1)
    for beta in rng.uniform(0.0, 3.0, size=2000):
        assert ising.ising_thresholds(beta) == oracle.thresholds(beta), beta


@pytest.mark.parametrize("beta", [-0.1, float("nan"), float("inf")])
def test_thresholds_reject_bad_beta(lib, beta):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_thresholds(beta)
    assert e.value.code == ising.ISING_EINVAL
    assert "beta" in ising.last_error()


@pytest.mark.parametrize("L,kernel", [(0, ising.PACKED), (96, ising.PACKED), (32, ising.PACKED),
                                      (12, ising.INT8), (4, ising.INT8), (2**21, ising.PACKED),
                                      # above 2^20, or rows too long for a whole-row tile when
                                      # L % 256 != 0 (no column blocks then): above 102,336
                                      ((1 << 20) + 256, ising.PACKED), (102_336 + 128, ising.PACKED),
                                      (185_408, ising.PACKED)])
def test_init_rejects_bad_sizes_before_device_work(lib, L, kernel):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_init_ex(L, 0.44, 1, ising.HOT, kernel)
    assert e.value.code == ising.ISING_EINVAL


def test_init_rejects_bad_start_and_kernel(lib):
    for start, kernel in ((7, ising.PACKED), (ising.HOT, 9)):
        with pytest.raises(ising.IsingError) as e:
            ising.ising_init_ex(64, 0.44, 1, start, kernel)
        assert e.value.code == ising.ISING_EINVAL


def test_thresholds3d_match_oracle(lib):
    rng = np.random.default_rng(2)
    for beta in np.concatenate([rng.uniform(0.0, 3.0, size=1000), [0.0, 0.2216546, 200.0]]):
        T = ising.ising_thresholds3d(float(beta))
        assert T == oracle.thresholds3d(float(beta)), beta
        assert T[:2] == ising.ising_thresholds(float(beta))


@pytest.mark.parametrize("L,start", [(0, ising.HOT), (96, ising.HOT), (32, ising.HOT), (16384, ising.HOT),
                                     (64, 7)])
def test_init3d_rejects_bad_arguments_before_device_work(lib, L, start):
    with pytest.raises(ising.IsingError) as e:
        ising.ising_init3d(L, 0.22, 1, start)
    assert e.value.code == ising.ISING_EINVAL
    with pytest.raises(ising.IsingError):
        ising.ising_thresholds3d(float("nan"))


def test_null_handles_are_rejected(lib):
    assert lib.ising_sweep(None, 1) == ising.ISING_EINVAL
    assert lib.ising_free(None) == ising.ISING_OK
    assert lib.ising_batch_free(None) == ising.ISING_OK
    M = ctypes.c_int64()
    assert lib.ising_observables(None, ctypes.byref(M), None, None) == ising.ISING_EINVAL


def test_version_string(lib):
    assert "sm_103a" in lib.ising_version().decode()


def checkpoint_header(L=128, kernel=ising.PACKED, start=ising.HOT, sweeps_done=0, lattice_bytes=None,
                      magic=b"ISINGCK1", version=1, beta=0.44, seed=1):
    """The 72-byte checkpoint header of ising_save: magic, then version, L, kernel,
    start, sweeps done and lattice bytes (int64), beta (double), seed (uint64)."""
    import struct
    if lattice_bytes is None:
        lattice_bytes = L * L if kernel == ising.INT8 else L * L // 8
    return struct.pack("<8s6qdQ", magic, version, L, kernel, start, sweeps_done, lattice_bytes, beta, seed)


@pytest.mark.parametrize("fields,extra", [
    (dict(magic=b"ISINGCK2"), 4096),
    (dict(version=2), 4096),
    (dict(kernel=7), 4096),
    (dict(kernel=-1), 4096),
    (dict(start=5), 4096),
    (dict(sweeps_done=-1), 4096),             # would size a negative history copy
    (dict(sweeps_done=1 << 40), 4096),        # beyond the 32-bit sweep counter
    (dict(sweeps_done=(1 << 63) // 16), 4096),  # 16 * sweeps_done wraps a 64-bit size
    (dict(lattice_bytes=-8), 4096),
    (dict(lattice_bytes=1 << 62), 4096),
    (dict(), 100),                            # planes of 2 KB cut short
])
def test_damaged_checkpoints_are_rejected_before_device_work(lib, fields, extra):
    """A damaged header is refused with EINVAL before any handle or device memory
    exists (on a machine without a GPU, reaching the device would report ECUDA)."""
    blob = checkpoint_header(**fields) + bytes(extra)
    buf = ctypes.create_string_buffer(blob, len(blob))
    h = ctypes.c_void_p()
    rc = lib.ising_load(ctypes.byref(h), buf, len(blob), None)
    assert rc == ising.ISING_EINVAL, (fields, rc, lib.ising_last_error())
    assert h.value is None
    assert lib.ising_load(ctypes.byref(h), buf, 40, None) == ising.ISING_EINVAL


@pytest.mark.parametrize("first,n", [(-1, 1), (0, -1), (0xFFFFFFFE, 1), (1, 0xFFFFFFFE),
                                     (1 << 62, 1 << 62), ((1 << 63) - 10, 20)])
def test_noalloc_sweep_range_is_checked_before_device_work(lib, first, n):
    """Sweep numbers must stay in 0 .. 2^32 - 2 (the 32-bit Philox sweep word);
    ranges whose end passes it -- including sums that wrap a signed 64-bit integer --
    are refused with EINVAL before any device work (which here would give ECUDA)."""
    vp1 = ctypes.c_void_p * 1
    planes = (ctypes.c_uint32 * 2048)()
    me = (ctypes.c_int64 * 64)()
    black = vp1(ctypes.cast(planes, ctypes.c_void_p))
    mes = vp1(ctypes.cast(me, ctypes.c_void_p))
    L = (ctypes.c_int64 * 1)(256)
    beta = (ctypes.c_double * 1)(0.44)
    seed = (ctypes.c_uint64 * 1)(1)
    rc = lib.ising_sweep_packed_noalloc(1, black, black, L, beta, seed, first, n, mes, None, 0)
    assert rc == ising.ISING_EINVAL, (first, n, rc, lib.ising_last_error())


def test_product_path_fails_loudly_without_a_device(lib):
    """No CPU fallback: where there is no GPU, creating a lattice or a batch reports
    the CUDA failure instead of running the sweep anywhere else."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for make in (lambda: ising.Lattice(128, 0.44, 1), lambda: ising.Lattice(128, 0.44, 1, ising.HOT, ising.INT8),
                 lambda: ising.Lattice3D(64, 0.22, 1), lambda: ising.Batch(2, 256, 1 << 20)):
        with pytest.raises(ising.IsingError) as e:
            make()
        assert e.value.code == ising.ISING_ECUDA


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    monkeypatch.setattr(ising, "_lib", None)
    monkeypatch.setattr(ising, "LIB_PATH", str(tmp_path / "libising_gb300.so"))
    with pytest.raises(RuntimeError, match="missing"):
        ising.lib()


def no_device_or_skip(lib):
    """The size sweeps below rely on accepted sides failing at the first device call;
    where a device answers, they would allocate up to 128 GB, so they skip."""
    h = ctypes.c_void_p()
    rc = lib.ising_init_ex(ctypes.byref(h), 64, 0.44, 1, ising.HOT, ising.PACKED, None)
    if rc == ising.ISING_OK:
        lib.ising_free(h)
    if rc != ising.ISING_ECUDA:
        pytest.skip("a device is present")


def test_accepted_sides_are_exactly_the_documented_ones(lib):
    """Every side up past each limit: EINVAL (before device work) exactly where
    include/ising.h says the side is outside the kernel's range; any other side gets
    as far as the device (ECUDA here).  Packed: L % 64 == 0, 64 <= L, and L <= 2^20
    when L % 256 == 0, else L <= 102,336.  int8: L % 8 == 0, 8 <= L <= 131,072.
    Cubic: L % 64 == 0, 64 <= L <= 8,192."""
    no_device_or_skip(lib)
    h = ctypes.c_void_p()

    def packed_ok(L):
        return L % 64 == 0 and L >= 64 and (L <= 1 << 20 if L % 256 == 0 else L <= 102_336)

    def int8_ok(L):
        return L % 8 == 0 and 8 <= L <= 131_072

    def cubic_ok(L):
        return L % 64 == 0 and 64 <= L <= 8192

    cases = [(ising.PACKED, packed_ok, list(range(-64, (1 << 20) + 2048, 32)) + [65, 100, 102_400 + 1]),
             (ising.INT8, int8_ok, list(range(-8, 131_072 + 256, 4)) + [9, 130_000 + 1])]
    for kernel, ok, sides in cases:
        for L in sides:
            rc = lib.ising_init_ex(ctypes.byref(h), L, 0.44, 1, ising.HOT, kernel, None)
            assert rc == (ising.ISING_ECUDA if ok(L) else ising.ISING_EINVAL), (kernel, L, rc)
    for L in list(range(-64, 8192 + 1024, 32)) + [65, 1 << 20]:
        rc = lib.ising_init3d(ctypes.byref(h), L, 0.22, 1, ising.HOT, None)
        assert rc == (ising.ISING_ECUDA if cubic_ok(L) else ising.ISING_EINVAL), ("cubic", L, rc)
    assert h.value is None


def test_batch_create_ex_arguments(lib):
    """ising_batch_create_ex: EINVAL unless 1 <= capacity <= 2^20, max_L a multiple of 64
    in 64 .. 2^20, threads in {0, 128, 256, 512} and arena_bytes >= 256; valid
    arguments get as far as the device."""
    no_device_or_skip(lib)
    b = ctypes.c_void_p()
    good = dict(capacity=4, max_L=1024, arena=1 << 20, threads=0)
    bad = [dict(capacity=0), dict(capacity=(1 << 20) + 1), dict(max_L=0), dict(max_L=100), dict(max_L=32),
           dict(max_L=(1 << 20) + 64), dict(threads=64), dict(threads=300), dict(threads=1024), dict(arena=255)]
    for change in bad + [dict()] + [dict(threads=t) for t in (128, 256, 512)] + [dict(max_L=1 << 20, capacity=1 << 20)]:
        a = {**good, **change}
        rc = lib.ising_batch_create_ex(ctypes.byref(b), a["capacity"], a["max_L"], a["arena"], a["threads"], None)
        assert rc == (ising.ISING_EINVAL if change in bad else ising.ISING_ECUDA), (change, rc)
    assert b.value is None


def test_batch_create_from_arrays_arguments(lib):
    """ising_batch_create (the array form): EINVAL, before any device work, for a
    null array, count outside 1 .. 2^20, or any lattice whose L is not a packed side,
    whose beta is not finite and >= 0, or whose start is neither hot nor cold (the
    message names the lattice); valid arrays get as far as the device."""
    no_device_or_skip(lib)
    b = ctypes.c_void_p()

    def call(Ls, betas=None, starts=None, count=None, null=None):
        n = len(Ls)
        arrs = [(ctypes.c_int64 * n)(*Ls), (ctypes.c_double * n)(*(betas or [0.44] * n)),
                (ctypes.c_uint64 * n)(*range(n)), (ctypes.c_int32 * n)(*(starts or [ising.HOT] * n))]
        if null is not None:
            arrs[null] = None
        return lib.ising_batch_create(ctypes.byref(b), n if count is None else count, *arrs)

    assert call([256, 512, 64]) == ising.ISING_ECUDA
    assert call([256, 512, 64], starts=[ising.HOT, ising.COLD, ising.COLD]) == ising.ISING_ECUDA
    for null in range(4):
        assert call([256], null=null) == ising.ISING_EINVAL
    assert call([256], count=0) == ising.ISING_EINVAL
    assert call([256], count=-3) == ising.ISING_EINVAL
    for L in (0, 32, 100, 65, 1 << 21, 102_464):
        assert call([256, L, 64]) == ising.ISING_EINVAL, L
        assert "lattice 1" in ising.last_error()
    for beta in (float("nan"), float("inf"), -0.1):
        assert call([256, 256], betas=[0.4, beta]) == ising.ISING_EINVAL
    assert call([256, 256], starts=[ising.HOT, 2]) == ising.ISING_EINVAL
    assert b.value is None


def test_noalloc_lattice_arguments(lib):
    """ising_sweep_packed_noalloc: per-lattice sides as documented (L % 64 == 0,
    64 <= L, L <= 163,840 when L % 256 == 0, else L <= 102,336), finite beta >= 0,
    non-null pointers and 1 <= count <= 64 -- all checked before device work."""
    no_device_or_skip(lib)
    vp = ctypes.c_void_p
    buf = (ctypes.c_uint32 * 16)()
    p = ctypes.cast(buf, vp)

    def call(Ls, betas=None, count=None, null_plane=False):
        n = len(Ls)
        planes = (vp * n)(*([None] if null_plane else []) + [p] * (n - int(null_plane)))
        mes = (vp * n)(*[p] * n)
        Larr = (ctypes.c_int64 * n)(*Ls)
        barr = (ctypes.c_double * n)(*(betas or [0.44] * n))
        sarr = (ctypes.c_uint64 * n)(*range(n))
        return lib.ising_sweep_packed_noalloc(n if count is None else count, planes, planes, Larr, barr, sarr,
                                             0, 1, mes, None, 0)

    def ok(L):
        return L % 64 == 0 and L >= 64 and (L <= 163_840 if L % 256 == 0 else L <= 102_336)

    for L in list(range(-64, 200_000, 32)) + [1 << 20, (1 << 20) + 64]:
        assert call([L]) == (ising.ISING_ECUDA if ok(L) else ising.ISING_EINVAL), L
    assert call([256, 100]) == ising.ISING_EINVAL          # any bad lattice refuses the call
    for beta in (float("nan"), float("inf"), -0.1):
        assert call([256], betas=[beta]) == ising.ISING_EINVAL
    assert call([256], betas=[0.0]) == ising.ISING_ECUDA
    assert call([256, 512], null_plane=True) == ising.ISING_EINVAL
    assert call([256], count=0) == ising.ISING_EINVAL
    assert call([256] * 65) == ising.ISING_EINVAL
    assert call([256] * 64) == ising.ISING_ECUDA


def test_specialize_mode_arguments(lib):
    """ising_set_specialize takes OFF, AUTO or ALWAYS only; ising_specialized needs a
    handle.  Both are host-only."""
    for mode in (ising.SPECIALIZE_OFF, ising.SPECIALIZE_ALWAYS, ising.SPECIALIZE_AUTO):
        assert lib.ising_set_specialize(mode) == ising.ISING_OK
    for mode in (-1, 3, 100):
        assert lib.ising_set_specialize(mode) == ising.ISING_EINVAL
    flag = ctypes.c_int32(7)
    assert lib.ising_specialized(None, ctypes.byref(flag), None, 0) == ising.ISING_EINVAL
    assert flag.value == 7


def test_batch_gather_arguments(lib):
    """ising_batch_gather refuses a null batch before touching the device."""
    idx = (ctypes.c_int32 * 1)(0)
    out = (ctypes.c_int64 * 3)()
    assert lib.ising_batch_gather(None, 1, idx, out) == ising.ISING_EINVAL
    assert list(out) == [0, 0, 0]


def test_batch_cluster_arguments(lib):
    """ising_batch_set_cluster and ising_batch_cluster_size refuse a null batch (and
    the mode constants agree with the header's)."""
    assert (ising.CLUSTER_OFF, ising.CLUSTER_AUTO, ising.CLUSTER_ALWAYS) == (0, 1, 2)
    for mode in (0, 1, 2, 3):
        assert lib.ising_batch_set_cluster(None, mode) == ising.ISING_EINVAL
    c = ctypes.c_int32(5)
    assert lib.ising_batch_cluster_size(None, ctypes.byref(c)) == ising.ISING_EINVAL
    assert c.value == 5
    with open(os.path.join(ROOT, "include", "ising.h")) as f:
        header = f.read()
    for name, v in (("OFF", 0), ("AUTO", 1), ("ALWAYS", 2)):
        assert f"#define ISING_CLUSTER_{name} {v}" in header
