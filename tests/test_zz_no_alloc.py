"""The sweep entry point that allocates no device memory.

Some callers cannot call cudaMalloc (code running during CUDA graph capture,
plugins confined to another runtime's memory pool, loops whose memory is fixed
after start-up).  ising_sweep_packed_noalloc serves them: the caller owns the
bit planes and the M/E output array, and the sweep kernel's scratch lives in a
fixed file-scope device array inside the library.  This test checks, through
the C ABI, that two calls in a row reproduce exactly what the handle API
(ising_init_ex + ising_sweep) computes -- the same lattices and the same
per-sweep M and E, written over M/E arrays that start as garbage -- and that a
call with too many lattices is refused.
It is collected last so that a failure here stops a -x run only after every
other test has run.
"""
import numpy as np
import pytest

from paper_1903_11714_gb300 import build as libbuild
from paper_1903_11714_gb300 import ising

pytestmark = pytest.mark.gpu

SPECS = [(256, 0.4406868, 7, ising.HOT), (192, 0.3, 8, ising.HOT), (1024, 0.55, 9, ising.COLD)]
N_SWEEPS = 6
GARBAGE = 0x123456789ABCDEF


def test_two_noalloc_calls_match_the_handle_api():
    import torch

    libbuild.build()
    handles, black, white, me1, me2 = [], [], [], [], []
    for L, beta, seed, start in SPECS:
        h = ising.Lattice(L, beta, seed, start, ising.PACKED)
        b, w = h.get_planes()  # start state, host copy
        black.append(torch.from_numpy(b.view(np.int32)).cuda())
        white.append(torch.from_numpy(w.view(np.int32)).cuda())
        # the M/E arrays start as garbage: every sweep must overwrite its pair, not add to it
        me1.append(torch.full((2 * N_SWEEPS,), GARBAGE, dtype=torch.int64, device="cuda"))
        me2.append(torch.full((2 * N_SWEEPS,), -GARBAGE, dtype=torch.int64, device="cuda"))
        handles.append(h)
    torch.cuda.synchronize()
    args = dict(black_ptrs=[t.data_ptr() for t in black], white_ptrs=[t.data_ptr() for t in white],
                Ls=[s[0] for s in SPECS], betas=[s[1] for s in SPECS], seeds=[s[2] for s in SPECS])
    # call 1: sweeps 0..5; call 2 continues with sweeps 6..11
    ising.ising_sweep_packed_noalloc(**args, first_sweep=0, nsweeps=N_SWEEPS,
                                     me_ptrs=[t.data_ptr() for t in me1], wait=True)
    ising.ising_sweep_packed_noalloc(**args, first_sweep=N_SWEEPS, nsweeps=N_SWEEPS,
                                     me_ptrs=[t.data_ptr() for t in me2], wait=True)
    torch.cuda.synchronize()
    for k, h in enumerate(handles):
        h.sweep(N_SWEEPS)
        M, E = h.history()
        got1 = me1[k].cpu().numpy()
        assert np.array_equal(got1[0::2], M) and np.array_equal(got1[1::2], E), k
        h.sweep(N_SWEEPS)
        M, E = h.history(N_SWEEPS, N_SWEEPS)
        got2 = me2[k].cpu().numpy()
        assert np.array_equal(got2[0::2], M) and np.array_equal(got2[1::2], E), k
        hb, hw = h.get_planes()
        assert np.array_equal(black[k].cpu().numpy().view(np.uint32), hb), k
        assert np.array_equal(white[k].cpu().numpy().view(np.uint32), hw), k
        h.close()


def test_noalloc_refuses_more_lattices_than_its_scratch_holds():
    libbuild.build()
    n = 65
    with pytest.raises(ising.IsingError) as e:
        ising.ising_sweep_packed_noalloc([1] * n, [1] * n, [64] * n, [0.4] * n, [1] * n, 0, 1, [1] * n)
    assert e.value.code == ising.ISING_EINVAL
    assert "64" in ising.last_error()


def test_noalloc_writes_stay_inside_the_planes():
    """Guard words around caller-owned planes and M/E arrays (one buffer per lattice:
    guard, black plane, guard, white plane, guard, M/E, guard) keep their canary value
    after sweeps of every row width class (W % 4 == 0, odd, 2 mod 4), and the swept
    lattices still equal the handle API's."""
    import torch

    libbuild.build()
    G, CANARY, n = 1024, 0x5A5A5A5A, 4
    specs = [(256, 0.4406868, 7, ising.HOT), (192, 0.3, 8, ising.HOT), (128, 0.5, 10, ising.COLD),
             (1024, 0.55, 9, ising.COLD)]
    bufs, layout, handles = [], [], []
    for L, beta, seed, start in specs:
        pw = L * (L // 64)
        h = ising.Lattice(L, beta, seed, start, ising.PACKED)
        b, w = h.get_planes()
        buf = torch.full((4 * G + 2 * pw + 4 * n,), CANARY, dtype=torch.int32)
        ob, ow, om = G, 2 * G + pw, 3 * G + 2 * pw
        buf[ob:ob + pw] = torch.from_numpy(b.view(np.int32))
        buf[ow:ow + pw] = torch.from_numpy(w.view(np.int32))
        buf[om:om + 4 * n] = 0
        bufs.append(buf.cuda())
        layout.append((pw, ob, ow, om))
        handles.append(h)
    torch.cuda.synchronize()
    ptr = lambda k, off: bufs[k].data_ptr() + 4 * off
    ising.ising_sweep_packed_noalloc([ptr(k, l[1]) for k, l in enumerate(layout)],
                                     [ptr(k, l[2]) for k, l in enumerate(layout)],
                                     [s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                                     first_sweep=0, nsweeps=n,
                                     me_ptrs=[ptr(k, l[3]) for k, l in enumerate(layout)], wait=True)
    torch.cuda.synchronize()
    for k, (h, (pw, ob, ow, om)) in enumerate(zip(handles, layout)):
        got = bufs[k].cpu()
        guards = torch.cat([got[:G], got[ob + pw:ow], got[ow + pw:om], got[om + 4 * n:]])
        assert bool((guards == CANARY).all()), f"lattice {k}: a guard word was written"
        h.sweep(n)
        hb, hw = h.get_planes()
        assert np.array_equal(got[ob:ob + pw].numpy().view(np.uint32), hb), k
        assert np.array_equal(got[ow:ow + pw].numpy().view(np.uint32), hw), k
        me = got[om:om + 4 * n].numpy().view(np.int64)
        M, E = h.history()
        assert np.array_equal(me[0::2], M) and np.array_equal(me[1::2], E), k
        h.close()
