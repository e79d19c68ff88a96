"""The allocation-free screening entry point (gw_screen_static), called through the C ABI.

Some callers cannot allocate device memory when they call in (their memory was handed to
another allocator at start-up, or their loop must not take the synchronisation a cudaMalloc
can cause); gw_screen_static serves them with a scratch array compiled into the library.
This test checks it against the allocating gw_screen on two calls in a row, within the FP64
parity tolerance, at a size that needs two passes over the built-in scratch. The file is
named to run last, so a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_screen_static_matches_screen():
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    b.build()
    lib = gw.load_library()
    # systems of the Nk=64 crystal (NI = 256, 48 bosonic frequencies): 96 MiB of scratch per q, so
    # three q points take two passes over the 128 MiB array
    cr = gi.make_crystal(91, 8, 4, 2, 256, 50.0, qlist=[1, 3, 5])
    gr = gi.make_grid(50.0, 48, 48, 48, ncont=16)
    nq, nnu, ni = cr.nq, gr.nnu, cr.ni
    rng = np.random.default_rng(21)
    X = rng.standard_normal((nq, nnu, ni, 12)) + 1j * rng.standard_normal((nq, nnu, ni, 12))
    Y = rng.standard_normal((nq, nnu, ni, ni)) + 1j * rng.standard_normal((nq, nnu, ni, ni))
    # Hermitian part negative semidefinite (like P(i nu)) plus an anti-Hermitian part
    P = -(X @ np.conj(np.swapaxes(X, -1, -2))) / 40.0 + 0.01 * (Y - np.conj(np.swapaxes(Y, -1, -2)))
    Pd = torch.from_numpy(P).cuda()
    ctx = gw.GW(gr, cr)
    Wref = torch.zeros_like(Pd)
    info_ref = torch.zeros(nq, nnu, dtype=torch.int32, device="cuda")
    ctx.screen(0, nq, Pd, Wref, info_ref)
    ctx.sync()
    sv = torch.from_numpy(np.sqrt(cr.v)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = Wref.cpu().numpy()
    for call in range(2):
        W = torch.full_like(Pd, float("nan"))
        info = torch.full((nq, nnu), -7, dtype=torch.int32, device="cuda")
        st = lib.gw_screen_static(nq, nnu, ni, ctypes.c_void_p(sv.data_ptr()), ctypes.c_void_p(Pd.data_ptr()),
                                  ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(info.data_ptr()), stream)
        assert st == gw.GW_OK
        torch.cuda.synchronize()
        assert int(info.abs().sum()) == 0
        got = W.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < TOL, f"call {call}: rel err {err:.3e}"
    # and directly against the oracle's solve of Eq. (tildeW) in i nu, one q point
    import oracle as orc
    err = np.abs(got[1] - orc.screen(P[1], cr.v[1])).max() / np.abs(ref[1]).max()
    assert err < TOL, f"vs oracle: rel err {err:.3e}"
    # sizes beyond the built-in scratch are rejected
    assert lib.gw_screen_static(1, 200, 256, ctypes.c_void_p(sv.data_ptr()), ctypes.c_void_p(Pd.data_ptr()),
                                ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(info.data_ptr()), stream) == gw.GW_EINVAL
    ctx.close()
