"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
symbol that include/gw.h declares, validates arguments, and builds the same
transform matrices as the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gw():
    import paper_1602_02313_gb300 as pkg
    from paper_1602_02313_gb300 import build as b
    b.build()
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    return sorted(set(re.findall(r"^(?:gw_status|const char\*|int64_t)\s+(gw_\w+)\(", src, re.M)))


def test_exports_every_declared_symbol(gw):
    lib = gw.load_library()
    names = _declared()
    assert len(names) >= 14
    assert sorted(gw.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("beta,ntau,nnu,nw", [(100.0, 16, 16, 16), (200.0, 48, 48, 48), (50.0, 24, 13, 20)])
def test_transform_matrices_match_oracle(gw, beta, ntau, nnu, nw):
    g = gi.make_grid(beta, ntau, nnu, nw, ncont=40)
    L = gw.transform_matrices(g)
    O = orc.transform_matrices(g)
    for k in ["B_fwd", "F_fwd", "F_cont", "B_bwd_re", "B_bwd_im", "F_bwd_re", "F_bwd_im"]:
        scale = np.abs(O[k]).max()
        assert np.abs(L[k] - O[k]).max() <= 1e-14 * scale, k


def test_invalid_arguments_rejected_on_host(gw):
    lib = gw.load_library()
    g = gi.make_grid(100.0, 16, 16, 16)
    keep = {}
    gs = gw._grid_struct(g, keep)
    # tau grid not closed under beta - tau
    bad = keep["tau"].copy()
    bad[0] *= 1.01
    gs.tau = bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.gw_transform_matrices(ctypes.byref(gs), None, None, None, None, None) == gw.GW_EINVAL
    gs = gw._grid_struct(g, keep)
    gs.npole = gs.ntau + 1
    assert lib.gw_transform_matrices(ctypes.byref(gs), None, None, None, None, None) == gw.GW_EINVAL
    # gw_create validates sizes before touching the GPU
    gs = gw._grid_struct(g, keep)
    kmq = np.zeros((1, 8), np.int32)
    v = np.ones((1, 40))
    s = gw._System(1, 8, 1, 16, 8, 40, 1.0, kmq.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0)   # ni = 40 not a multiple of 32
    h = ctypes.c_void_p()
    assert lib.gw_create(ctypes.byref(h), ctypes.byref(gs), ctypes.byref(s), 0, None) == gw.GW_EINVAL
    assert lib.gw_create(None, ctypes.byref(gs), ctypes.byref(s), 0, None) == gw.GW_EINVAL
    v32 = np.ones((1, 32))
    s = gw._System(1, 8, 1, 16, 8, 32, 1.0, kmq.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   v32.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0, 7)  # no M mode 7
    assert lib.gw_create(ctypes.byref(h), ctypes.byref(gs), ctypes.byref(s), 0, None) == gw.GW_EINVAL
    assert lib.gw_sync(None) == gw.GW_EINVAL
    assert lib.gw_set_stream(None, None) == gw.GW_EINVAL
    assert lib.gw_set_tuning(None, gw.GW_TUNE_POL_SEG_CHUNKS, 16) == gw.GW_EINVAL
    assert lib.gw_kernel_timing(None, 1) == gw.GW_EINVAL
    assert lib.gw_measure_alu(0, None, None) == gw.GW_EINVAL
    assert lib.gw_tau_to_freq_many(None, gw.GW_BOSE, gw.GW_TAU_TO_IW, 1, 1, None, gw.GW_FP64, None) == gw.GW_EINVAL
    assert lib.gw_screen_tau(None, 0, 3, None, None, None, None) == gw.GW_EINVAL
    assert lib.gw_dyson_tau(None, 1, 4, None, None, None, None, None, None) == gw.GW_EINVAL
    assert lib.gw_sigma_star(None, 1, None, 1, None, None) == gw.GW_EINVAL
    assert lib.gw_selfenergy_offdiag(None, 0, None, None, None, None, None) == gw.GW_EINVAL
    assert lib.gw_dyson_matrix(None, None, None, None, None, None, None, None) == gw.GW_EINVAL
    assert lib.gw_mlp_sync(None) == gw.GW_EINVAL
