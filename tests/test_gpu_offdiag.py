"""Off-diagonal self-energy (Eqs. sigc, sigx as full band matrices) on the GPU against the oracle,
and its diagonal against gw_selfenergy."""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc
from oracle import offdiag as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_offdiag_selfenergy_vs_oracle(gw):
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.3)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(43)
    c16 = dict(dtype=torch.complex128, device="cuda")
    S = torch.zeros((cr.nk, cr.nb, cr.nb, gr.ntau), **c16)
    Sx = torch.zeros((cr.nk, cr.nb, cr.nb), **c16)
    Sd = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
    Sxd = torch.zeros((cr.nk, cr.nb), dtype=torch.float64, device="cuda")
    Sref, Sxref = 0.0, 0.0
    for iq in range(cr.nq):
        X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
        W = -(X @ np.conj(np.swapaxes(X, 1, 2))) / cr.ni
        ctx.selfenergy_offdiag(iq, dev(G), dev(occ), dev(W), S, Sx)
        ctx.selfenergy(iq, dev(G), dev(occ), dev(W), Sd, Sxd, gw.GW_FP64)
        sc, sx = od.selfenergy_offdiag(gi.m_for_q(cr, iq), G, W, cr.v[iq], cr.kmq[iq], occ, omega=1.3)
        Sref, Sxref = Sref + sc, Sxref + sx
    ctx.sync()
    Sg, Sxg = S.cpu().numpy(), Sx.cpu().numpy()
    e, ex = rel(Sg, Sref), rel(Sxg, Sxref)
    d = np.arange(cr.nb)
    ed = rel(Sg[:, d, d, :].real, Sd.cpu().numpy())
    print(f"off-diagonal Sigma: GPU vs oracle {e:.1e} (Sigma^x {ex:.1e}); diagonal vs gw_selfenergy {ed:.1e}")
    assert e < 1e-10 and ex < 1e-10 and ed < 1e-12
    ctx.close()


def test_offdiag_selfenergy_chunked_rows(gw):
    """Nb = 64 and NI = 256 (the nk64_nb64 band and basis sizes): W~ a_j no longer fits beside the
    accumulator, so it is formed in chunks of rows (136 + a ragged 120); against the oracle."""
    import torch
    cr = gi.make_crystal(44, 2, 64, 32, 256, 60.0, qlist=[1])
    gr = gi.make_grid(60.0, 8, 8, 8, ncont=16)
    ctx = gw.GW(gr, cr, omega=1.3)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(45)
    X = rng.standard_normal((gr.ntau, cr.ni, 16)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 16))
    W = -(X @ np.conj(np.swapaxes(X, 1, 2))) / 16
    c16 = dict(dtype=torch.complex128, device="cuda")
    S = torch.zeros((cr.nk, cr.nb, cr.nb, gr.ntau), **c16)
    Sx = torch.zeros((cr.nk, cr.nb, cr.nb), **c16)
    ctx.selfenergy_offdiag(0, dev(G), dev(occ), dev(W), S, Sx)
    ctx.sync()
    sc, sx = od.selfenergy_offdiag(gi.m_for_q(cr, 0), G, W, cr.v[0], cr.kmq[0], occ, omega=1.3)
    e, ex = rel(S.cpu().numpy(), sc), rel(Sx.cpu().numpy(), sx)
    print(f"off-diagonal Sigma, NI 256 in row chunks: {e:.1e} (Sigma^x {ex:.1e})")
    assert e < 1e-10 and ex < 1e-10
    ctx.close()
