"""The batched workload's crystal shapes against the oracle: for each distinct (Nb, NI) of
gwinputs.batch_crystals() -- (96, 384), (64, 256) at Nk = 27, (128, 512), (32, 128) -- the
polarization (Eq. irpol) and the correlation self-energy (Eq. sigc) of one q, on the FP64 path
and on the tensor cores, against the oracle at sampled tau (and sampled k for Sigma^c). These are
the NI = 384 and 512 shapes that the chain comparisons at small sizes do not reach.

Tolerances: FP64 path 1e-10 relative (max norm over the sample); tensor cores 2e-5 (22-bit split
operands, FP32 accumulation in K segments)."""
import functools

import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_TC = 2e-5


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


@functools.lru_cache(maxsize=1)
def _shapes():
    """The first crystal of each distinct (Nb, NI) of the batched workload (built on first use:
    the twelve grids take seconds, too long for collection)."""
    seen, out = set(), []
    for cr, gr in gi.batch_crystals():
        if (cr.nb, cr.ni) not in seen:
            seen.add((cr.nb, cr.ni))
            out.append((cr, gr))
    return out


N_SHAPES = 4   # (96, 384), (64, 256), (128, 512), (32, 128); checked in the test


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("idx", range(N_SHAPES), ids=[f"shape{i}" for i in range(N_SHAPES)])
def test_batch_shape_vs_oracle(gw, idx):
    import torch
    shapes = _shapes()
    assert len(shapes) == N_SHAPES
    cr, gr = shapes[idx]
    iq = 1
    sub = gi.subset_q(cr, iq, 1)                  # one q; the generator counter stays q = 1
    ctx = gw.GW(gr, sub, omega=gi.OMEGA_SI, q0=iq, m_mode=1)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    Gd, occd = torch.from_numpy(G).cuda(), torch.from_numpy(occ).cuda()
    its = [0, gr.ntau // 2, gr.ntau - 1]
    ks = [0, cr.nk - 1]
    M = gi.m_for_q(cr, iq)
    Pr = orc.polarization(M, G, cr.kmq[iq], omega=gi.OMEGA_SI, its=its)
    rng = np.random.default_rng(idx)
    X = rng.standard_normal((gr.ntau, cr.ni, 8)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 8))
    W = -30.0 * (X @ np.conj(np.swapaxes(X, 1, 2))) / 8           # Hermitian, like W~(tau)
    Sr, _, _ = orc.selfenergy(M[ks], G, W, cr.v[iq], cr.kmq[iq], occ, omega=gi.OMEGA_SI, ks=ks, its=its)
    Wd = torch.from_numpy(W).cuda()
    errs = {}
    for name, prec, tol in [("fp64", gw.GW_FP64, TOL), ("fp16x2", gw.GW_FP16X2, TOL_TC)]:
        P = torch.zeros((gr.ntau, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
        S = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
        ctx.polarization(0, Gd, P, prec)
        ctx.selfenergy(0, Gd, occd, Wd, S, None, prec)
        ctx.sync()
        eP = rel(P.cpu().numpy()[its], Pr)
        Sg = S.cpu().numpy()
        eS = max(rel(Sg[k][:, its], Sr[k][:, its]) for k in ks)
        errs[name] = (eP, eS)
        assert eP < tol and eS < tol, (name, eP, eS)
    print(f"Nb {cr.nb} NI {cr.ni} Nk {cr.nk} Ntau {gr.ntau}: P fp64 {errs['fp64'][0]:.1e} tc {errs['fp16x2'][0]:.1e}; "
          f"Sigma^c fp64 {errs['fp64'][1]:.1e} tc {errs['fp16x2'][1]:.1e}")
    ctx.close()
