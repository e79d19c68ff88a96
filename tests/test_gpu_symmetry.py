"""Crystal-symmetry reduction (Sec. III.C) on the GPU: the G0W0 chain over the irreducible q
points of a synthetic Oh crystal, each q's self-energy carried to its star (gw_sigma_star),
against the same chain over every q of the mesh."""
import numpy as np
import pytest

import gwinputs as gi
from gwinputs import symmetric as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def _chain(gw, c, gr, qs, prec, star=None):
    import torch
    from paper_1602_02313_gb300.driver import Chain
    cq = sy.restrict_q(c, qs)
    M = torch.from_numpy(cq.M).cuda()
    ctx = gw.GW(gr, cq, omega=2.0, M=M)
    kinv = None if star is None else [torch.from_numpy(star[q]).cuda() for q in qs]
    ch = Chain(ctx, torch.from_numpy(c.eps).cuda(), prec=prec, qb=len(qs), cont_method=gw.GW_CPE, star=kinv,
               screen_prec=gw.GW_FP64 if prec == gw.GW_FP64 else None)
    ch.step()
    ch.check()
    out = tuple(t.cpu().numpy().copy() for t in (ch.S, ch.Sx, ch.eqp))
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_irreducible_chain_equals_full_chain(gw, prec):
    p = {"fp64": gw.GW_FP64, "fp16x2": gw.GW_FP16X2}[prec]
    c = sy.make_symmetric_crystal(n=2, nb=8, nocc=4, beta=50.0, seed=11)
    gr = gi.make_grid(c.beta, 16, 16, 16, ncont=64)
    star = {q: sy.star_kinv(c, q) for q in c.ibz}
    S_full, Sx_full, E_full = _chain(gw, c, gr, list(range(c.nq)), p)
    S_red, Sx_red, E_red = _chain(gw, c, gr, c.ibz, p, star)
    eS = np.abs(S_red - S_full).max() / np.abs(S_full).max()
    eX = np.abs(Sx_red - Sx_full).max() / np.abs(Sx_full).max()
    dE = np.abs(E_red - E_full).max()
    print(f"symmetry ({prec}): {len(c.ibz)} of {c.nq} q; Sigma^c {eS:.1e}, Sigma^x {eX:.1e}, max |dE_qp| {dE:.1e} Ha")
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert eS < tol and eX < tol
    assert dE < (1e-9 if prec == "fp64" else 1e-5)
