"""Crystal-symmetry reduction (Sec. III.C) on the GPU: the G0W0 chain over the irreducible q
points of a synthetic Oh crystal, each q's self-energy carried to its star (gw_sigma_star),
against the oracle's sum over every q of the mesh and against the same GPU chain over every q;
gw_sigma_star itself against the oracle's star sum."""
import functools

import numpy as np
import pytest

import gwinputs as gi
import oracle as orc
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


def _crystal():
    c = sy.make_symmetric_crystal(n=2, nb=8, nocc=4, beta=50.0, seed=11)
    gr = gi.make_grid(c.beta, 16, 16, 16, ncont=64)
    return c, gr


@functools.lru_cache(maxsize=1)
def _oracle_full_sum():
    """The oracle's G0W0 Sigma^c(tau), Sigma^x summed over every q of the mesh (Eqs. sigc, sigx)."""
    c, gr = _crystal()
    G, occ = orc.green_tau0(c.eps, gr.tau, gr.beta)
    Sc, Sx = 0.0, 0.0
    for q in range(c.nq):
        P = orc.polarization(c.M[q], G, c.kmq[q], omega=2.0)
        Wt = orc.nu_to_tau(orc.screen(orc.tau_to_nu(P, gr), c.v[q]), gr)
        sc, sx, _ = orc.selfenergy(c.M[q], G, Wt, c.v[q], c.kmq[q], occ, omega=2.0)
        Sc, Sx = Sc + sc, Sx + sx
    return Sc, Sx


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec", ["fp64", "fp16x2"])
def test_irreducible_chain_equals_full_chain(gw, prec):
    p = {"fp64": gw.GW_FP64, "fp16x2": gw.GW_FP16X2}[prec]
    c, gr = _crystal()
    star = {q: sy.star_kinv(c, q) for q in c.ibz}
    S_full, Sx_full, E_full = _chain(gw, c, gr, list(range(c.nq)), p)
    S_red, Sx_red, E_red = _chain(gw, c, gr, c.ibz, p, star)
    eS, eX = rel(S_red, S_full), rel(Sx_red, Sx_full)
    dE = np.abs(E_red - E_full).max()
    Sc_o, Sx_o = _oracle_full_sum()
    oS, oX = rel(S_red, Sc_o), rel(Sx_red, Sx_o)
    print(f"symmetry ({prec}): {len(c.ibz)} of {c.nq} q; vs full GPU chain Sigma^c {eS:.1e}, Sigma^x {eX:.1e}, "
          f"max |dE_qp| {dE:.1e} Ha; vs oracle full-mesh sum Sigma^c {oS:.1e}, Sigma^x {oX:.1e}")
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert eS < tol and eX < tol
    assert dE < (1e-9 if prec == "fp64" else 1e-5)
    # against the oracle: the FP64 bar, and the tensor-core bar of the mixed chain (Sigma^x is
    # float-float there)
    assert oS < (1e-10 if prec == "fp64" else 2e-5)
    assert oX < (1e-10 if prec == "fp64" else 1e-11)


def test_sigma_star_matches_oracle(gw):
    """gw_sigma_star against the oracle's star sum, every element, for each irreducible q's star
    (all star sizes of the 2 x 2 x 2 Oh mesh), with an entry outside the mesh skipped."""
    import torch
    c, gr = _crystal()
    cq = sy.restrict_q(c, c.ibz)
    ctx = gw.GW(gr, cq, omega=2.0, M=torch.from_numpy(cq.M).cuda())
    rng = np.random.default_rng(3)
    for q in c.ibz:
        kinv = sy.star_kinv(c, q)
        T = rng.standard_normal((c.nk, c.nb, gr.ntau))
        S0 = rng.standard_normal((c.nk, c.nb, gr.ntau))
        S = torch.from_numpy(S0.copy()).cuda()
        ctx.sigma_star(torch.from_numpy(kinv).cuda(), torch.from_numpy(T).cuda(), S)
        ctx.sync()
        ref = S0 + orc.symmetry.sigma_star(T, kinv)
        assert np.abs(S.cpu().numpy() - ref).max() <= 1e-15 * np.abs(ref).max(), q
    # entries of kinv outside [0, nk) are skipped
    kinv = sy.star_kinv(c, c.ibz[-1]).copy()
    keep = kinv.copy()
    kinv[0, 0] = -1
    T = rng.standard_normal((c.nk, 3))
    S = torch.zeros(c.nk, 3, dtype=torch.float64, device="cuda")
    ctx.sigma_star(torch.from_numpy(kinv).cuda(), torch.from_numpy(T).cuda(), S)
    ctx.sync()
    ref = orc.symmetry.sigma_star(T, keep)
    ref[0] -= T[keep[0, 0]]
    assert np.abs(S.cpu().numpy() - ref).max() <= 1e-15 * np.abs(ref).max()
    ctx.close()
