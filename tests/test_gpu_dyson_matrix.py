"""The full-matrix Dyson update (gw_dyson_matrix: Eq. dysonGF without the diagonal approximation,
posed in i w with the exact matrix tail) against the oracle (oracle.offdiag.dyson_matrix_iw,
pinned by the downfolding closed form of a pole self-energy), through the C ABI, FP64 at 1e-10;
its diagonal reduction against gw_green_tau; and the off-diagonal chain gw_selfenergy_offdiag ->
gw_dyson_matrix against the same chain in the oracle."""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc
from oracle import offdiag as od

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def _herm(rng, nk, nb, s):
    X = rng.standard_normal((nk, nb, nb)) + 1j * rng.standard_normal((nk, nb, nb))
    return s * (X + np.conj(np.swapaxes(X, 1, 2))) / 2


def _run(gw, ctx, cr, gr, eps, Sx, vxc, Sc):
    import torch
    G = torch.zeros((cr.nk, cr.nb, cr.nb, gr.ntau), dtype=torch.complex128, device="cuda")
    occ = torch.zeros((cr.nk, cr.nb, cr.nb), dtype=torch.complex128, device="cuda")
    info = torch.full((cr.nk,), -1, dtype=torch.int32, device="cuda")
    ctx.dyson_matrix(dev(eps), None if Sx is None else dev(Sx), None if vxc is None else dev(vxc),
                     None if Sc is None else dev(Sc), G, occ, info)
    ctx.sync()
    return G.cpu().numpy(), occ.cpu().numpy(), info.cpu().numpy()


@pytest.mark.parametrize("nb", [16, 7])
def test_dyson_matrix_vs_oracle(gw, nb):
    """A random Hermitian static part (so H~ is not diagonal) and a Hermitian Sigma^c(tau) built as a
    sum of matrix poles; nb = 7 exercises the odd size (one padded, decoupled Jacobi index)."""
    cr = gi.make_crystal(31, 4, nb, nb // 2, 32, 40.0, qlist=[1])
    gr = gi.make_grid(40.0, 24, 24, 24, ncont=32)
    ctx = gw.GW(gr, cr, omega=1.0)
    rng = np.random.default_rng(nb)
    Sx, vxc = _herm(rng, cr.nk, nb, 0.2), _herm(rng, cr.nk, nb, 0.05)
    # Sigma^c(tau) = sum_p C_p G0(E_p, tau) C_p^+ per k: Hermitian at every tau
    E = rng.uniform(-1.5, 1.5, 3)
    C = 0.2 * (rng.standard_normal((cr.nk, nb, 3)) + 1j * rng.standard_normal((cr.nk, nb, 3)))
    g0, _ = orc.green_tau0(E[None, :], gr.tau, gr.beta)
    Sc = np.einsum("knp,pt,kmp->knmt", C, g0[0], np.conj(C))
    G, occ, info = _run(gw, ctx, cr, gr, cr.eps, Sx, vxc, Sc)
    Gr, occr = od.dyson_matrix_iw(cr.eps, Sx, vxc, orc.sigma_tau_to_iw(Sc, gr), gr)
    assert np.all(info == 0)
    eG, eo = rel(G, Gr), rel(occ, occr)
    print(f"nb {nb}: G {eG:.2e}, occupation matrix {eo:.2e}")
    assert eG < TOL and eo < TOL
    assert np.abs(G - np.conj(np.swapaxes(G, 1, 2))).max() < 1e-12 * np.abs(G).max()   # Hermitian at every tau
    # no self-energy: G = U G0(lambda) U^+ exactly, the oracle's G0 of H~ by eigh
    G0, occ0, info = _run(gw, ctx, cr, gr, cr.eps, Sx, vxc, None)
    H = np.einsum("kn,nm->knm", cr.eps, np.eye(nb)) + Sx - vxc
    lam, U = np.linalg.eigh(H)
    g, f = orc.green_tau0(lam, gr.tau, gr.beta)
    assert rel(G0, np.einsum("kna,kat,kma->knmt", U, g, np.conj(U))) < 1e-13
    assert rel(occ0, np.einsum("kna,ka,kma->knm", U, f, np.conj(U))) < 1e-13
    ctx.close()


def test_dyson_matrix_diagonal_reduces_to_gw_green_tau(gw):
    """Diagonal inputs: the matrix update's diagonal is the diagonal update of gw_green_tau (and of the
    oracle's dyson_iw), off-diagonal elements zero."""
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    rng = np.random.default_rng(2)
    sx, vx = rng.uniform(-0.2, 0.2, (cr.nk, cr.nb)), rng.uniform(-0.1, 0.1, (cr.nk, cr.nb))
    E = rng.uniform(-1, 1, (cr.nk, cr.nb))
    r = rng.uniform(0.05, 0.2, (cr.nk, cr.nb)) ** 2
    g0, _ = orc.green_tau0(E, gr.tau, gr.beta)
    sc = r[..., None] * g0                                                  # one pole per state, in tau
    d = np.arange(cr.nb)
    M3 = lambda x: np.einsum("kn,nm->knm", x, np.eye(cr.nb)).astype(complex)  # noqa: E731
    Sm = np.zeros((cr.nk, cr.nb, cr.nb, gr.ntau), complex)
    Sm[:, d, d, :] = sc
    G, occ, info = _run(gw, ctx, cr, gr, cr.eps, M3(sx), M3(vx), Sm)
    Gd = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
    occd = torch.zeros((cr.nk, cr.nb), dtype=torch.float64, device="cuda")
    siw = orc.sigma_tau_to_iw(sc, gr)
    ctx.green_tau(dev(cr.eps), Gd, occd, dev(sx), dev(vx), dev(siw))
    ctx.sync()
    Gref, occref = orc.dyson_iw(cr.eps, sx, vx, siw, gr)
    assert np.all(info == 0)
    assert rel(G[:, d, d, :], Gd.cpu().numpy()) < 1e-12 and rel(G[:, d, d, :].real, Gref) < TOL
    assert np.abs(occ[:, d, d] - occref).max() < 1e-12
    G[:, d, d, :] = 0.0
    assert np.abs(G).max() < 1e-13
    ctx.close()


def test_offdiag_chain_vs_oracle(gw):
    """G0 -> P -> W~ (FP64 GPU chain) -> off-diagonal Sigma^c, Sigma^x (gw_selfenergy_offdiag) -> matrix
    Dyson (gw_dyson_matrix), against the same chain in the oracle."""
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    z = lambda *s, dt=torch.float64: torch.zeros(s, dtype=dt, device="cuda")  # noqa: E731
    c16 = torch.complex128
    G, occ = z(cr.nk, cr.nb, gr.ntau), z(cr.nk, cr.nb)
    ctx.green_tau(dev(cr.eps), G, occ)
    P, Piv, Wiv, Wt = (z(gr.ntau, cr.ni, cr.ni, dt=c16), z(gr.nnu, cr.ni, cr.ni, dt=c16),
                       z(gr.nnu, cr.ni, cr.ni, dt=c16), z(gr.ntau, cr.ni, cr.ni, dt=c16))
    info = z(1, gr.nnu, dt=torch.int32)
    ctx.polarization(0, G, P, gw.GW_FP64)
    ctx.tau_to_freq(gw.GW_BOSE, gw.GW_TAU_TO_IW, cr.ni * cr.ni, P, Piv)
    ctx.screen(0, 1, Piv, Wiv, info)
    ctx.tau_to_freq(gw.GW_BOSE, gw.GW_IW_TO_TAU, cr.ni, Wiv, Wt)
    Sc, Sx = z(cr.nk, cr.nb, cr.nb, gr.ntau, dt=c16), z(cr.nk, cr.nb, cr.nb, dt=c16)
    ctx.selfenergy_offdiag(0, G, occ, Wt, Sc, Sx)
    # oracle
    M = gi.m_for_q(cr, 0)
    G0, f0 = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    Wr = orc.nu_to_tau(orc.screen(orc.tau_to_nu(orc.polarization(M, G0, cr.kmq[0]), gr), cr.v[0]), gr)
    Scr, Sxr = od.selfenergy_offdiag(M, G0, Wr, cr.v[0], cr.kmq[0], f0)
    # the reference potential: the oracle's Sigma^x with its diagonal flattened, so H~ keeps the
    # off-diagonal exchange
    vxc = Sxr.copy()
    d = np.arange(cr.nb)
    vxc[:, d, d] = vxc[:, d, d].real.mean()
    G1 = z(cr.nk, cr.nb, cr.nb, gr.ntau, dt=c16)
    occ1 = z(cr.nk, cr.nb, cr.nb, dt=c16)
    inf = torch.full((cr.nk,), -1, dtype=torch.int32, device="cuda")
    ctx.dyson_matrix(dev(cr.eps), Sx, dev(vxc), Sc, G1, occ1, inf)
    ctx.sync()
    Gr, occr = od.dyson_matrix_iw(cr.eps, Sxr, vxc, orc.sigma_tau_to_iw(Scr, gr), gr)
    assert np.all(inf.cpu().numpy() == 0)
    eS, eX = rel(Sc.cpu().numpy(), Scr), rel(Sx.cpu().numpy(), Sxr)
    eG, eo = rel(G1.cpu().numpy(), Gr), rel(occ1.cpu().numpy(), occr)
    print(f"off-diagonal chain: Sigma^c {eS:.1e}, Sigma^x {eX:.1e}, G {eG:.1e}, occupation {eo:.1e}")
    assert eS < TOL and eX < TOL and eG < TOL and eo < TOL
    ctx.close()
