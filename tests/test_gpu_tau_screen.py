"""The paper's tau-domain screened interaction (Eq. tildeW on the uniform power mesh, Sec. III.B.3)
on the GPU (gw_screen_tau) against the oracle's solve of the same discrete system, and against
the closed form of a one-mode polarization."""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 elimination vs LAPACK on the same system


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def crystal_P_pair(cr, gr, iq, tau, omega):
    """P(tau_p - tau_r) of the synthetic crystal's iq-th q at every pair of the mesh: the oracle's
    Eq. (irpol) with G0 on the distinct differences (closed under beta - tau with beta added)."""
    d, idx = gi.tau_pairs(tau, gr.beta)
    order = np.argsort(d)
    dd = np.concatenate([d[order], [gr.beta]])
    G, _ = orc.green_tau0(cr.eps, dd, gr.beta)
    P = orc.polarization(gi.m_for_q(cr, iq), G, cr.kmq[iq], omega=omega)[:-1]
    Pd = np.empty_like(P)
    Pd[order] = P
    return Pd[idx]


@pytest.mark.parametrize("p,m", [(4, 2), (3, 3)])
def test_screen_tau_parity_crystal(gw, p, m):
    """NI = 64 (the Nk=8 crystal), UPM(p, m): (2pm + 1) 64 unknowns; P from the crystal's own
    polarization at every mesh difference, not symmetric under tau -> beta - tau."""
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    omega = gi.OMEGA_SI
    tau = gi.upm_grid(gr.beta, p, m)
    Pp = crystal_P_pair(cr, gr, 0, tau, omega)
    ref = orc.screen_tau.screen_tau(Pp, cr.v[0], tau)
    ctx = gw.GW(gr, cr, omega=omega)
    W = torch.zeros((len(tau), cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.screen_tau(0, tau, dev(Pp), W, info)
    ctx.sync()
    assert host(info)[0] == 0
    e = rel(host(W), ref)
    print(f"tau-domain W~ UPM({p},{m}), {len(tau) * cr.ni} unknowns: GPU vs oracle {e:.2e}")
    assert e < TOL
    ctx.close()


def test_screen_tau_closed_form_on_gpu(gw):
    """NI = 32, uniform v and P(tau) = U diag(p_s(tau)) U^+ with one bosonic mode per direction:
    the GPU solve equals the oracle's and converges to U diag(W_s(tau)) U^+ (the scalar closed
    forms) at second order in the step."""
    import torch
    st = orc.screen_tau
    rng = np.random.default_rng(23)
    beta, v, ni = 20.0, 1.5, 32
    a, E = rng.uniform(0.1, 0.6, ni), rng.uniform(0.3, 1.5, ni)
    U, _ = np.linalg.qr(rng.standard_normal((ni, ni)) + 1j * rng.standard_normal((ni, ni)))
    cr = gi.make_crystal(seed=7, nk=1, nb=2, nocc=1, ni=ni, beta=beta)
    cr.v[:] = v
    gr = gi.make_grid(beta, 16, 16, 16, ncont=16)
    ctx = gw.GW(gr, cr, omega=1.0)
    errs = []
    for m in (8, 16):
        tau = gi.upm_grid(beta, 3, m)
        d, idx = gi.tau_pairs(tau, beta)
        Pd = np.einsum("is,ns,js->nij", U, np.stack([st.single_pole_P(d, a[s], E[s], beta) for s in range(ni)], 1),
                       U.conj())
        Pp = np.ascontiguousarray(Pd[idx])
        W = torch.zeros((len(tau), ni, ni), dtype=torch.complex128, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        ctx.screen_tau(0, tau, dev(Pp), W, info)
        ctx.sync()
        assert host(info)[0] == 0
        Wg = host(W)
        assert rel(Wg, st.screen_tau(Pp, np.full(ni, v), tau)) < TOL
        Wex = np.einsum("is,ns,js->nij", U,
                        np.stack([st.single_pole_Wt(tau, a[s], E[s], v, beta) for s in range(ni)], 1), U.conj())
        errs.append(rel(Wg, Wex))
    print(f"tau-domain W~ vs closed form, UPM(3, 8) / UPM(3, 16): {errs[0]:.2e} / {errs[1]:.2e}")
    assert errs[0] / errs[1] > 3.5 and errs[1] < 1e-2, errs
    ctx.close()


def test_screen_tau_rejects_bad_mesh(gw):
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    W = torch.zeros((3, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = torch.zeros((3, 3, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GwError):
        ctx.screen_tau(0, np.array([0.0, 2.0, 1.0]), P, W, info)   # not increasing
    with pytest.raises(gw.GwError):
        ctx.screen_tau(5, np.array([0.0, 1.0, 2.0]), P, W, info)   # q index out of range
    ctx.close()
