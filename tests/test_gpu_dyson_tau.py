"""The paper's tau-domain Dyson equation (Eqs. dysongf-dysong, Sec. III.B.5) on the GPU
(gw_dyson_tau) against the oracle's solve of the same discrete system per state, and against
the closed form of a one-pole self-energy."""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

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


def _run(gw, ctx, tu, eps, s, sig):
    import torch
    n = int(round(tu[-1] / (tu[1] - tu[0])))
    G = torch.zeros((len(eps), n + 1), dtype=torch.float64, device="cuda")
    info = torch.ones(len(eps), dtype=torch.int32, device="cuda")
    ctx.dyson_tau(tu, dev(eps), dev(s), dev(sig), G, info)
    ctx.sync()
    assert np.all(info.cpu().numpy() == 0)
    return G.cpu().numpy()


@pytest.mark.parametrize("p,m", [(3, 4), (4, 4)])
def test_dyson_tau_parity_crystal_states(gw, p, m):
    """All 128 states of the Nk=8 crystal (its band energies), random static shifts and a
    three-pole Sigma^c(tau) per state on UPM(p, m) at beta = 20."""
    cr, gr = gi.make_config("nk8_nb16")
    beta = 20.0
    tu = gi.upm_grid(beta, p, m)
    rng = np.random.default_rng(31)
    eps = cr.eps.reshape(-1).copy()
    nprob = len(eps)
    s = rng.uniform(-0.2, 0.2, nprob)
    sig = np.zeros((nprob, len(tu)))
    for _ in range(3):
        c2, E = rng.uniform(0.01, 0.1, nprob), rng.uniform(-1.5, 1.5, nprob)
        sig += c2[:, None] * np.stack([orc.dyson_tau.g0_tau(E[i], tu, beta) for i in range(nprob)])
    ctx = gw.GW(gr, cr, omega=1.0)
    G = _run(gw, ctx, tu, eps, s, sig)
    ref = np.stack([orc.dyson_tau.dyson_tau(eps[i], s[i], sig[i], tu)[0] for i in range(nprob)])
    e = np.abs(G - ref).max() / np.abs(ref).max()
    print(f"tau-domain Dyson UPM({p},{m}), {nprob} states x {G.shape[1]} points: GPU vs oracle {e:.2e}")
    assert e < TOL
    ctx.close()


def test_dyson_tau_closed_form_on_gpu(gw):
    """One-pole Sigma^c(i w) = c^2 / (i w - E) and a static shift: G has the two poles of
    (x - eps - s)(x - E) = c^2; the GPU solve converges to it at first order."""
    dt = orc.dyson_tau
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    beta, eps, s, c, E = 20.0, 0.4, -0.1, 0.3, -0.6
    r = np.roots([1.0, -(eps + s + E), (eps + s) * E - c * c])
    errs = []
    for m in (8, 16):
        tu = gi.upm_grid(beta, 3, m)
        G = _run(gw, ctx, tu, np.array([eps]), np.array([s]), (c * c * dt.g0_tau(E, tu, beta))[None])[0]
        t = dt.dense_mesh(tu)
        ex = sum(((ri - E) / (ri - rj)) * dt.g0_tau(ri, t, beta) for ri, rj in [(r[0], r[1]), (r[1], r[0])])
        errs.append(np.abs(G - ex).max() / np.abs(ex).max())
    print(f"tau-domain Dyson vs closed form, UPM(3, 8) / UPM(3, 16): {errs[0]:.2e} / {errs[1]:.2e}")
    assert 1.8 < errs[0] / errs[1] < 2.3 and errs[1] < 1e-2, errs
    ctx.close()


def test_dyson_tau_rejects_bad_mesh(gw):
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    sig = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    G = torch.zeros((1, 64), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gw.GwError):
        ctx.dyson_tau(np.array([0.0, 1.0, 2.5, 4.0]), z, z, sig, G, info)   # 2.5 not a multiple of 1
    with pytest.raises(gw.GwError):
        ctx.dyson_tau(np.array([0.5, 1.0, 2.0, 4.0]), z, z, sig, G, info)   # does not start at 0
    ctx.close()
