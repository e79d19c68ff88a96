"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes a property that the paper or the mathematics determines, so
that a plausible slip in the oracle (dropped term, wrong sign or index,
transposed operand) fails at least one of them.
"""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc
from oracle import transforms as tr


def _kf(tau, e, beta):
    tau = np.asarray(tau, float)
    if e >= 0:
        return np.exp(-e * tau) / (1 + np.exp(-beta * e))
    return np.exp(e * (beta - tau)) / (1 + np.exp(beta * e))


@pytest.fixture(scope="module")
def g1():
    return gi.make_grid(100.0, 16, 16, 16)


# ----------------------------------------------------------------------- G0
def test_g0_boundaries_and_particle_number():
    cr = gi.make_crystal(11, 8, 16, 8, 4, 100.0)
    t = np.array([1e-14, 100.0 - 1e-14])
    G, occ = orc.green_tau0(cr.eps, t, cr.beta)
    # G(0+) + G(beta-) = -1 (anticommutator), G(beta-) = -f (Sec. III.B.3)
    assert np.allclose(G[..., 0] + G[..., 1], -1.0, atol=1e-12)
    assert np.allclose(G[..., 1], -occ, atol=1e-12)
    # valence: G(0+) -> 0, G(beta-) -> -1; conduction the reverse (to e^{-beta 0.05})
    assert abs(occ.sum() - 8 * 8) < 8 * 16 * np.exp(-100 * 0.05)
    # overflow-free form equals the textbook form where the latter is finite
    e = np.array([-0.3, 0.2])
    tt = np.linspace(0.1, 99.9, 7)
    Gt, _ = orc.green_tau0(e, tt, 100.0)
    one_minus_nf = 1 / (1 + np.exp(-100.0 * e))       # 1 - n_F without cancellation
    ref = -np.exp(-e[:, None] * tt[None, :]) * one_minus_nf[:, None]
    assert np.allclose(Gt, ref, rtol=1e-13)
    assert np.all(G <= 0)


# ----------------------------------------------------------------------- P
def _fine_sym_grid(beta, npan=40, order=16, t0=1e-5):
    """Composite Gauss-Legendre on geometric panels of [0, beta/2], mirrored."""
    edges = np.concatenate([[0.0], np.geomspace(t0, beta / 2, npan)])
    x, w = np.polynomial.legendre.leggauss(order)
    ts, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        ts.append(0.5 * (b - a) * x + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * w)
    t = np.concatenate(ts)
    w = np.concatenate(ws)
    return np.concatenate([t, beta - t[::-1]]), np.concatenate([w, w[::-1]])


def _tiny_system(seed=5, nk=2, nb=4, nocc=2, ni=3, beta=20.0):
    cr = gi.make_crystal(seed, nk, nb, nocc, ni, beta)
    M = gi.m_for_q(cr, 1)
    return cr, M


def test_polarization_matches_lindhard():
    """int_0^beta e^{i nu tau} P(tau) dtau of Eq. (irpol) with G0 equals the Lindhard sum."""
    cr, M = _tiny_system()
    t, w = _fine_sym_grid(cr.beta)
    G, _ = orc.green_tau0(cr.eps, t, cr.beta)
    P = orc.polarization(M, G, cr.kmq[1], omega=1.7)
    nidx = np.arange(0, 6)
    nu = 2 * np.pi * nidx / cr.beta
    Piv = np.einsum("j,jab->ab", w, P)[None] if False else np.einsum("i,ni,iab->nab", w,
                                                                       np.exp(1j * np.outer(nu, t)), P)
    ref = orc.lindhard_iv(M, cr.eps, cr.kmq[1], nidx, cr.beta, omega=1.7)
    assert np.abs(Piv - ref).max() < 1e-10 * np.abs(ref).max()


def test_polarization_hermitian_negative():
    cr, M = _tiny_system(nk=8, nb=6, nocc=3, ni=5, beta=50.0)
    g = gi.make_grid(50.0, 16, 8, 8)
    G, _ = orc.green_tau0(cr.eps, g.tau, cr.beta)
    P = orc.polarization(M, G, cr.kmq[1])
    assert np.abs(P - np.conj(np.swapaxes(P, 1, 2))).max() < 1e-15 * np.abs(P).max()
    for i in range(g.ntau):
        assert np.linalg.eigvalsh(P[i]).max() < 1e-14 * np.abs(P).max()
    # P(tau) depends only on Q_ab(tau): P(beta - tau) differs (no time reversal for generic M)
    # but the static Lindhard value is Hermitian and negative definite
    L0 = orc.lindhard_iv(M, cr.eps, cr.kmq[1], [0], cr.beta)[0]
    assert np.abs(L0 - L0.conj().T).max() < 1e-14 * np.abs(L0).max()
    assert np.linalg.eigvalsh(L0).max() < 0


# ----------------------------------------------------------------------- transforms
def test_transforms_exact_on_basis(g1):
    T = orc.transform_matrices(g1)
    b = g1.beta
    w = (2 * g1.w_idx + 1) * np.pi / b
    nu = 2 * g1.nu_idx * np.pi / b
    wc = (2 * np.arange(g1.ncont) + 1) * np.pi / b
    for e in g1.poles[[0, 3, len(g1.poles) // 2, -2]]:
        f = _kf(g1.tau, e, b)
        assert np.abs(T["F_fwd"] @ f - (-1 / (1j * w - e))).max() < 1e-12
        assert np.abs(T["F_cont"] @ f - (-1 / (1j * wc - e))).max() < 1e-12
        with np.errstate(invalid="ignore", divide="ignore"):
            kb = -np.tanh(b * e / 2) / (1j * nu - e)
        kb = np.where((nu == 0) & (e == 0), b / 2, kb)
        assert np.abs(T["B_fwd"] @ f - kb).max() < 1e-12
        assert np.abs(T["B_bwd_re"] @ kb.real + T["B_bwd_im"] @ kb.imag - f).max() < 1e-12
        fi = -1 / (1j * w - e)
        assert np.abs(T["F_bwd_re"] @ fi.real + T["F_bwd_im"] @ fi.imag - f).max() < 1e-12
        assert abs(T["F_bwd_beta_re"] @ fi.real + T["F_bwd_beta_im"] @ fi.imag - _kf(b, e, b)) < 1e-12
        assert abs(T["tau_to_beta"] @ f - _kf(b, e, b)) < 1e-12


def test_g0_transform_with_eps_on_pole(g1):
    """G0 with eps equal to a grid pole transforms to 1/(i w - eps) (Eq. trans)."""
    e = g1.poles[g1.poles > 0][2]
    G, _ = orc.green_tau0(np.array([[e]]), g1.tau, g1.beta)
    S = orc.sigma_tau_to_iw(G, g1)
    ref = orc.green_iw0(np.array([[e]]), g1.w_idx, g1.beta)
    assert np.abs(S - ref).max() < 1e-12


def test_transform_accuracy_off_grid():
    """Discretisation error (not a parity bar): G0 at energies off the pole grid."""
    g = gi.make_grid(200.0, 48, 48, 48)
    for e in [0.37, -0.05, 1.0, 30.0]:
        G, _ = orc.green_tau0(np.array([[e]]), g.tau, g.beta)
        S = orc.sigma_tau_to_iw(G, g, cont=True)
        ref = 1 / (1j * (2 * np.arange(g.ncont) + 1) * np.pi / g.beta - e)
        assert np.abs(S - ref).max() < 2e-3


# ----------------------------------------------------------------------- screen
def test_screen_scalar_closed_form():
    """NI = 1: W~ = v^2 P / (1 - v P) (iν form of Eq. tildeW)."""
    P = np.array([-0.3 + 0.1j, -2.0, -0.01j]).reshape(3, 1, 1)
    v = np.array([7.0])
    W = orc.screen(P, v)
    ref = 49.0 * P[:, 0, 0] / (1 - 7.0 * P[:, 0, 0])
    assert np.allclose(W[:, 0, 0], ref, rtol=1e-14)


def test_screen_residual_and_static_sign():
    cr, M = _tiny_system(nk=8, nb=6, nocc=3, ni=5, beta=50.0)
    L = orc.lindhard_iv(M, cr.eps, cr.kmq[1], [0, 1, 7], cr.beta)
    v = cr.v[1]
    W = orc.screen(L, v)
    sv = np.sqrt(v)
    for j in range(3):
        Pi = sv[:, None] * L[j] * sv[None, :]
        X = W[j] / sv[:, None] / sv[None, :]
        assert np.abs((np.eye(5) - Pi) @ X - Pi).max() < 1e-12 * (1 + np.abs(Pi).max())
    # static screening: W~(0) = W - v is Hermitian negative semidefinite
    assert np.abs(W[0] - W[0].conj().T).max() < 1e-12 * np.abs(W[0]).max()
    assert np.linalg.eigvalsh(W[0]).max() < 1e-12


# ----------------------------------------------------------------------- whole chain, one mode
def _one_pair_model(g, omega=1.3):
    """Nk = 1, Nb = 2, NI = 1, one active pair a = 0 (occ) -> b = 1 (unocc) whose
    transition energy D and screened pole E = D + v w both sit on the pole grid,
    so every transform is exact and the chain has a closed form."""
    pos = g.poles[g.poles > 0.1]
    D, E = pos[1], pos[3]
    beta = g.beta
    eps = np.array([[-D / 2, D / 2]])
    fa, fb = 1 / (np.exp(beta * eps[0, 0]) + 1), 1 / (np.exp(beta * eps[0, 1]) + 1)
    v = np.array([2.5])
    w = (E - D) / v[0]                       # weight of P(i nu) = w / (i nu - D)
    m2 = w * omega / (fa - fb)               # |M|^2 with 1/(Omega Nk) folded in
    M = np.zeros((1, 1, 2, 2), complex)
    M[0, 0, 0, 1] = np.sqrt(m2) * np.exp(0.4j)
    return dict(D=D, E=E, eps=eps, fa=fa, fb=fb, v=v, w=w, m2=m2, M=M, omega=omega, beta=beta)


def test_chain_closed_form_single_mode(g1):
    m = _one_pair_model(g1)
    beta, kmq = m["beta"], np.array([0])
    G, occ = orc.green_tau0(m["eps"], g1.tau, beta)
    P = orc.polarization(m["M"], G, kmq, m["omega"])
    # Eq. (irpol): P(tau) = -(1 - f_b) f_a |M|^2 e^{-D tau} / Omega
    Pref = -(1 - m["fb"]) * m["fa"] * m["m2"] / m["omega"] * np.exp(-m["D"] * g1.tau)
    assert np.abs(P[:, 0, 0] - Pref).max() < 1e-15 + 1e-13 * np.abs(Pref).max()
    Piv = orc.tau_to_nu(P, g1)
    nu = 2 * np.pi * g1.nu_idx / beta
    assert np.abs(Piv[:, 0, 0] - m["w"] / (1j * nu - m["D"])).max() < 1e-12
    W = orc.screen(Piv, m["v"])
    c = m["v"][0] * m["w"]
    assert np.abs(W[:, 0, 0] - m["v"][0] * c / (1j * nu - m["E"])).max() < 1e-11
    Wt = orc.nu_to_tau(W, g1)
    E = m["E"]
    Wref = -m["v"][0] * c * np.exp(-E * g1.tau) / (1 - np.exp(-beta * E))
    assert np.abs(Wt[:, 0, 0] - Wref).max() < 1e-11 * np.abs(Wref).max()
    sc, sx, im = orc.selfenergy(m["M"], G, Wt, m["v"], kmq, occ, m["omega"])
    # Eq. (sigc): only band n = 1 (b) couples, through j = 0 (a)
    s_ref = -(G[0, 0, :] * m["m2"] * Wref) / m["omega"]
    # error bound of a product G W~: W~(tau) carries ~1e-12 of max|W~| from the backward map
    scale = m["m2"] * np.abs(Wref).max() / m["omega"]
    assert np.abs(sc[0, 1] - s_ref).max() < 1e-11 * scale
    assert np.abs(sc[0, 0]).max() == 0.0
    # Eq. (sigx): -f_a v |M|^2 / Omega on band b, zero on band a
    assert abs(sx[0, 1] - (-occ[0, 0] * m["v"][0] * m["m2"] / m["omega"])) < 1e-14
    assert sx[0, 0] == 0.0


def test_sigma_iw_closed_form_single_mode(g1):
    """Sigma^c(i w) of the one-mode chain against int_0^beta e^{i w tau} of its closed form."""
    m = _one_pair_model(g1)
    beta = m["beta"]
    # choose a model whose Sigma(tau) exponent eps_a + E also sits on the pole grid
    a = m["eps"][0, 0] + m["E"]
    G, occ = orc.green_tau0(m["eps"], g1.tau, beta)
    E = m["E"]
    c = m["v"][0] * m["w"]
    Wref = -m["v"][0] * c * np.exp(-E * g1.tau) / (1 - np.exp(-beta * E))
    s = -(G[0, 0, :] * m["m2"] * Wref) / m["omega"]        # = C e^{-a tau}
    C = s[0] / np.exp(-a * g1.tau[0])
    assert np.allclose(s, C * np.exp(-a * g1.tau), rtol=1e-12)
    S = orc.sigma_tau_to_iw(s[None, None, :], g1, cont=True)[0, 0]
    wc = (2 * np.arange(g1.ncont) + 1) * np.pi / beta
    ref = C * (-(1 + np.exp(-a * beta))) / (1j * wc - a)
    # a is off the pole grid: discretisation-level agreement only
    assert np.abs(S - ref).max() < 1e-2 * np.abs(ref).max()


def test_sigx_direct_occupied_sum():
    """Product-basis Eq. (sigx) against an explicit loop over occupied states."""
    cr, M = _tiny_system(nk=4, nb=5, nocc=2, ni=3, beta=30.0)
    g = gi.make_grid(30.0, 16, 8, 8)
    G, occ = orc.green_tau0(cr.eps, g.tau, cr.beta)
    W0 = np.zeros((g.ntau, 3, 3), complex)
    _, sx, _ = orc.selfenergy(M, G, W0, cr.v[1], cr.kmq[1], occ, omega=2.0)
    ref = np.zeros((4, 5))
    for k in range(4):
        for n in range(5):
            s = 0.0
            for j in range(5):
                f = 1.0 / (np.exp(cr.beta * cr.eps[cr.kmq[1][k], j]) + 1.0)
                for I in range(3):
                    s += f * cr.v[1][I] * abs(M[k, I, j, n]) ** 2
            ref[k, n] = -s / (2.0 * 4)
    assert np.allclose(sx, ref, rtol=1e-13, atol=1e-16)


def test_sigma_brute_force_matsubara():
    """Sigma^c(i w) of the chain against the direct Matsubara convolution
    -1/beta sum_nu G(i w - i nu) W~(i nu) with exact Lindhard P (tiny system,
    discretisation-level tolerance)."""
    beta = 10.0
    cr, M = _tiny_system(seed=9, nk=1, nb=3, nocc=1, ni=2, beta=beta)
    kmq = np.array([0])
    M = gi.m_for_q(cr, 0)
    v = cr.v[0] * 0.05
    g = gi.make_grid(beta, 48, 48, 48, ncont=4, lam=300.0)
    G, occ = orc.green_tau0(cr.eps, g.tau, beta)
    P = orc.polarization(M, G, kmq)
    W = orc.screen(orc.tau_to_nu(P, g), v)
    Wt = orc.nu_to_tau(W, g)
    sc, _, _ = orc.selfenergy(M, G, Wt, v, kmq, occ)
    S = orc.sigma_tau_to_iw(sc, g, cont=True)[0]              # [nb, ncont]
    # brute force
    N = 20000
    n = np.arange(-N, N + 1)
    nu = 2 * np.pi * n / beta
    Lnu = orc.lindhard_iv(M, cr.eps, kmq, np.abs(n), beta)
    Lnu = np.where((n < 0)[:, None, None], np.conj(np.swapaxes(Lnu, 1, 2)), Lnu)
    Wnu = orc.screen(Lnu, v)
    A = M[0].reshape(2, 9)
    d = np.einsum("Ip,nIJ,Jp->np", A.conj(), Wnu, A).reshape(len(n), 3, 3)  # [nu, a, n]
    eps = cr.eps[0]
    for m_ in range(4):
        wm = (2 * m_ + 1) * np.pi / beta
        Gm = 1.0 / (1j * (wm - nu)[:, None] - eps[None, :])                  # [nu, a]
        ref = -(Gm[:, :, None] * d).sum((0, 1)) / beta
        assert np.abs(S[:, m_] - ref).max() < 5e-3 * np.abs(ref).max()


def test_sigma_brute_force_matsubara_k_minus_q():
    """Eq. (sigc) at Nk = 3 with q != 0, so that k - q != k and the bands at k - q differ from
    those at k: Sigma^c_n(k|i w) of the chain against the direct Matsubara convolution
    -1/(Omega N_k beta) sum_nu sum_j G_j(k - q|i w - i nu) a_jn^+ W~(i nu) a_jn, with G and the
    Lindhard P written out here with the k - q index (k - q) mod Nk of the 3 x 1 x 1 mesh."""
    beta, nk, nb, ni, iq, omega = 10.0, 3, 3, 2, 1, 1.7
    cr = gi.make_crystal(13, nk, nb, 1, ni, beta, qlist=[iq])
    # the generator pins the band edges; draw band energies that differ at every k instead
    cr.eps = np.sort(np.random.default_rng(4).uniform(-1.0, 1.0, (nk, nb)), axis=1)
    M = gi.m_for_q(cr, 0)                                         # [k, I, a, b], a at k - q
    kmq = [(k - iq) % nk for k in range(nk)]
    assert list(cr.kmq[0]) == kmq and all(kmq[k] != k for k in range(nk))
    v = cr.v[0] * 0.05
    g = gi.make_grid(beta, 48, 48, 48, ncont=4, lam=300.0)
    G, occ = orc.green_tau0(cr.eps, g.tau, beta)
    P = orc.polarization(M, G, cr.kmq[0], omega=omega)
    W = orc.screen(orc.tau_to_nu(P, g), v)
    Wt = orc.nu_to_tau(W, g)
    sc, _, _ = orc.selfenergy(M, G, Wt, v, cr.kmq[0], occ, omega=omega)
    S = orc.sigma_tau_to_iw(sc, g, cont=True)                    # [k, n, ncont]
    # brute force over nu_n, |n| <= N
    N = 20000
    n = np.arange(-N, N + 1)
    nu = 2 * np.pi * n / beta
    f = 1.0 / (np.exp(beta * cr.eps) + 1.0)
    L = np.zeros((len(n), ni, ni), complex)
    for k in range(nk):
        ka = kmq[k]
        A = M[k].reshape(ni, nb * nb)
        wgt = (f[ka][:, None] - f[k][None, :]).reshape(-1)                         # f_a(k-q) - f_b(k)
        d = (cr.eps[k][None, :] - cr.eps[ka][:, None]).reshape(-1)
        L += np.einsum("Ip,np,Jp->nIJ", A, wgt[None, :] / (1j * nu[:, None] - d[None, :]), A.conj())
    L /= omega * nk
    sv = np.sqrt(v)
    Pi = sv[None, :, None] * L * sv[None, None, :]
    Wnu = sv[None, :, None] * (np.linalg.inv(np.eye(ni)[None] - Pi) - np.eye(ni)[None]) * sv[None, None, :]
    worst, slip = 0.0, 0.0
    for k in range(nk):
        A = M[k].reshape(ni, nb * nb)
        dd = np.einsum("Ip,nIJ,Jp->np", A.conj(), Wnu, A).reshape(len(n), nb, nb)  # [nu, j, n]
        for m_ in range(4):
            wm = (2 * m_ + 1) * np.pi / beta
            Gm = 1.0 / (1j * (wm - nu)[:, None] - cr.eps[kmq[k]][None, :])          # G_j(k-q|i w - i nu)
            ref = -(Gm[:, :, None] * dd).sum((0, 1)) / (beta * omega * nk)
            worst = max(worst, np.abs(S[k, :, m_] - ref).max() / np.abs(ref).max())
            Gk = 1.0 / (1j * (wm - nu)[:, None] - cr.eps[k][None, :])               # the slip G_j(k)
            bad = -(Gk[:, :, None] * dd).sum((0, 1)) / (beta * omega * nk)
            slip = max(slip, np.abs(bad - ref).max() / np.abs(ref).max())
    assert worst < 1e-4, worst             # measured 1.3e-5 (transform discretisation)
    assert slip > 1e3 * 1e-4, slip         # the pin tells G at k - q from G at k (measured 2.1)


# ----------------------------------------------------------------------- Dyson
def test_dyson_zero_and_static(g1):
    cr = gi.make_crystal(3, 2, 4, 2, 2, g1.beta)
    G0, occ0 = orc.green_tau0(cr.eps, g1.tau, g1.beta)
    z = np.zeros((2, 4, g1.nw), complex)
    sx = np.full((2, 4), -3.0)
    G, occ = orc.dyson_iw(cr.eps, sx, sx, z, g1)
    assert np.abs(G - G0).max() < 1e-14 and np.abs(occ - occ0).max() < 1e-14
    s = 0.013
    G, occ = orc.dyson_iw(cr.eps, sx + s, sx, z, g1)
    Gs, occs = orc.green_tau0(cr.eps + s, g1.tau, g1.beta)
    assert np.abs(G - Gs).max() < 1e-14 and np.abs(occ - occs).max() < 1e-14


def test_dyson_single_pole_sigma():
    """Sigma^c(i w) = g^2/(i w - E0): G has two poles (roots of a quadratic)."""
    g = gi.make_grid(100.0, 48, 48, 48)
    e0, g2, E0 = 0.3, 0.04, 1.1
    w = (2 * g.w_idx + 1) * np.pi / g.beta
    sig = (g2 / (1j * w - E0))[None, None, :]
    G, occ = orc.dyson_iw(np.array([[e0]]), np.zeros((1, 1)), np.zeros((1, 1)), sig, g)
    # poles x1, x2 of 1/(z - e0 - g2/(z - E0)); residues r_i = (x_i - E0)/(x_i - x_j)
    tr_, det = e0 + E0, e0 * E0 - g2
    x1, x2 = (tr_ - np.sqrt(tr_ ** 2 - 4 * det)) / 2, (tr_ + np.sqrt(tr_ ** 2 - 4 * det)) / 2
    r1, r2 = (x1 - E0) / (x1 - x2), (x2 - E0) / (x2 - x1)
    ref = np.zeros_like(g.tau)
    for x, r in [(x1, r1), (x2, r2)]:
        gt, _ = orc.green_tau0(np.array([x]), g.tau, g.beta)
        ref += r * gt[0]
    assert np.abs(G[0, 0] - ref).max() < 2e-3
    # anticommutator sum rule G(0+) + G(beta-) = -1 survives the update
    T = orc.transform_matrices(g)
    gz = T["tau_to_zero"] @ G[0, 0]
    assert abs(gz - occ[0, 0] + 1.0) < 1e-2


# ----------------------------------------------------------------------- continuation
def test_pade_recovers_pole_model():
    beta = 100.0
    e = np.array([-0.7, 0.2, 1.5])
    r = np.array([0.3, 0.5, 0.2])
    model = lambda z: (r[None, :] / (np.asarray(z)[:, None] - e[None, :])).sum(1)  # noqa: E731
    zs = 1j * (2 * np.arange(16) + 1) * np.pi / beta
    a = orc.pade_coeffs(zs, model(zs))
    x = np.linspace(-2, 2, 9) + 0.05j
    assert np.abs(orc.pade_eval(a, zs, x) - model(x)).max() < 1e-8


def test_cpe_kernel_asymptote_and_exact_recovery():
    from scipy.integrate import quad
    x = orc.cpe_grid(32, 0.05, 20.0)
    z = np.array([0.3 + 0.5j, 2j, -5 + 0.1j, 40j])
    K = orc.cpe_kernel(x, z)
    for m_ in [0, 7, 16, 31]:
        x0, x1, x2 = x[m_], x[m_ + 1], x[m_ + 2]
        hat = lambda s: (s - x0) / (x1 - x0) if s <= x1 else (x2 - s) / (x2 - x1)  # noqa: E731
        for iz, zz in enumerate(z):
            re = quad(lambda s: (hat(s) / (zz - s)).real, x0, x2, points=[x1], epsabs=1e-13, limit=200)[0]
            im = quad(lambda s: (hat(s) / (zz - s)).imag, x0, x2, points=[x1], epsabs=1e-13, limit=200)[0]
            assert abs(K[iz, m_] - (re + 1j * im)) < 1e-9 * (1 + abs(K[iz, m_]))
    rng = np.random.default_rng(0)
    b = np.zeros(32)
    b[[5, 6, 20]] = rng.uniform(0.1, 1.0, 3)
    w = (2 * np.arange(128) + 1) * np.pi / 100.0
    data = orc.cpe_kernel(x, 1j * w) @ b
    bf, res = orc.cpe_fit(w, data, x)
    assert res < 1e-10 * np.linalg.norm(data)
    assert np.all(bf >= 0)
    fit = orc.cpe_kernel(x, 1j * w) @ bf
    assert np.abs(fit - data).max() < 1e-10 * np.abs(data).max()
    # causality: Im Sigma(w + i0) = -pi rho(w) <= 0
    xs = np.linspace(-15, 15, 301) + 1e-9j
    assert (orc.cpe_kernel(x, xs) @ bf).imag.max() < 1e-7


def test_qp_quadratic_closed_form():
    eps, sx, vxc, g2, E0 = 0.2, -1.0, -1.1, 0.03, 0.9013  # pole off the 0.005 Ha scan grid
    resig = lambda E: g2 / (E - E0)  # noqa: E731
    E, Z, ok = orc.qp_solve(eps, sx, vxc, resig)
    # E - eps - sx + vxc = g2/(E - E0)  ->  quadratic, root nearest eps
    a0 = eps + sx - vxc
    roots = np.roots([1.0, -(a0 + E0), a0 * E0 - g2])
    want = roots[np.argmin(np.abs(roots - eps))]
    assert ok and abs(E - want) < 1e-12
    assert abs(Z - 1 / (1 + g2 / (want - E0) ** 2)) < 1e-6
    assert orc.band_gap(np.array([[-1, 0.5], [-0.8, 0.3]]), 1) == pytest.approx(1.1)


def _two_pole_roots(a0, e, r):
    """Real zeros of F(E) = E - a0 - sum_p r_p / (E - e_p) for two poles: the cubic
    (E - a0)(E - e1)(E - e2) - r1 (E - e2) - r2 (E - e1) = 0 (all three real and rising for r > 0)."""
    (e1, e2), (r1, r2) = e, r
    c = np.polymul(np.polymul([1.0, -a0], [1.0, -e1]), [1.0, -e2])
    c = np.polysub(c, np.polyadd(np.polymul([r1], [1.0, -e2]), np.polymul([r2], [1.0, -e1])))
    z = np.roots(c)
    assert np.abs(z.imag).max() < 1e-12
    return np.sort(z.real)


@pytest.mark.parametrize("case", ["separated", "close"])
def test_qp_two_pole_closed_form(case):
    """Several quasiparticle solutions (Sec. III.B.6 assumes one): with a two-pole Sigma^c every zero
    of F rises (Z = 1 / (1 + sum_p r_p / (E - e_p)^2) > 0), and qp_solve must return the one nearest
    eps, located independently of any energy mesh by the cubic's roots. The close case puts two zeros
    and a pole within 5 mHa of eps."""
    if case == "separated":
        e, r, s = (-0.3, 0.4), (0.02, 0.03), 0.05
        epss = np.linspace(-0.8, 0.8, 17)
    else:
        e, r, s = (-0.7, 0.2015), (0.01, 4e-6), -0.011
        epss = [0.2017, 0.203, 0.20325]
    for eps in epss:
        sx, vxc = -1.0, -1.0 - s
        def resig(E):
            with np.errstate(divide="ignore"):      # a mesh point may sit on a pole: F = -inf there
                return r[0] / (E - e[0]) + r[1] / (E - e[1])
        zs = _two_pole_roots(eps + s, e, r)
        want = zs[np.argmin(np.abs(zs - eps))]
        E, Z, ok = orc.qp_solve(eps, sx, vxc, resig)
        assert ok and abs(E - want) < 1e-12, (eps, E, zs)
        assert abs(Z - 1.0 / (1.0 + r[0] / (want - e[0]) ** 2 + r[1] / (want - e[1]) ** 2)) < 1e-6
        inwin = zs[np.abs(zs - eps) < orc.continuation.QP_WINDOW]
        got = orc.continuation.qp_roots(eps, sx, vxc, resig)
        assert len(got) == len(inwin) and np.abs(np.array(got) - inwin).max() < 1e-12
    if case == "close":
        assert np.sort(np.abs(zs - eps))[1] < 5e-3       # two zeros within 5 mHa of eps


def test_qp_no_zero_in_window_falls_back():
    """A static shift of 5 Ha puts the only zero outside eps +- 1 Ha: Newton from eps reaches it
    (E = eps + 5) and the result is flagged."""
    E, Z, ok = orc.qp_solve(0.3, -2.0, -2.0, lambda E: 5.0 + 0.0 * np.asarray(E))
    assert not ok and abs(E - 5.3) < 1e-12 and abs(Z - 1.0) < 1e-6


# ----------------------------------------------------------------------- learned CPE seed
def test_mlp_gradient_finite_differences():
    """Backward pass of the oracle MLP against central finite differences of its loss."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    sizes = [6, 8, 8, 5]
    params = mlp.init_params(sizes, rng)
    x = rng.standard_normal((7, 6))
    A = rng.standard_normal((6, 5)) * 0.3
    loss, grads = mlp.loss_and_grad(params, x, A)
    h = 1e-6
    for l in range(len(params)):
        W, b = params[l]
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = W.copy(); Wp[i, j] += h
            Wm = W.copy(); Wm[i, j] -= h
            lp, _ = mlp.loss_and_grad(params[:l] + [(Wp, b)] + params[l + 1:], x, A)
            lm, _ = mlp.loss_and_grad(params[:l] + [(Wm, b)] + params[l + 1:], x, A)
            assert abs((lp - lm) / (2 * h) - grads[l][0][i, j]) < 1e-7 * (1 + abs(grads[l][0][i, j]))
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        lp, _ = mlp.loss_and_grad(params[:l] + [(W, bp)] + params[l + 1:], x, A)
        lm, _ = mlp.loss_and_grad(params[:l] + [(W, bm)] + params[l + 1:], x, A)
        assert abs((lp - lm) / (2 * h) - grads[l][1][1]) < 1e-7 * (1 + abs(grads[l][1][1]))
    # activations: gelu(0) = 0, gelu'(0) = 1/2, softplus >= 0, softplus' = sigmoid
    assert mlp.gelu(np.array([0.0]))[0] == 0.0 and abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    z = np.linspace(-30, 30, 13)
    assert np.all(mlp.softplus(z) >= 0)
    assert np.allclose((mlp.softplus(z + 1e-6) - mlp.softplus(z - 1e-6)) / 2e-6, mlp.sigmoid(z), atol=1e-8)


# ------------------------------------------------------------------ tau-domain screening (Eq. tildeW, Sec. III.B.3)
def test_upm_grid_and_increments():
    beta = 50.0
    for p, m in [(3, 2), (5, 4), (8, 3)]:
        t = gi.upm_grid(beta, p, m)
        assert len(t) == 2 * p * m + 1
        assert t[0] == 0.0 and t[-1] == beta and np.all(np.diff(t) > 0)
        assert np.allclose(t + t[::-1], beta, rtol=0, atol=1e-12 * beta)
        assert np.isclose(np.diff(t).min(), beta / 2 ** p / m)      # densest at the ends
        dt = orc.screen_tau.trapezoid_weights(t)
        # the increments of the paper are the trapezoid rule: exact on linear functions
        assert np.isclose(dt.sum(), beta, rtol=1e-14)
        assert np.isclose(dt @ (3.0 * t - 1.0), 1.5 * beta ** 2 - beta, rtol=1e-13)
        d, idx = gi.tau_pairs(t, beta)
        assert np.allclose(d[idx], np.mod(t[:, None] - t[None, :], beta) % beta, atol=1e-9)
        assert idx[0, 0] == idx[-1, 0] == idx[0, -1] and d[idx[0, 0]] == 0.0   # 0 and +-beta are P(0)


def _scalar_case(model, p, m, beta=20.0, a=0.3, E=0.8, v=2.0):
    st = orc.screen_tau
    t = gi.upm_grid(beta, p, m)
    d, idx = gi.tau_pairs(t, beta)
    if model == "pole":
        Pd, ex = st.single_pole_P(d, a, E, beta), st.single_pole_Wt(t, a, E, v, beta)
    else:  # exponential: not symmetric under tau -> beta - tau, so the pair order matters
        Pd = -a * np.exp(-E * d) / (1.0 - np.exp(-beta * E))
        Ep = E + a * v
        ex = -a * v * v * np.exp(-Ep * t) / (1.0 - np.exp(-beta * Ep))
    W = st.screen_tau(Pd[idx][:, :, None, None], np.array([v]), t)[:, 0, 0]
    # the exponential model jumps at tau = 0 mod beta; W~(beta) is W~(0^-), compare below it
    sl = slice(None) if model == "pole" else slice(0, -1)
    return np.abs(W[sl] - ex[sl]).max() / np.abs(ex).max()


def test_screen_tau_single_pole_closed_form():
    """One bosonic mode P(i nu) = -2 a E / (nu^2 + E^2): W~(tau) = -a v^2 E cosh(Om (tau - beta/2)) /
    (Om sinh(Om beta/2)), Om^2 = E^2 + 2 a v E. The trapezoid solve converges at second order."""
    e = [_scalar_case("pole", 3, m) for m in (4, 8, 16, 32)]
    assert all(e[i] / e[i + 1] > 3.5 for i in range(3)), e
    assert e[-1] < 1e-3


def test_screen_tau_exponential_closed_form():
    """P(tau) = -a e^{-E tau} / (1 - e^{-beta E}) (P(i nu) = -a / (E - i nu)): W~(tau) = -a v^2 e^{-E' tau} /
    (1 - e^{-beta E'}), E' = E + a v. P jumps at tau = 0 mod beta, so first order; the wrong pair order
    (P(tau_r - tau_p)) converges to W~(beta - tau) instead."""
    e = [_scalar_case("exp", 3, m) for m in (8, 16, 32)]
    assert all(e[i] / e[i + 1] > 1.7 for i in range(2)), e
    assert e[-1] < 0.06


def test_screen_tau_matrix_in_common_eigenbasis():
    """NI = 3, uniform v and P(tau) = U diag(p_s(tau)) U^dagger with one mode per direction: W~(tau) =
    U diag(W_s(tau)) U^dagger from the scalar closed forms; also Hermitian at every tau."""
    st = orc.screen_tau
    rng = np.random.default_rng(17)
    beta, v, ni = 20.0, 1.5, 3
    a = np.array([0.2, 0.5, 0.9])
    E = np.array([0.4, 1.1, 2.0])
    U, _ = np.linalg.qr(rng.standard_normal((ni, ni)) + 1j * rng.standard_normal((ni, ni)))
    errs = []
    for m in (16, 32):
        t = gi.upm_grid(beta, 3, m)
        d, idx = gi.tau_pairs(t, beta)
        Pd = np.einsum("is,ns,js->nij", U, np.stack([st.single_pole_P(d, a[s], E[s], beta) for s in range(ni)], 1),
                       U.conj())
        W = st.screen_tau(Pd[idx], np.full(ni, v), t)
        Wex = np.einsum("is,ns,js->nij", U,
                        np.stack([st.single_pole_Wt(t, a[s], E[s], v, beta) for s in range(ni)], 1), U.conj())
        errs.append(np.abs(W - Wex).max() / np.abs(Wex).max())
        assert np.abs(W - np.conj(np.swapaxes(W, 1, 2))).max() < 1e-12 * np.abs(W).max()
    assert errs[0] / errs[1] > 3.5 and errs[1] < 5e-3, errs


# ------------------------------------------------------------------ tau-domain Dyson (Eqs. dysongf-dysong, Sec. III.B.5)
def test_dyson_tau_pieces():
    dt = orc.dyson_tau
    beta = 20.0
    tu = gi.upm_grid(beta, 3, 4)
    t = dt.dense_mesh(tu)
    h = tu[1] - tu[0]
    assert np.allclose(np.diff(t), h) and np.isclose(t[-1], beta)
    assert np.all(np.min(np.abs(tu[:, None] - t[None, :]), axis=1) < 1e-12 * beta)   # the UPM points lie on it
    # natural spline: through the nodes, exact on linear data, and scipy's natural spline
    from scipy.interpolate import CubicSpline
    y = np.sin(tu / 3.0) + 0.1 * tu
    assert np.allclose(dt.natural_spline(tu, y, tu), y, atol=1e-13)
    assert np.allclose(dt.natural_spline(tu, 2.0 * tu - 1.0, t), 2.0 * t - 1.0, atol=1e-12)
    assert np.abs(dt.natural_spline(tu, y, t) - CubicSpline(tu, y, bc_type="natural")(t)).max() < 1e-12
    # antiperiodic extension of G0 against G0's definition below zero: G0(tau < 0) = e^{-E tau} n_F(E)
    n = len(t) - 1
    for E in (0.7, -0.4):
        F = dt._antiperiodic(dt.g0_tau(E, t, beta), n)
        d = (np.arange(2 * n + 1) - n) * h
        nF = 1.0 / (np.exp(beta * E) + 1.0)
        exact = np.where(d < 0, np.exp(-E * d) * nF, -np.exp(-E * d) * (1.0 - nF))
        assert np.allclose(F, exact, rtol=1e-12, atol=0)


def _dyson_err(model, m, beta=20.0):
    dt = orc.dyson_tau
    tu = gi.upm_grid(beta, 3, m)
    if model == "static":
        eps, s = 0.4, -0.15
        G, t = dt.dyson_tau(eps, s, np.zeros(len(tu)), tu)
        ex = dt.g0_tau(eps + s, t, beta)
    else:
        # Sigma^c(i w) = c^2 / (i w - E): G(i w) = 1 / (i w - eps - s - c^2 / (i w - E)) has the two poles
        # r of (x - eps - s)(x - E) = c^2 with weights (r_i - E) / (r_i - r_j)
        eps, s, c, E = 0.4, -0.1, 0.3, -0.6
        G, t = dt.dyson_tau(eps, s, c * c * dt.g0_tau(E, tu, beta), tu)
        r = np.roots([1.0, -(eps + s + E), (eps + s) * E - c * c])
        ex = sum(((ri - E) / (ri - rj)) * dt.g0_tau(ri, t, beta) for ri, rj in [(r[0], r[1]), (r[1], r[0])])
    return np.abs(G - ex).max() / np.abs(ex).max()


@pytest.mark.parametrize("model", ["static", "pole"])
def test_dyson_tau_closed_forms(model):
    """Static shift: G = G0 at eps + s. One-pole Sigma^c: a two-pole G. The kernels jump at zero
    difference, so the trapezoid solve converges at first order."""
    e = [_dyson_err(model, m) for m in (4, 8, 16)]
    assert all(1.8 < e[i] / e[i + 1] < 2.3 for i in range(2)), e
    assert e[-1] < 1.5e-2


# ------------------------------------------------------------------ off-diagonal self-energy (Eqs. sigc, sigx, full band matrix)
def test_offdiag_selfenergy_pins():
    from oracle import offdiag as od
    cr, gr = gi.make_config("nk8_nb16")
    rng = np.random.default_rng(41)
    M = gi.m_for_q(cr, 0)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
    W = -(X @ np.conj(np.swapaxes(X, 1, 2))) / cr.ni                  # Hermitian, like W~(tau)
    Sc, Sx = od.selfenergy_offdiag(M, G, W, cr.v[0], cr.kmq[0], occ, omega=1.3)
    sc, sx, _ = orc.selfenergy(M, G, W, cr.v[0], cr.kmq[0], occ, omega=1.3)
    d = np.arange(cr.nb)
    assert np.allclose(Sc[:, d, d, :].real, sc, rtol=0, atol=1e-12 * np.abs(sc).max())   # the diagonal
    assert np.allclose(Sx[:, d, d].real, sx, rtol=0, atol=1e-12 * np.abs(sx).max())
    assert np.abs(Sc - np.conj(np.swapaxes(Sc, 1, 2))).max() < 1e-12 * np.abs(Sc).max()  # Hermitian
    assert np.abs(Sx - np.conj(np.swapaxes(Sx, 1, 2))).max() < 1e-12 * np.abs(Sx).max()
    # a unitary change of the k-side bands, M -> M U, gives Sigma -> U^+ Sigma U
    U, _ = np.linalg.qr(rng.standard_normal((cr.nb, cr.nb)) + 1j * rng.standard_normal((cr.nb, cr.nb)))
    Sc2, Sx2 = od.selfenergy_offdiag(M @ U, G, W, cr.v[0], cr.kmq[0], occ, omega=1.3)
    assert np.abs(Sc2 - np.einsum("an,kabt,bm->knmt", U.conj(), Sc, U)).max() < 1e-12 * np.abs(Sc).max()
    assert np.abs(Sx2 - np.einsum("an,kab,bm->knm", U.conj(), Sx, U)).max() < 1e-12 * np.abs(Sx).max()


def _matrix_dyson_case(nt, seed=7, nb=6, na=3):
    from oracle import offdiag as od
    gr = gi.make_grid(20.0, nt, nt, nt, ncont=64)
    rng = np.random.default_rng(seed)
    w = (2 * np.asarray(gr.w_idx) + 1) * np.pi / gr.beta
    eps = np.sort(rng.uniform(-1, 1, (1, nb)), 1)

    def herm(s):
        X = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
        return s * (X + X.conj().T) / 2

    Sx, Vx = herm(0.1)[None], herm(0.05)[None]
    E = rng.uniform(-1.5, 1.5, na)
    C = 0.2 * (rng.standard_normal((nb, na)) + 1j * rng.standard_normal((nb, na)))
    Sc = np.einsum("na,aw,ma->nmw", C, 1.0 / (1j * w[None, :] - E[:, None]), C.conj())[None]
    G, occ = od.dyson_matrix_iw(eps, Sx, Vx, Sc, gr)
    # downfolding: Sigma^c(i w) = C (i w - E)^-1 C^+ makes G the system block of the enlarged
    # Hermitian problem [[H~, C], [C^+, diag(E)]], whose tau form is exact by eigendecomposition
    Hb = np.zeros((nb + na, nb + na), complex)
    Hb[:nb, :nb] = np.diag(eps[0]) + Sx[0] - Vx[0]
    Hb[:nb, nb:], Hb[nb:, :nb], Hb[nb:, nb:] = C, C.conj().T, np.diag(E)
    lam, U = np.linalg.eigh(Hb)
    g0, f0 = orc.green_tau0(lam[None, :], gr.tau, gr.beta)
    Gex = np.einsum("na,at,ma->nmt", U[:nb], g0[0], U[:nb].conj())
    occx = (U[:nb] * f0[0][None, :]) @ U[:nb].conj().T
    return gr, (eps, Sx, Vx, Sc), G, occ, Gex, occx


def test_matrix_dyson_pins():
    from oracle import offdiag as od
    errs = []
    for nt in (48, 64):
        gr, args, G, occ, Gex, occx = _matrix_dyson_case(nt)
        errs.append(np.abs(G[0] - Gex).max() / np.abs(Gex).max())
        assert np.abs(G - np.conj(np.swapaxes(G, 1, 2))).max() < 1e-12 * np.abs(G).max()   # Hermitian
    assert errs[1] < 1e-5 and errs[0] > errs[1], errs          # the sparse-grid transform converges
    assert np.abs(occ[0] - occx).max() < 5e-5                  # G(beta^-) from the same transform
    # a unitary change of bands: every matrix -> U^+ X U gives G -> U^+ G U
    eps, Sx, Vx, Sc = args
    nb = eps.shape[1]
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb)))
    H = np.diag(eps[0]) + Sx[0] - Vx[0]
    G2, _ = od.dyson_matrix_iw(np.zeros((1, nb)), (U.conj().T @ H @ U)[None], np.zeros((1, nb, nb)),
                               np.einsum("an,kabw,bm->knmw", U.conj(), Sc, U), gr)
    assert np.abs(G2 - np.einsum("an,kabt,bm->knmt", U.conj(), G, U)).max() < 1e-12 * np.abs(G).max()
    # diagonal matrices reduce to the diagonal Dyson oracle
    cr, grd = gi.make_config("nk8_nb16")
    w = (2 * np.asarray(grd.w_idx) + 1) * np.pi / grd.beta
    r = np.random.default_rng(1)
    sx, vx = r.uniform(-0.2, 0.2, (cr.nk, cr.nb)), r.uniform(-0.1, 0.1, (cr.nk, cr.nb))
    sc = (r.uniform(0.05, 0.2, (cr.nk, cr.nb)) ** 2)[..., None] / (1j * w - r.uniform(-1, 1, (cr.nk, cr.nb))[..., None])
    Gd, occd = orc.dyson_iw(cr.eps, sx, vx, sc, grd)
    d = np.arange(cr.nb)
    M3 = lambda x: np.einsum("kn,nm->knm", x, np.eye(cr.nb)).astype(complex)  # noqa: E731
    Sm = np.zeros((cr.nk, cr.nb, cr.nb, len(w)), complex)
    Sm[:, d, d, :] = sc
    Gm, occm = od.dyson_matrix_iw(cr.eps, M3(sx), M3(vx), Sm, grd)
    assert np.abs(Gm[:, d, d, :] - Gd).max() < 1e-13 * np.abs(Gd).max()
    assert np.abs(occm[:, d, d] - occd).max() < 1e-12
