"""Plain FP64 statement of the GW cycle (test infrastructure; see the package docstring).

Notation follows Chu et al. (arXiv:1602.02313), Sec. III.B, with the pair
index relabelled so that one matrix-element tensor serves Eqs. (irpol) and
(sigc): M[k, I, a, b] = M^I_ab(k, q) with band a at k - q and band b at k.
Energies are in Ha, relative to the chemical potential mu = 0.
"""
from __future__ import annotations

import numpy as np

from .transforms import (apply_bwd_hermitian, apply_bwd_real, apply_fwd,
                         transform_matrices)

__all__ = ["green_tau0", "polarization", "screen", "selfenergy", "sigma_tau_to_iw",
           "dyson_iw", "tau_to_nu", "nu_to_tau", "mirror_index", "lindhard_iv",
           "green_iw0"]


def mirror_index(ntau):
    """Position of beta - tau_i in the (mirror-symmetric) tau grid."""
    return np.arange(ntau)[::-1]


def green_tau0(eps, tau, beta):
    """Reference Green's function, Sec. III.B.1:
    G0_j(k|tau) = -exp(-eps tau) [1 - n_F(eps)], 0 <= tau <= beta,
    written without overflow: for eps > 0 as -exp(-eps tau)/(1 + exp(-beta eps)),
    for eps <= 0 as -exp(eps (beta - tau))/(1 + exp(beta eps)).
    Also returns the occupations f = G(0^-) = -G(beta^-) = n_F(eps)
    (Sec. III.B.3, after Eq. sigx).
    """
    eps = np.asarray(eps, float)[..., None]
    tau = np.asarray(tau, float)
    pos = eps > 0
    a = np.abs(eps)
    den = 1.0 + np.exp(-beta * a)
    G = np.where(pos, -np.exp(-a * tau) / den, -np.exp(-a * (beta - tau)) / den)
    e = eps[..., 0]
    occ = np.where(e > 0, np.exp(-beta * np.abs(e)) / (1.0 + np.exp(-beta * np.abs(e))),
                   1.0 / (1.0 + np.exp(-beta * np.abs(e))))
    return G, occ


def green_iw0(eps, w_idx, beta):
    """G0(i w_n) = 1 / (i w_n - eps), the transform of green_tau0 (Eq. trans)."""
    w = (2 * np.asarray(w_idx) + 1) * np.pi / beta
    return 1.0 / (1j * w[None, None, :] - np.asarray(eps)[..., None])


def polarization(M, G, kmq, omega=1.0, its=None):
    """Irreducible polarization for one q, Eq. (irpol):

    P_II'(q|tau) = 1/(Omega N_k) sum_k sum_ab M^I_ab Q_ab(k, q|tau) conj(M^I'_ab),
    Q_ab = G_b(k|tau) G_a(k - q|-tau),  G(-tau) = -G(beta - tau)  (Sec. II),

    M: [nk, ni, nb, nb] complex (a at k - q, b at k); G: [nk, nb, ntau] real;
    kmq: [nk] index of k - q. Spin factor 1 (spinor M). Returns [ntau, ni, ni]
    (or [len(its), ni, ni] for the tau indices its).
    """
    nk, ni, nb, _ = M.shape
    ntau = G.shape[-1]
    mir = mirror_index(ntau)
    its = list(range(ntau)) if its is None else list(its)
    P = np.zeros((len(its), ni, ni), complex)
    for o, i in enumerate(its):
        acc = np.zeros((ni, ni), complex)
        for k in range(nk):
            Gb = G[k, :, i]                       # G_b(k|tau)
            Ga_m = -G[kmq[k], :, mir[i]]          # G_a(k-q|-tau) = -G_a(k-q|beta - tau)
            Q = Ga_m[:, None] * Gb[None, :]       # [a, b]
            A = M[k].reshape(ni, nb * nb)
            acc += (A * Q.reshape(-1)[None, :]) @ A.conj().T
        P[o] = acc / (omega * nk)
    return P


def lindhard_iv(M, eps, kmq, nu_idx, beta, omega=1.0):
    """Matsubara transform of polarization() for the reference G0, in closed form:
    P(i nu) = 1/(Omega N_k) sum M M* (f_a - f_b) / (i nu - (eps_b - eps_a)),
    with the nu = 0, eps_a = eps_b limit -beta f (1 - f). Used only to pin
    polarization() and the transforms."""
    nk, ni, nb, _ = M.shape
    _, occ = green_tau0(eps, np.array([0.5]), beta)
    nu = 2 * np.pi * np.asarray(nu_idx) / beta
    out = np.zeros((len(nu), ni, ni), complex)
    for j, z in enumerate(nu):
        for k in range(nk):
            fa = occ[kmq[k]][:, None]
            fb = occ[k][None, :]
            d = eps[k][None, :] - eps[kmq[k]][:, None]
            with np.errstate(divide="ignore", invalid="ignore"):
                w = (fa - fb) / (1j * z - d)
            if z == 0:
                same = np.abs(d) < 1e-14
                w = np.where(same, -beta * fb * (1 - fb), w)
            A = M[k].reshape(ni, nb * nb)
            out[j] += (A * w.reshape(-1)[None, :]) @ A.conj().T
    return out / (omega * nk)


def tau_to_nu(P_tau, grid):
    """P(i nu_j) for nu_j = 2 pi n_j / beta, n_j in grid.nu_idx, of a tau-function
    (transform of Eq. trans at bosonic frequencies). P_tau [ntau, ...]."""
    T = transform_matrices(grid)["B_fwd"]
    return np.einsum("ji,i...->j...", T, P_tau)


def nu_to_tau(W_iv, grid):
    """W(tau) from W(i nu_j), nu_j >= 0, for a Hermitian-matrix function."""
    T = transform_matrices(grid)
    return apply_bwd_hermitian(T["B_bwd_re"], T["B_bwd_im"], W_iv)


def screen(P_iv, v):
    """Screened interaction minus bare Coulomb, W~ = W - v (Sec. III.B.3), posed at
    bosonic Matsubara frequencies where Eq. (tildeW) is algebraic:
    Pi = v^1/2 P v^1/2, solve (1 - Pi) X = Pi, W~ = v^1/2 X v^1/2.
    P_iv [nnu, ni, ni], v [ni] (diagonal Coulomb). Returns [nnu, ni, ni]."""
    sv = np.sqrt(np.asarray(v, float))
    out = np.empty_like(P_iv)
    eye = np.eye(P_iv.shape[-1])
    for j in range(P_iv.shape[0]):
        Pi = sv[:, None] * P_iv[j] * sv[None, :]
        X = np.linalg.solve(eye - Pi, Pi)
        out[j] = sv[:, None] * X * sv[None, :]
    return out


def selfenergy(M, G, W_tau, v, kmq, occ, omega=1.0, ks=None, its=None):
    """Contribution of one q to the correlation and exchange self-energies.

    Eq. (sigc): Sigma^c_n(k|tau) = -1/(Omega N_k) sum_GG' sum_j
                [M^{k-q}_jn(G,q)]^* G_j(k-q|tau) W~_GG'(q|tau) M^{k-q}_jn(G',q)
    Eq. (sigx) in the product basis with diagonal v:
                Sigma^x_n(k) = -1/(Omega N_k) sum_j f_j(k-q) sum_I v_I |M^I_jn|^2.
    M [nk, ni, nb, nb] (j = a at k - q, n = b at k); G [nk, nb, ntau];
    W_tau [ntau, ni, ni]; occ [nk, nb]. Returns (Sigc [nk, nb, ntau] real,
    Sigx [nk, nb]); ks / its restrict the k points and tau indices computed
    (M then holds only those k: M[len(ks), ...], W_tau all tau).
    """
    nkm, ni, nb, _ = M.shape
    nk = G.shape[0]
    ntau = G.shape[-1]
    ks = list(range(nk)) if ks is None else list(ks)
    its = list(range(ntau)) if its is None else list(its)
    sc = np.zeros((nk, nb, ntau), complex)
    sx = np.zeros((nk, nb))
    for m_, k in enumerate(ks):
        A = M[m_].reshape(ni, nb * nb)           # column (a, n)
        for i in its:
            d = (A.conj() * (W_tau[i] @ A)).sum(0).reshape(nb, nb)  # a^H W a per column (a, n)
            sc[k, :, i] = -(G[kmq[k], :, i][:, None] * d).sum(0) / (omega * nk)
        vm = (np.asarray(v)[:, None] * np.abs(A) ** 2).sum(0).reshape(nb, nb)
        sx[k] = -(occ[kmq[k]][:, None] * vm).sum(0) / (omega * nk)
    return sc.real, sx, np.abs(sc.imag).max()


def sigma_tau_to_iw(S_tau, grid, cont=False):
    """Sigma(i w_n) = int_0^beta e^{i w_n tau} Sigma(tau) dtau (Eq. trans) on the sparse
    fermionic set (cont=False) or on the dense first ncont frequencies (cont=True)."""
    T = transform_matrices(grid)["F_cont" if cont else "F_fwd"]
    return apply_fwd(T, S_tau)


def dyson_iw(eps, sigx, vxc, sigc_iw, grid):
    """Diagonal Dyson update of G (Eqs. dysongf, zxjk, zcjk), posed in i w_n:

    G_j(k|i w) = 1 / (i w - eps_j - [Sigma^x_j - Sigma_0,j] - Sigma^c_j(i w)),

    with Sigma_0 = vxc (Hartree change zero under the diagonal approximation).
    Back to tau: subtract 1/(i w - eps~), eps~ = eps + Sigma^x - vxc, whose tau form
    is green_tau0(eps~) exactly, and map the O(w^-2) remainder with the fermionic
    backward transform. Returns (G [nk, nb, ntau], occ = -G(beta^-) [nk, nb])."""
    T = transform_matrices(grid)
    beta = grid.beta
    w = (2 * np.asarray(grid.w_idx) + 1) * np.pi / beta
    et = np.asarray(eps) + np.asarray(sigx) - np.asarray(vxc)
    Giw = 1.0 / (1j * w[None, None, :] - et[..., None] - sigc_iw)
    Gref = 1.0 / (1j * w[None, None, :] - et[..., None])
    R = Giw - Gref
    G0t, occ0 = green_tau0(et, grid.tau, beta)
    G = G0t + apply_bwd_real(T["F_bwd_re"], T["F_bwd_im"], R)
    g_beta = (R.real @ T["F_bwd_beta_re"]) + (R.imag @ T["F_bwd_beta_im"])
    occ = occ0 - g_beta
    return G, occ
