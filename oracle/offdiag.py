"""Off-diagonal self-energy in the band basis (Eqs. sigc and sigx without the diagonal
approximation of Sec. III.B; the paper names the full band matrix as future work): test
infrastructure, FP64, plain numpy.

For one q (M[k][I][a][b], a at k - q, b at k):
    Sigma^c_nm(k|tau) = -1/(Omega N_k) sum_j G_j(k - q|tau) sum_IJ conj(M^I_jn) W~_IJ(q|tau) M^J_jm,
    Sigma^x_nm(k)     = -1/(Omega N_k) sum_j occ_j(k - q) sum_I v_I conj(M^I_jn) M^I_jm.

Parity status: pinned in tests/test_oracle.py by its diagonal (the pinned diagonal self-energy
of oracle.selfenergy), by Hermiticity for Hermitian W~(tau), and by covariance under a unitary
change of the k-side band basis (M -> M U gives Sigma -> U^+ Sigma U), which a dropped
conjugate or transposed index breaks. The matrix Dyson update (dyson_matrix_iw) is pinned by
the downfolding closed form of a pole self-energy (converging with the grid), its reduction to
the diagonal oracle and unitary covariance; it has no GPU counterpart yet.
"""
import numpy as np


def selfenergy_offdiag(M, G, W_tau, v, kmq, occ, omega=1.0):
    """Sigma^c [nk][nb][nb][ntau] (complex) and Sigma^x [nk][nb][nb] (complex) of one q."""
    nk, ni, nb, _ = M.shape
    ntau = W_tau.shape[0]
    pref = -1.0 / (omega * nk)
    Sc = np.zeros((nk, nb, nb, ntau), complex)
    Sx = np.zeros((nk, nb, nb), complex)
    for k in range(nk):
        A = M[k]                                              # [I][j][n]
        Gk = G[kmq[k]]                                        # [j][tau]
        for it in range(ntau):
            Y = np.einsum("IJ,Jjm->Ijm", W_tau[it], A)        # (W~ a_jm)_I
            Sc[k, :, :, it] = pref * np.einsum("j,Ijn,Ijm->nm", Gk[:, it], A.conj(), Y)
        Sx[k] = pref * np.einsum("j,I,Ijn,Ijm->nm", occ[kmq[k]], v, A.conj(), A)
    return Sc, Sx


def dyson_matrix_iw(eps, Sx, vxc, Sc_iw, grid):
    """Dyson update of the full band matrix (Eqs. dysongf-zcjk without the diagonal approximation),
    posed in i w_n like the diagonal oracle.dyson_iw, for every k:
        G(k|i w) = [i w - H~ - Sigma^c(k|i w)]^-1,   H~ = diag(eps) + Sigma^x - Sigma_0,
    Sigma_0 = vxc (matrices). Back to tau: subtract (i w - H~)^-1, whose tau form is
    U diag(G0(lambda, tau)) U^+ (H~ = U diag(lambda) U^+), and map the O(w^-2) remainder R with the
    fermionic backward transform of real tau-functions: Re G_nm(tau) from (R_nm + R_mn) / 2 and
    Im G_nm(tau) from (R_nm - R_mn) / 2i (G(-i w) = G(i w)^+).

    eps [nk][nb]; Sx, vxc [nk][nb][nb] (Hermitian); Sc_iw [nk][nb][nb][nw]. Returns
    G [nk][nb][nb][ntau] (complex, Hermitian at each tau) and the occupation matrices -G(beta^-)."""
    from .gw import green_tau0
    from .transforms import apply_bwd_real, transform_matrices
    T = transform_matrices(grid)
    beta = grid.beta
    w = (2 * np.asarray(grid.w_idx) + 1) * np.pi / beta
    nk, nb = np.asarray(eps).shape
    nt = len(grid.tau)
    G = np.zeros((nk, nb, nb, nt), complex)
    occ = np.zeros((nk, nb, nb), complex)
    for k in range(nk):
        Ht = np.diag(eps[k]).astype(complex) + Sx[k] - vxc[k]
        lam, U = np.linalg.eigh(Ht)
        R = np.empty((nb, nb, len(w)), complex)
        for iw, wn in enumerate(w):
            Giw = np.linalg.inv(1j * wn * np.eye(nb) - Ht - Sc_iw[k, :, :, iw])
            Gref = (U / (1j * wn - lam)[None, :]) @ U.conj().T
            R[:, :, iw] = Giw - Gref
        g0, f0 = green_tau0(lam[None, :], grid.tau, beta)          # [1][nb][ntau], [1][nb]
        G[k] = np.einsum("na,at,ma->nmt", U, g0[0], U.conj())
        occ[k] = (U * f0[0][None, :]) @ U.conj().T
        ghat = 0.5 * (R + np.swapaxes(R, 0, 1))
        hhat = -0.5j * (R - np.swapaxes(R, 0, 1))
        re = apply_bwd_real(T["F_bwd_re"], T["F_bwd_im"], ghat.reshape(nb * nb, -1)).reshape(nb, nb, nt)
        im = apply_bwd_real(T["F_bwd_re"], T["F_bwd_im"], hhat.reshape(nb * nb, -1)).reshape(nb, nb, nt)
        G[k] += re + 1j * im
        gb = lambda X: (X.real @ T["F_bwd_beta_re"]) + (X.imag @ T["F_bwd_beta_im"])  # noqa: E731
        occ[k] -= (gb(ghat.reshape(nb * nb, -1)) + 1j * gb(hhat.reshape(nb * nb, -1))).reshape(nb, nb)
    return G, occ
