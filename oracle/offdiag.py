"""Off-diagonal self-energy in the band basis (Eqs. sigc and sigx without the diagonal
approximation of Sec. III.B; the paper names the full band matrix as future work): test
infrastructure, FP64, plain numpy.

For one q (M[k][I][a][b], a at k - q, b at k):
    Sigma^c_nm(k|tau) = -1/(Omega N_k) sum_j G_j(k - q|tau) sum_IJ conj(M^I_jn) W~_IJ(q|tau) M^J_jm,
    Sigma^x_nm(k)     = -1/(Omega N_k) sum_j occ_j(k - q) sum_I v_I conj(M^I_jn) M^I_jm.

Parity status: pinned in tests/test_oracle.py by its diagonal (the pinned diagonal self-energy
of oracle.selfenergy), by Hermiticity for Hermitian W~(tau), and by covariance under a unitary
change of the k-side band basis (M -> M U gives Sigma -> U^+ Sigma U), which a dropped
conjugate or transposed index breaks.
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
