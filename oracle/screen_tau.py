"""The paper's tau-domain form of the screened interaction (Sec. III.B.3, Eq. tildeW), after
Stan et al.: test infrastructure, FP64, plain numpy.

W~(tau) = W(tau) - v delta(tau) obeys W~(tau) = v P(tau) v + int_0^beta dtau' v P(tau - tau') W~(tau').
On a grid tau_0 = 0 < tau_1 < ... < tau_M = beta with the trapezoid increments of the paper
(dtau_i = (tau_{i+1} - tau_{i-1}) / 2 inside, half the end intervals at both ends) this becomes
one linear system of (M + 1) NI unknowns per column J':

    sum_r sum_J [delta_IJ delta_pr - A_IJ(tau_p - tau_r) dtau_r] W~_JJ'(tau_r) = A_IJ'(tau_p) v_J',
    A(tau) = v P(tau)   (v diagonal in the product basis).

P is bosonic: P(tau - beta) = P(tau), so a negative difference is taken modulo beta, and both
tau_p - tau_r = 0 and = +-beta use P(0).

Parity status: pinned in tests/test_oracle.py by the single-pole closed form (W~(tau) of a
one-mode polarization, reached at second order in the step as the grid is refined), by its
matrix version in a common eigenbasis, and by the exactness of the increments on linear
functions.
"""
import numpy as np


def trapezoid_weights(tau):
    """The increments dtau_r of Eq. (tildeW) (Sec. III.B.3): (tau_{r+1} - tau_{r-1}) / 2 for
    0 < r < M, (tau_1 - tau_0) / 2 and (tau_M - tau_{M-1}) / 2 at the ends."""
    tau = np.asarray(tau, float)
    d = np.empty_like(tau)
    d[1:-1] = 0.5 * (tau[2:] - tau[:-2])
    d[0] = 0.5 * (tau[1] - tau[0])
    d[-1] = 0.5 * (tau[-1] - tau[-2])
    return d


def screen_tau(P_pair, v, tau):
    """W~(tau_r), r = 0..M, from Eq. (tildeW) in the tau domain (Sec. III.B.3).

    P_pair: complex [npts][npts][ni][ni], P_pair[p][r] = P(tau_p - tau_r) (bosonic, modulo beta);
    v: [ni] diagonal Coulomb; tau: [npts] with tau_0 = 0 and tau_M = beta.
    Returns complex [npts][ni][ni].
    """
    P_pair = np.asarray(P_pair, complex)
    v = np.asarray(v, float)
    npts, ni = P_pair.shape[0], P_pair.shape[2]
    dt = trapezoid_weights(tau)
    n = npts * ni
    K = np.zeros((n, n), complex)
    B = np.zeros((n, ni), complex)
    for p in range(npts):
        for r in range(npts):
            A = v[:, None] * P_pair[p, r]                      # A(tau_p - tau_r) = v P
            blk = -A * dt[r]
            if p == r:
                blk = blk + np.eye(ni)
            K[p * ni:(p + 1) * ni, r * ni:(r + 1) * ni] = blk
        B[p * ni:(p + 1) * ni, :] = (v[:, None] * P_pair[p, 0]) * v[None, :]   # A(tau_p) v, tau_0 = 0
    X = np.linalg.solve(K, B)
    return X.reshape(npts, ni, ni)


def single_pole_P(tau, a, E, beta):
    """P(tau) = -a cosh(E (tau - beta/2)) / sinh(E beta / 2) for 0 <= tau <= beta: the
    polarization whose Matsubara transform is -2 a E / (nu^2 + E^2) (one bosonic mode)."""
    tau = np.asarray(tau, float)
    return -a * np.cosh(E * (tau - 0.5 * beta)) / np.sinh(0.5 * E * beta)


def single_pole_Wt(tau, a, E, v, beta):
    """Closed form of W~(tau) for that P and a scalar v: W~(i nu) = v^2 P / (1 - v P) =
    -2 a v^2 E / (nu^2 + Om^2) with Om^2 = E^2 + 2 a v E, whose transform to tau is
    -a v^2 E cosh(Om (tau - beta/2)) / (Om sinh(Om beta / 2))."""
    tau = np.asarray(tau, float)
    om = np.sqrt(E * E + 2.0 * a * v * E)
    return -a * v * v * E * np.cosh(om * (tau - 0.5 * beta)) / (om * np.sinh(0.5 * om * beta))
