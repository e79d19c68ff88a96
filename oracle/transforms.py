"""Imaginary-time <-> Matsubara transforms of the oracle, built in 60-digit
decimal arithmetic (test infrastructure; see the package docstring).

The paper transforms Sigma(tau) to Sigma(i w_n) = int_0^beta e^{i w_n tau}
Sigma(tau) dtau (Eq. trans) and solves the screened interaction in tau
(Eq. tildeW). The GPU path poses the screening at bosonic Matsubara
frequencies instead, so it needs tau -> i nu, i nu -> tau, tau -> i w and
i w -> tau maps. All of them are read off one model: a real-valued function
of tau on [0, beta] is a sum of Lehmann kernels

    f(tau) = sum_l c_l K(tau, E_l),   K(tau, E) = exp(-E tau) / (1 + exp(-beta E))

(E < 0 written as exp(E (beta - tau)) / (1 + exp(beta E))), whose transform
at any Matsubara frequency is closed form:

    fermionic  int_0^beta e^{i w tau} K dtau = -1 / (i w - E)
    bosonic    int_0^beta e^{i nu tau} K dtau = -tanh(beta E / 2) / (i nu - E)
               (beta / 2 at nu = E = 0)

* forward (tau -> i z):  c = least-squares fit of f(tau_i); f(i z_j) = sum_l c_l Khat(z_j, E_l)
* backward (i z -> tau): real c = least-squares fit of Re/Im f(i z_j); f(tau_i) = sum_l c_l K(tau_i, E_l)

The least-squares problems are badly conditioned (cond ~ 1e9 on the
Gauss-Legendre-in-log grids), so the matrices are formed in decimal
arithmetic with 60 significant digits and rounded to FP64 once at the end.
"""
from __future__ import annotations

import functools
from decimal import Decimal, localcontext

import numpy as np

_PI = Decimal("3.14159265358979323846264338327950288419716939937510582097494459230781640628620899")
_PREC = 60


def _kernel_tau(tau, E, beta):
    """K(tau, E) in decimal, overflow-free form chosen by the sign of E."""
    one = Decimal(1)
    if E >= 0:
        return (-E * tau).exp() / (one + (-beta * E).exp())
    return (E * (beta - tau)).exp() / (one + (beta * E).exp())


def _kernel_hat(n, E, beta, fermionic):
    """Matsubara transform of K(., E) at index n: returns (re, im) decimals."""
    z = ((2 * n + 1) if fermionic else (2 * n)) * _PI / beta
    den = z * z + E * E
    if fermionic:
        # -1/(i z - E) = (E + i z) / (z^2 + E^2)
        return E / den, z / den
    if n == 0 and E == 0:
        return beta / 2, Decimal(0)
    one = Decimal(1)
    if E >= 0:
        x = (-beta * E).exp()
        th = (one - x) / (one + x)
    else:
        x = (beta * E).exp()
        th = -(one - x) / (one + x)
    # -tanh(beta E/2)/(i z - E) = tanh(beta E/2) (E + i z)/(z^2 + E^2)
    return th * E / den, th * z / den


def _solve_normal(A, B):
    """Least-squares solution X of A X = B via normal equations, in decimal.

    A: list of rows (m x p); B: list of rows (m x r). Gauss-Jordan elimination
    with partial pivoting on A^T A (p x p)."""
    m, p = len(A), len(A[0])
    r = len(B[0])
    N = [[sum(A[i][a] * A[i][b] for i in range(m)) for b in range(p)] for a in range(p)]
    R = [[sum(A[i][a] * B[i][c] for i in range(m)) for c in range(r)] for a in range(p)]
    for col in range(p):
        piv = max(range(col, p), key=lambda i: abs(N[i][col]))
        N[col], N[piv] = N[piv], N[col]
        R[col], R[piv] = R[piv], R[col]
        d = N[col][col]
        inv = Decimal(1) / d
        N[col] = [x * inv for x in N[col]]
        R[col] = [x * inv for x in R[col]]
        for i in range(p):
            if i != col and N[i][col] != 0:
                f = N[i][col]
                N[i] = [x - f * y for x, y in zip(N[i], N[col])]
                R[i] = [x - f * y for x, y in zip(R[i], R[col])]
    return R


def _pinv_rows(A):
    """Pseudo-inverse (p x m) of the m x p decimal matrix A."""
    m = len(A)
    eye = [[Decimal(1) if i == j else Decimal(0) for j in range(m)] for i in range(m)]
    return _solve_normal(A, eye)


@functools.lru_cache(maxsize=16)
def _matrices_cached(key):
    beta_f, tau_t, poles_t, nu_t, w_t, ncont = key
    with localcontext() as ctx:
        ctx.prec = _PREC
        beta = Decimal(beta_f)
        tau = [Decimal(t) for t in tau_t]
        E = [Decimal(e) for e in poles_t]
        Kt = [[_kernel_tau(t, e, beta) for e in E] for t in tau]       # ntau x npole
        Kbeta = [_kernel_tau(beta, e, beta) for e in E]                # tau = beta^-
        Kzero = [_kernel_tau(Decimal(0), e, beta) for e in E]          # tau = 0^+
        Kt_pinv = _pinv_rows(Kt)                                       # npole x ntau

        def fwd(idx, fermionic):
            out_re, out_im = [], []
            for n in idx:
                h = [_kernel_hat(int(n), e, beta, fermionic) for e in E]
                re = [sum(h[l][0] * Kt_pinv[l][i] for l in range(len(E))) for i in range(len(tau))]
                im = [sum(h[l][1] * Kt_pinv[l][i] for l in range(len(E))) for i in range(len(tau))]
                out_re.append(re)
                out_im.append(im)
            return (np.array([[float(x) for x in row] for row in out_re])
                    + 1j * np.array([[float(x) for x in row] for row in out_im]))

        def bwd(idx, fermionic):
            rows = []
            for n in idx:
                h = [_kernel_hat(int(n), e, beta, fermionic) for e in E]
                rows.append([x[0] for x in h])
            for n in idx:
                h = [_kernel_hat(int(n), e, beta, fermionic) for e in E]
                rows.append([x[1] for x in h])
            Hp = _pinv_rows(rows)                                      # npole x 2 nidx
            nz = len(idx)
            T = [[sum(Kt[i][l] * Hp[l][j] for l in range(len(E))) for j in range(2 * nz)]
                 for i in range(len(tau))]
            Tb = [sum(Kbeta[l] * Hp[l][j] for l in range(len(E))) for j in range(2 * nz)]
            Tz = [sum(Kzero[l] * Hp[l][j] for l in range(len(E))) for j in range(2 * nz)]
            T = np.array([[float(x) for x in row] for row in T])
            Tb = np.array([float(x) for x in Tb])
            Tz = np.array([float(x) for x in Tz])
            return T[:, :nz], T[:, nz:], Tb[:nz], Tb[nz:], Tz[:nz], Tz[nz:]

        out = {}
        out["B_fwd"] = fwd(nu_t, False)
        out["F_fwd"] = fwd(w_t, True)
        out["F_cont"] = fwd(tuple(range(ncont)), True)
        bre, bim, _, _, _, _ = bwd(nu_t, False)
        out["B_bwd_re"], out["B_bwd_im"] = bre, bim
        fre, fim, fbre, fbim, fzre, fzim = bwd(w_t, True)
        out["F_bwd_re"], out["F_bwd_im"] = fre, fim
        out["F_bwd_beta_re"], out["F_bwd_beta_im"] = fbre, fbim
        out["F_bwd_zero_re"], out["F_bwd_zero_im"] = fzre, fzim
        # value at tau = beta^- / 0^+ of the tau-fit
        out["tau_to_beta"] = np.array([float(sum(Kbeta[l] * Kt_pinv[l][i] for l in range(len(E))))
                                       for i in range(len(tau))])
        out["tau_to_zero"] = np.array([float(sum(Kzero[l] * Kt_pinv[l][i] for l in range(len(E))))
                                       for i in range(len(tau))])
        return out


def transform_matrices(grid):
    """All transform matrices of a gwinputs.Grid (cached per grid).

    Returns a dict of FP64 arrays:
      B_fwd  [nnu, ntau] complex : f(i nu_j)  = B_fwd  @ f(tau)        (bosonic)
      F_fwd  [nw,  ntau] complex : f(i w_j)   = F_fwd  @ f(tau)        (fermionic sparse set)
      F_cont [ncont, ntau] complex: f(i w_n), n = 0..ncont-1           (continuation set)
      B_bwd_re/B_bwd_im [ntau, nnu] real : g(tau) = re @ Re g(i nu) + im @ Im g(i nu)
                                           for a REAL function g of tau
      F_bwd_re/F_bwd_im [ntau, nw] real  : same for fermionic frequencies
      F_bwd_beta_re/im [nw] : value at tau = beta^- of the backward fit
      F_bwd_zero_re/im [nw] : value at tau = 0^+ of the backward fit
      tau_to_beta / tau_to_zero [ntau] : value at beta^- / 0^+ of the tau fit
    """
    key = (float(grid.beta), tuple(float(t) for t in grid.tau),
           tuple(float(e) for e in grid.poles), tuple(int(n) for n in grid.nu_idx),
           tuple(int(n) for n in grid.w_idx), int(grid.ncont))
    return _matrices_cached(key)


def apply_fwd(T, f_tau):
    """f_tau [..., ntau] complex or real -> [..., nfreq] complex."""
    return np.einsum("ji,...i->...j", T, f_tau)


def apply_bwd_real(Tre, Tim, g_freq):
    """Backward map for a real tau-function: g_freq [..., nfreq] complex -> [..., ntau] real."""
    return np.einsum("ij,...j->...i", Tre, g_freq.real) + np.einsum("ij,...j->...i", Tim, g_freq.imag)


def apply_bwd_hermitian(Tre, Tim, W_freq):
    """Backward bosonic map of a Hermitian-matrix-valued function.

    W_freq [nnu, n, n] holds W(i nu_j) for nu_j >= 0. W(tau) is Hermitian, so
    its real part g = Re W(tau) (symmetric) and imaginary part h = Im W(tau)
    (antisymmetric) are real tau-functions with transforms
    ghat = (W + W^T)/2 and hhat = (W - W^T)/(2i)  (W(-i nu) = W(i nu)^dagger).
    Returns W(tau) [ntau, n, n] complex.
    """
    Wt = np.swapaxes(W_freq, -1, -2)
    ghat = 0.5 * (W_freq + Wt)
    hhat = (W_freq - Wt) / 2j
    g = np.einsum("ij,jab->iab", Tre, ghat.real) + np.einsum("ij,jab->iab", Tim, ghat.imag)
    h = np.einsum("ij,jab->iab", Tre, hhat.real) + np.einsum("ij,jab->iab", Tim, hhat.imag)
    return g + 1j * h
