"""Analytic continuation and quasiparticle energies (Sec. III.B.6), FP64, plain
loops (test infrastructure; see the package docstring).

* Pade: Vidberg-Serene continued fraction (J. Low Temp. Phys. 29, 179 (1977)),
  the comparison method named in the paper.
* CPE: continuous-pole expansion (Staar et al. 2014, the paper's Eqs. after
  Eq. trans): Im Sigma(w + i eta) is piecewise linear on a real grid with
  coefficients of fixed sign (causality, Im Sigma <= 0), so
  Sigma(z) = sum_m b_m Phi_m(z),  b_m >= 0,  Phi_m(z) = int h_m(x) / (z - x) dx
  with h_m the hat function at node x_m. The b are the non-negative
  least-squares minimisers of sum_n |Sigma~(i w_n) - Sigma(i w_n)|^2
  (Lawson-Hanson NNLS via SciPy).
* QP: root of E - eps - Sigma^x + Sigma_0 - Re Sigma^c(E) = 0 nearest eps with positive
  quasiparticle weight (G(w) = 1/[G0(w)^-1 - Sigma^xc(w) - Sigma^H] peaks where this vanishes).
"""
from __future__ import annotations

import numpy as np
import scipy.optimize as _so


# ---------------------------------------------------------------- Pade
def pade_coeffs(z, u):
    """Continued-fraction coefficients a_p from points z_p and values u_p:
    g_1(z_i) = u_i; g_p(z_i) = (g_{p-1}(z_{p-1}) - g_{p-1}(z_i)) / ((z_i - z_{p-1}) g_{p-1}(z_i));
    a_p = g_p(z_p)."""
    z = np.asarray(z, complex)
    g = np.array(u, complex)
    n = len(z)
    a = np.zeros(n, complex)
    a[0] = g[0]
    for p in range(1, n):
        prev = g[p - 1]
        for i in range(p, n):
            g[i] = (prev - g[i]) / ((z[i] - z[p - 1]) * g[i])
        a[p] = g[p]
    return a


def pade_eval(a, z, x):
    """C(x) = a_1 / (1 + a_2 (x - z_1) / (1 + a_3 (x - z_2) / (1 + ...))), bottom-up."""
    x = np.asarray(x, complex)
    n = len(a)
    t = np.ones_like(x)
    for p in range(n - 1, 0, -1):
        t = 1.0 + a[p] * (x - z[p - 1]) / t
    return a[0] / t


# ---------------------------------------------------------------- CPE
def cpe_grid(nhat=128, xmin=0.01, xmax=200.0):
    """Real-frequency nodes x_0 < ... < x_{nhat+1}: +-geomspace(xmin, xmax, nhat/2)
    plus end nodes +-xmax * r (r the geometric ratio); hats sit on the nhat
    interior nodes and vanish at the two end nodes."""
    h = nhat // 2
    g = np.geomspace(xmin, xmax, h)
    r = g[1] / g[0]
    x = np.concatenate([[-xmax * r], -g[::-1], g, [xmax * r]])
    return x


def cpe_kernel(x, z):
    """Phi_m(z) = int h_m(s)/(z - s) ds for hats on interior nodes x_1..x_M.

    Rising part on [x0, x1] (h = x1 - x0): ((z - x0)/h) (log(z - x0) - log(z - x1)) - 1.
    Falling part on [x1, x2] (h' = x2 - x1): ((x2 - z)/h') (log(z - x1) - log(z - x2)) + 1.
    Principal logs; z in the upper half plane (or real, taken from above).
    Returns [len(z), M] complex."""
    z = np.asarray(z, complex)[:, None]
    x0, x1, x2 = x[None, :-2], x[None, 1:-1], x[None, 2:]
    l0 = np.log(z - x0)
    l1 = np.log(z - x1)
    l2 = np.log(z - x2)
    rise = (z - x0) / (x1 - x0) * (l0 - l1) - 1.0
    fall = (x2 - z) / (x2 - x1) * (l1 - l2) + 1.0
    return rise + fall


def cpe_fit(w, sig, x, ridge=0.0):
    """b >= 0 minimising sum_n |sig_n - sum_m b_m Phi_m(i w_n)|^2 + lambda^2 |b|^2,
    lambda = ridge * ||A||_F (A the real-stacked kernel; ridge = 0 is the plain CPE
    norm). Solved as NNLS on the stacked matrix [A; lambda I]. Returns (b, residual norm)."""
    K = cpe_kernel(x, 1j * np.asarray(w))
    A = np.vstack([K.real, K.imag])
    y = np.concatenate([np.asarray(sig).real, np.asarray(sig).imag])
    if ridge > 0:
        lam = ridge * np.linalg.norm(A)
        A = np.vstack([A, lam * np.eye(A.shape[1])])
        y = np.concatenate([y, np.zeros(A.shape[1])])
    b, res = _so.nnls(A, y, maxiter=50 * A.shape[1])
    return b, res


def cpe_eval(b, x, z):
    return cpe_kernel(x, z) @ b


ETA = 1e-4  # real-axis offset (Ha) at which continued self-energies are evaluated


def pade_resig(a, z):
    """Re Sigma(E + i eta) of a Pade continued fraction, for a scalar or an array of E."""
    return lambda E: pade_eval(a, z, np.asarray(E, float) + 1j * ETA).real


def cpe_resig(b, x):
    """Re Sigma(E + i eta) of a CPE fit, for a scalar or an array of E."""
    def f(E):
        E = np.asarray(E, float)
        return (cpe_kernel(x, E.reshape(-1) + 1j * ETA) @ b).real.reshape(E.shape)
    return f


# ---------------------------------------------------------------- QP
QP_WINDOW = 1.0      # Ha: quasiparticle energies are searched within eps +- QP_WINDOW
QP_H = 2.5e-4        # Ha: spacing of the sign search, on points eps + i QP_H


def qp_roots(eps, sigx, vxc, resig):
    """Every zero of F(E) = E - eps - sigx + vxc - Re Sigma^c(E) in eps +- QP_WINDOW at which F
    rises (F' > 0, i.e. quasiparticle weight Z = 1/F' > 0), ascending.

    Zeros are bracketed by the sign changes F(E_i) < 0 <= F(E_{i+1}) on the points
    E_i = eps + i QP_H, |i| <= QP_WINDOW / QP_H (a mesh centred on the problem's own eps), and
    each bracket is refined by Brent's method to the last bit."""
    n = int(round(QP_WINDOW / QP_H))
    Es = eps + QP_H * np.arange(-n, n + 1)
    Fs = Es - eps - sigx + vxc - np.asarray(resig(Es), float)
    F = lambda E: E - eps - sigx + vxc - float(np.asarray(resig(np.array([E])))[0])  # noqa: E731
    roots = []
    for i in np.nonzero((Fs[:-1] < 0.0) & (Fs[1:] >= 0.0))[0]:
        if Fs[i + 1] == 0.0:
            roots.append(float(Es[i + 1]))
        else:
            roots.append(_so.brentq(F, Es[i], Es[i + 1], xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=200))
    return roots


def qp_solve(eps, sigx, vxc, resig, de=1e-6, tol=1e-12, maxit=100):
    """Quasiparticle energy (Sec. III.B.6): the pole of G(w) = 1/[w - eps - Sigma^x + Sigma_0 - Sigma^c(w)]
    nearest the reference energy eps, i.e. the zero of F(E) = E - eps - sigx + vxc - Re Sigma^c(E)
    with positive weight Z = 1/F'(E) that lies nearest eps (the paper takes one solution per
    state; where F has several zeros this is the reading taken). The candidates are those of
    qp_roots. Without any, Newton iteration from eps (central-difference derivative, steps
    clamped to 0.5 Ha) is the fallback. Returns (E, Z, ok) with ok False for the fallback."""
    roots = qp_roots(eps, sigx, vxc, resig)
    r1 = lambda E: float(np.asarray(resig(np.array([E])))[0])  # noqa: E731
    if roots:
        E = min(roots, key=lambda r: abs(r - eps))
        ok = True
    else:
        E = float(eps)
        ok = False
        for _ in range(maxit):
            Fv = E - eps - sigx + vxc - r1(E)
            dF = 1.0 - (r1(E + de) - r1(E - de)) / (2 * de)
            if dF == 0 or not np.isfinite(dF):
                break
            step = max(-0.5, min(0.5, Fv / dF))
            E -= step
            if abs(step) < tol * max(1.0, abs(E)):
                break
    dS = (r1(E + de) - r1(E - de)) / (2 * de)
    return E, 1.0 / (1.0 - dS), ok


def band_gap(E, nocc):
    """min_k E[k, nocc] - max_k E[k, nocc-1] (0-based band index)."""
    E = np.asarray(E)
    return E[:, nocc].min() - E[:, nocc - 1].max()
