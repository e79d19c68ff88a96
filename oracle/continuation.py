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

import math

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
    return lambda E: pade_eval(a, z, np.array([E + 1j * ETA]))[0].real


def cpe_resig(b, x):
    return lambda E: (cpe_kernel(x, np.array([E + 1j * ETA])) @ b)[0].real


# ---------------------------------------------------------------- QP
QP_STEP = 0.005      # Ha: the scan visits the energies j * QP_STEP within eps +- QP_RANGE
QP_RANGE = 1.0       # Ha
QP_BISECT = 60


def qp_solve(eps, sigx, vxc, resig, de=1e-6, tol=1e-12, maxit=100):
    """Quasiparticle energy: root of F(E) = E - eps - sigx + vxc - Re Sigma^c(E) nearest eps
    (G(w) = 1/[G0(w)^-1 - Sigma^xc(w) - Sigma^H] peaks where F vanishes).

    F is scanned on the fixed energy grid E_j = j 0.005 Ha, for the integers j with
    eps - 1 <= E_j <= eps + 1 Ha (j from ceil((eps - 1) / 0.005) to floor((eps + 1) / 0.005));
    among the upward crossings F_j < 0 <= F_{j+1} (quasiparticle weight Z > 0) the one whose
    midpoint is nearest eps is refined by 60 bisections. Without a crossing, Newton iteration from eps (central-difference
    derivative, steps clamped to 0.5 Ha) is the fallback. Returns (E, Z, ok) with ok False for
    the fallback or a Newton failure."""
    F = lambda E: E - eps - sigx + vxc - resig(E)  # noqa: E731
    j0 = math.ceil((eps - QP_RANGE) / QP_STEP)
    j1 = math.floor((eps + QP_RANGE) / QP_STEP)
    Es = [j * QP_STEP for j in range(j0, j1 + 1)]
    Fs = [F(E) for E in Es]
    best = None
    for j in range(len(Es) - 1):
        if Fs[j] < 0.0 <= Fs[j + 1]:
            d = abs(0.5 * (Es[j] + Es[j + 1]) - eps)
            if best is None or d < best[0]:
                best = (d, j)
    if best is not None:
        lo, hi = Es[best[1]], Es[best[1] + 1]
        for _ in range(QP_BISECT):
            mid = 0.5 * (lo + hi)
            if F(mid) < 0.0:
                lo = mid
            else:
                hi = mid
        E = 0.5 * (lo + hi)
        ok = True
    else:
        E = float(eps)
        ok = False
        for _ in range(maxit):
            Fv = F(E)
            dF = 1.0 - (resig(E + de) - resig(E - de)) / (2 * de)
            if dF == 0 or not np.isfinite(dF):
                break
            step = max(-0.5, min(0.5, Fv / dF))
            E -= step
            if abs(step) < tol * max(1.0, abs(E)):
                break
    dS = (resig(E + de) - resig(E - de)) / (2 * de)
    return E, 1.0 / (1.0 - dS), ok


def band_gap(E, nocc):
    """min_k E[k, nocc] - max_k E[k, nocc-1] (0-based band index)."""
    E = np.asarray(E)
    return E[:, nocc].min() - E[:, nocc - 1].max()
