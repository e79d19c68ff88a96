"""The paper's tau-domain Dyson equation for the diagonal Green's function (Sec. III.B.5, Eqs.
dysongf, zxjk, zcjk, dysong): test infrastructure, FP64, plain numpy.

For one state (j, k):
    G(tau) = G0(tau) + int_0^beta dtau2 Z(tau, tau2) G(tau2),
    Z = Z^x + Z^c,  Z^x(tau, tau2) = G0(tau - tau2) s,   s = Sigma^x + Sigma^H - Sigma_0,
    Z^c(tau, tau2) = int_0^beta dtau1 G0(tau - tau1) Sigma^c(tau1 - tau2).
Sigma^c is given on a uniform power mesh; as the paper prescribes it is carried by a cubic
spline to the uniform mesh whose step is the mesh's smallest (tau_1 - tau_0), where every
difference of two points is again a point. Both integrals use the trapezoid rule on that
mesh, and Eq. (dysong) is the linear system
    sum_r [delta_pr - dtau_r Z(tau_p, tau_r)] G(tau_r) = G0(tau_p).
Fermionic functions are antiperiodic: f(tau - beta) = -f(tau), so a negative difference d
takes -f(d + beta); a zero difference takes the value at 0+ (a reading: the paper does not say
which side of the jump).

Parity status: pinned in tests/test_oracle.py by the closed forms of a static shift (G0 at
eps + s) and of a one-pole Sigma^c (two-pole G), reached at first order in the step (the
kernels jump at zero difference), and the spline by exactness on linear data and agreement
with scipy's natural cubic spline.
"""
import numpy as np


def natural_spline(x, y, xe):
    """Natural cubic spline through (x, y) (second derivative zero at both ends), evaluated at
    xe: the second derivatives M solve the tridiagonal system
    h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1} = 6 (d_i - d_{i-1}), d_i = (y_{i+1} - y_i) / h_i."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    n = len(x)
    h = np.diff(x)
    d = np.diff(y) / h
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    A[0, 0] = A[-1, -1] = 1.0
    for i in range(1, n - 1):
        A[i, i - 1], A[i, i], A[i, i + 1] = h[i - 1], 2.0 * (h[i - 1] + h[i]), h[i]
        rhs[i] = 6.0 * (d[i] - d[i - 1])
    M = np.linalg.solve(A, rhs)
    xe = np.asarray(xe, float)
    i = np.clip(np.searchsorted(x, xe, side="right") - 1, 0, n - 2)
    t0, t1 = xe - x[i], x[i + 1] - xe
    hi = h[i]
    return (M[i] * t1 ** 3 + M[i + 1] * t0 ** 3) / (6.0 * hi) + (y[i] / hi - M[i] * hi / 6.0) * t1 \
        + (y[i + 1] / hi - M[i + 1] * hi / 6.0) * t0


def dense_mesh(tau):
    """The uniform mesh of step tau_1 - tau_0 on [0, beta] (the mesh's end point)."""
    tau = np.asarray(tau, float)
    h = tau[1] - tau[0]
    n = int(round(tau[-1] / h))
    return h * np.arange(n + 1)


def g0_tau(eps, t, beta):
    """G0(tau) = -exp(-eps tau) (1 - n_F(eps)), 0 <= tau <= beta (Sec. III.B.1), overflow-free."""
    t = np.asarray(t, float)
    if eps >= 0:
        return -np.exp(-eps * t) / (1.0 + np.exp(-beta * eps))
    return -np.exp(eps * (beta - t)) / (1.0 + np.exp(beta * eps))


def _antiperiodic(f, n):
    """f on the uniform mesh (n + 1 points, f[0] the value at 0+) -> F with F[p - r + n] =
    f(tau_p - tau_r) for -n <= p - r <= n: f(d) for d >= 0, and f(d) = -f(d + beta) below, which
    for d = (i - n) h is -f[i]."""
    return np.concatenate([-np.asarray(f)[:n], f])


def dyson_tau(eps, s, sigc_upm, tau_upm):
    """G(tau) on the dense uniform mesh (and that mesh) for one state, Eqs. (dysongf)-(dysong).

    eps: band energy; s: Sigma^x + Sigma^H - Sigma_0 (static); sigc_upm: Sigma^c on tau_upm
    (tau_upm[0] = 0, tau_upm[-1] = beta, the UPM)."""
    t = dense_mesh(tau_upm)
    beta = t[-1]
    n = len(t) - 1
    h = t[1] - t[0]
    w = np.full(n + 1, h)
    w[0] = w[-1] = 0.5 * h                                   # trapezoid increments
    g0 = g0_tau(eps, t, beta)
    sc = natural_spline(tau_upm, sigc_upm, t)
    G0d = _antiperiodic(g0, n)
    Scd = _antiperiodic(sc, n)
    idx = np.arange(n + 1)
    D = idx[:, None] - idx[None, :] + n                      # position of tau_p - tau_r
    G0m = G0d[D]                                             # G0(tau_p - tau_r)
    Scm = Scd[D]                                             # Sigma^c(tau_p - tau_r)
    Z = G0m * s + (G0m * w[None, :]) @ Scm                   # Eqs. (zxjk), (zcjk)
    K = np.eye(n + 1) - Z * w[None, :]
    return np.linalg.solve(K, g0), t
