"""Crystal-symmetry reduction of the self-energy sum (Sec. III.C), FP64 (test infrastructure; see
the package docstring).

The contribution of q' = R q to Sigma_n(k) (Eq. sigc, Eq. sigx) equals the contribution of q at
R^-1 k, because M, v and eps transform as the paper states. So with the self-energy T of an
irreducible q alone, its whole star contributes S[k] = sum_r T[R_r^-1 k], one term per distinct
member R_r q of the star.
"""
from __future__ import annotations

import numpy as np


def sigma_star(T, kinv):
    """S[k, ...] = sum_r T[kinv[r, k], ...]: T [nk, ...] the contribution of one irreducible q,
    kinv [nrep, nk] the index of R_r^-1 k for each member of its star."""
    T = np.asarray(T)
    S = np.zeros_like(T)
    for inv in np.asarray(kinv):
        for k in range(T.shape[0]):
            S[k] += T[inv[k]]
    return S
