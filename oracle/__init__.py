"""FP64 CPU oracle for the Matsubara-time GW hot path (test infrastructure).

This package is the independent reference that the GPU library is checked
against. It is test infrastructure only: the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the GPU library and its
Python binding never do. It shares no code with the library: only the seeded
input generators in ``gwinputs`` serve both sides.

Every function cites the passage of Chu et al., "All-electron self-consistent
GW in the Matsubara-time domain" (arXiv:1602.02313) that it follows.

Parity status per function (what pins it; see tests/test_oracle_*.py):

* green_tau0        -- closed form of the reference G0 (Sec. III.B.1), pinned by
                       boundary values and particle number.
* polarization      -- Eq. (irpol), pinned by the Lindhard closed form of its
                       Matsubara transform, Hermiticity and P(tau) <= 0.
* transforms        -- Lehmann-basis least squares; pinned by exactness on
                       basis functions and by closed-form transforms of G0.
* screen            -- iν form of Eq. (tildeW); pinned by the one-mode secular
                       closed form and the residual of the linear system.
* selfenergy        -- Eq. (sigc) and the product-basis form of Eq. (sigx);
                       pinned by brute-force Matsubara convolution on tiny
                       inputs (Nk = 1, and Nk = 3 with k - q != k and band
                       energies that differ between k and k - q) and the
                       direct occupied-state sum.
* dyson_iw          -- diagonal Dyson (Eqs. dysongf-zcjk) posed in iω; pinned
                       by the zero and static self-energy closed forms.
* pade / cpe / qp   -- analytic continuation (Sec. III.B.6); pinned by exact
                       recovery of few-pole models and causality. qp_solve finds
                       every rising zero near eps on its own mesh centred on eps
                       and refines it by Brent's method; pinned by the closed
                       forms of one- and two-pole self-energies (several zeros,
                       two zeros and a pole within 5 mHa) and the fallback.
* mlp               -- not in the paper; pinned by central finite differences.
* screen_tau        -- the paper's tau-domain form of Eq. (tildeW) on the uniform power
                       mesh (Sec. III.B.3); pinned by closed forms of one-mode and
                       exponential polarizations (second and first order in the step).
* dyson_tau         -- the paper's tau-domain Dyson equation (Eqs. dysongf-dysong) on the
                       spline-densified uniform mesh; pinned by the closed forms of a static
                       shift and of a one-pole Sigma^c (first order), the antiperiodic
                       extension by G0's own definition below zero, and the spline by
                       scipy's natural spline.
* offdiag           -- the full band matrix of Sigma^c and Sigma^x (Eqs. sigc, sigx without
                       the diagonal approximation); pinned by its diagonal (oracle.selfenergy),
                       Hermiticity and covariance under a unitary change of bands. Its matrix
                       Dyson update (dyson_matrix_iw) is pinned by the downfolding closed form
                       of a pole self-energy, its diagonal reduction and unitary covariance.
* symmetry          -- the star sum of Sec. III.C (the self-energy of an irreducible q carried
                       to every member of its star); pinned by the equality of the reduced sum
                       and the full sum over the q mesh on a synthetic Oh crystal.
"""
from .gw import *  # noqa: F401,F403
from .transforms import transform_matrices  # noqa: F401
from . import mlp  # noqa: F401
from . import screen_tau  # noqa: F401
from . import dyson_tau  # noqa: F401
from . import offdiag  # noqa: F401
from . import symmetry  # noqa: F401
from .continuation import (pade_coeffs, pade_eval, cpe_grid, cpe_kernel, cpe_fit,  # noqa: F401
                           cpe_eval, qp_solve, band_gap, pade_resig, cpe_resig, ETA)
