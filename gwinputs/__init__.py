"""Seeded synthetic inputs for the Matsubara-time GW hot path.

This module is shared by the FP64 CPU oracle and by the GPU library's tests
and benchmark. It holds only input generation -- random numbers, synthetic
crystals and the discretisation grid -- and none of the GW arithmetic
(no Green's function, polarization, screening, self-energy or transform).

Synthetic crystal (stand-in for the paper's FP-LAPW crystals, which are not
available; the paper's workloads are 4x4x4 k-meshes with >=150 empty bands,
Sec. "Computational Details"):

* band energies eps[k, b]: eigenvalues of a seeded complex Gaussian Hermitian
  H_k (Nb x Nb), mapped per k affinely so that the lowest Nocc land on
  [-1, -0.05] Ha and the rest on [0.05, 1] Ha (0.1 Ha gap at mu = 0; the
  paper measures energies from mu, Sec. "Green's function in the reference
  K-S system").
* Coulomb diagonal v[q, I] = 4 pi / (0.05 + g^2), g ~ U[0, 3]
  (diagonal like the paper's v_GG'(q) = 4 pi delta_GG' / |q+G|^2).
* plane-wave matrix elements M^I_ab(k, q) (paper Eq. mmatrix) replaced by
  complex Gaussian numbers with E|M|^2 = 1/Nb, drawn from Philox4x32-10
  (Salmon, Moraes, Dror, Shaw, SC'11) keyed by the seed, with the flat index
  of (q, k, I, a, b) as counter, then Box-Muller in FP32 with the logarithm,
  sine and cosine evaluated by a fixed sequence of round-to-nearest FP32
  operations (series written out here). The GPU library implements the same
  generator on its own; the matrix elements are bitwise equal.

Grid (discretisation input, passed explicitly to both sides):

* tau nodes: Gauss-Legendre nodes in s = ln(tau) on [ln tau_min, ln(beta/2)],
  mirrored to beta - tau, so the set is closed under tau -> beta - tau.
* real-frequency poles E_l of the fermionic Lehmann kernel
  K(tau, E) = exp(-E tau) / (1 + exp(-beta E)), chosen by column-pivoted QR
  over a fine pole set (the discrete Lehmann representation of Kaye, Chen and
  Parcollet, 2022).
* bosonic / fermionic Matsubara index sets chosen by pivoted QR over the
  Lehmann kernel's Matsubara transforms; plus the dense first-N fermionic set
  used for analytic continuation (the paper uses 128, Sec. "Computational
  Details").
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as _sl

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11): multipliers and Weyl key increments.
# ---------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# Stream tags used in counter word 2, so that different synthetic tensors
# never share Philox counters.
STREAM_M = 0x4D  # plane-wave matrix elements


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on numpy arrays of 32-bit values.

    Each round multiplies counter words 0 and 2 by the two Philox constants,
    xors the high halves with words 1/3 and the key, and the key is bumped by
    the Weyl constants between rounds. Returns four uint64 arrays holding
    32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK32
        hi1, lo1 = p1 >> _S32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        k0 = (k0 + PHILOX_W0) & _MASK32
        k1 = (k1 + PHILOX_W1) & _MASK32
    return c0, c1, c2, c3


# ---------------------------------------------------------------------------
# Box-Muller in FP32 with a fixed sequence of round-to-nearest operations.
# The logarithm and the sine / cosine are not library calls but the evaluations below: only
# IEEE-754 round-to-nearest FP32 additions, multiplications, one division and one square root,
# in a fixed order, so that the GPU generator (which performs the same operations with
# explicitly rounded intrinsics) produces bit-identical matrix elements.
#   ln u: u = 2^e m with m in [sqrt(1/2), sqrt(2)) (exact), ln m = 2 atanh(s), s = (m - 1)/(m + 1),
#         by the odd series 2 (s + s^3/3 + ... + s^11/11) (|s| <= 0.172, truncation < 2e-9);
#         ln u = e ln 2 + ln m.
#   cos / sin (2 pi u): t = 4 u splits exactly into the quadrant o and f in [0, 1); x = (pi/2) f;
#         Taylor series of sin x to x^13 and of cos x to x^12 (truncation < 1e-8 on [0, pi/2]);
#         the quadrant by exact sign and order changes.
# The series coefficients are 1/k and 1/k! rounded to FP32.
# ---------------------------------------------------------------------------
_F = np.float32
_LN2 = _F(0.6931471805599453)
_HALF_PI = _F(1.5707963267948966)
_SQRT_HALF = _F(0.7071067811865476)
_ATANH_C = [_F(1.0 / k) for k in (11, 9, 7, 5, 3)]                       # s^11 .. s^3 terms
_SIN_C = [_F((-1.0) ** (k // 2) / math.factorial(k)) for k in (13, 11, 9, 7, 5, 3)]
_COS_C = [_F((-1.0) ** (k // 2) / math.factorial(k)) for k in (12, 10, 8, 6, 4, 2)]


def log_f32(u):
    """ln u for float32 u in (0, 1], by the fixed evaluation described above."""
    u = np.asarray(u, np.float32)
    m, e = np.frexp(u)                        # u = m 2^e, m in [0.5, 1)
    low = m < _SQRT_HALF
    m = np.where(low, m * _F(2.0), m)
    e = np.where(low, e - 1, e).astype(np.float32)
    f = m - _F(1.0)                           # exact (Sterbenz)
    s = f / (_F(2.0) + f)
    z = s * s
    p = z * _ATANH_C[0] + _ATANH_C[1]
    for c in _ATANH_C[2:]:
        p = p * z + c
    p = p * z                                 # s^2 / 3 + s^4 / 5 + ...
    s2 = s + s
    lm = s2 + s2 * p
    return e * _LN2 + lm


def sincos_turn_f32(u):
    """(cos 2 pi u, sin 2 pi u) for float32 u in [0, 1), by the fixed evaluation described above."""
    u = np.asarray(u, np.float32)
    t = u * _F(4.0)
    o = np.floor(t)
    f = t - o
    o = o.astype(np.int64)
    x = f * _HALF_PI
    x2 = x * x
    q = x2 * _SIN_C[0] + _SIN_C[1]
    for c in _SIN_C[2:]:
        q = q * x2 + c
    q = q * x2
    sn = x + x * q
    r = x2 * _COS_C[0] + _COS_C[1]
    for c in _COS_C[2:]:
        r = r * x2 + c
    r = r * x2
    cs = _F(1.0) + r
    c_out = np.select([o == 0, o == 1, o == 2], [cs, -sn, -cs], sn)
    s_out = np.select([o == 0, o == 1, o == 2], [sn, cs, -sn], -cs)
    return c_out.astype(np.float32), s_out.astype(np.float32)


def m_flat_index(q, k, I, a, b, nk, ni, nb):
    """Flat Philox counter of element M^I_ab(k, q): ((((q*nk + k)*ni + I)*nb + a)*nb + b)."""
    return ((((np.uint64(q) * np.uint64(nk) + np.uint64(k)) * np.uint64(ni)
              + np.asarray(I, np.uint64)) * np.uint64(nb) + np.asarray(a, np.uint64))
            * np.uint64(nb) + np.asarray(b, np.uint64))


def m_values_from_index(idx, seed, nb):
    """Complex Gaussian M values for flat indices idx (uint64 array).

    counter = (idx mod 2^32, idx div 2^32, STREAM_M, 0), key = (seed lo, seed hi);
    24-bit uniforms u1 = (x0 >> 8) + 1) 2^-24 in (0, 1] and u2 = (x1 >> 8) 2^-24 in [0, 1) from the
    first two output words; Box-Muller in FP32: r = sqrt(-2 ln u1), (c, s) = (cos, sin)(2 pi u2)
    (log_f32, sincos_turn_f32), re = r c and im = r s rounded to FP32; M = (re + i im) sqrt(1/(2 nb))
    with the last product in FP64. E|M|^2 = 1/nb.
    """
    idx = np.asarray(idx, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(idx & _MASK32, idx >> _S32,
                                 np.full(idx.shape, STREAM_M, np.uint64),
                                 np.zeros(idx.shape, np.uint64),
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = ((x0 >> np.uint64(8)).astype(np.float32) + _F(1.0)) * _F(2.0 ** -24)
    u2 = (x1 >> np.uint64(8)).astype(np.float32) * _F(2.0 ** -24)
    w = log_f32(u1) * _F(-2.0)
    r = np.sqrt(w)
    c, s = sincos_turn_f32(u2)
    re = (r * c).astype(np.float64)
    im = (r * s).astype(np.float64)
    sc = math.sqrt(0.5 / nb)
    return re * sc + 1j * (im * sc)


def m_block(seed, q, k, nk, ni, nb):
    """M^I_ab(k, q) for all I, a, b as a complex array [ni, nb, nb].

    Index convention: a is a band at k - q, b a band at k (paper Eq. irpol
    relabelled k -> k - q, so that the same tensor serves Eq. sigc).
    """
    I, a, b = np.meshgrid(np.arange(ni), np.arange(nb), np.arange(nb), indexing="ij")
    idx = m_flat_index(q, k, I, a, b, nk, ni, nb)
    return m_values_from_index(idx, seed, nb)


# ---------------------------------------------------------------------------
# Synthetic crystal
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Crystal:
    seed: int
    nk: int
    nq: int
    nb: int
    nocc: int
    ni: int
    beta: float
    eps: np.ndarray        # [nk, nb] float64, Ha, relative to mu = 0, ascending per k
    v: np.ndarray          # [nq, ni] float64
    kmq: np.ndarray        # [nq, nk] int32: index of k - q on the k grid
    qidx: np.ndarray       # [nq] int32: which grid vector each q is
    mesh: tuple            # (n1, n2, n3) k mesh

    @property
    def mseed(self):
        return self.seed


def kmesh_shape(nk):
    n = round(nk ** (1.0 / 3.0))
    if n ** 3 == nk:
        return (n, n, n)
    return (nk, 1, 1)


def kminusq_table(mesh, qlist):
    """k - q on a periodic mesh: k = (i1, i2, i3) flattened row-major."""
    n1, n2, n3 = mesh
    nk = n1 * n2 * n3
    ks = np.array(np.unravel_index(np.arange(nk), mesh)).T
    out = np.zeros((len(qlist), nk), np.int32)
    for iq, q in enumerate(qlist):
        qv = np.array(np.unravel_index(q, mesh))
        d = (ks - qv[None, :]) % np.array(mesh)[None, :]
        out[iq] = np.ravel_multi_index(d.T, mesh)
    return out


def make_crystal(seed, nk, nb, nocc, ni, beta, nq=None, qlist=None):
    """Seeded synthetic crystal; eps from seeded Hermitian H_k (see module doc)."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    mesh = kmesh_shape(nk)
    eps = np.zeros((nk, nb))
    for k in range(nk):
        x = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
        h = 0.5 * (x + x.conj().T)
        lam = np.linalg.eigvalsh(h)
        lo, hi = lam[:nocc], lam[nocc:]
        e = np.empty(nb)
        if nocc > 1:
            e[:nocc] = -1.0 + (lo - lo[0]) * (0.95 / (lo[-1] - lo[0]))
        else:
            e[:nocc] = -0.05
        if nb - nocc > 1:
            e[nocc:] = 0.05 + (hi - hi[0]) * (0.95 / (hi[-1] - hi[0]))
        else:
            e[nocc:] = 0.05
        eps[k] = e
    if qlist is None:
        qlist = list(range(nk if nq is None else nq))
    qlist = [int(q) % nk for q in qlist]
    nq = len(qlist)
    g = rng.uniform(0.0, 3.0, size=(nq, ni))
    v = 4.0 * np.pi / (0.05 + g * g)
    return Crystal(seed=seed, nk=nk, nq=nq, nb=nb, nocc=nocc, ni=ni, beta=float(beta),
                   eps=eps, v=v, kmq=kminusq_table(mesh, qlist),
                   qidx=np.array(qlist, np.int32), mesh=mesh)


def subset_q(cr: Crystal, start: int, count: int) -> Crystal:
    """The q points start .. start+count-1 of a crystal (same eps, v rows and k - q rows);
    the matrix-element counter of q stays its global position, passed as q0."""
    return dataclasses.replace(cr, nq=count, v=cr.v[start:start + count].copy(),
                               kmq=cr.kmq[start:start + count].copy(), qidx=cr.qidx[start:start + count].copy())


def m_for_q(cr: Crystal, iq: int, ks=None):
    """M^I_ab(k, q) for the iq-th q and the listed k: complex [len(ks), ni, nb, nb].

    The counter uses the position iq of q in the crystal's q list.
    """
    if ks is None:
        ks = range(cr.nk)
    return np.stack([m_block(cr.seed, iq, k, cr.nk, cr.ni, cr.nb) for k in ks])


# ---------------------------------------------------------------------------
# Grid
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Grid:
    beta: float
    tau: np.ndarray      # [ntau] ascending, closed under beta - tau
    wtau: np.ndarray     # [ntau] quadrature weights (sum ~ beta - 2 tau_min)
    poles: np.ndarray    # [npole] real frequencies of the Lehmann basis
    nu_idx: np.ndarray   # [nnu] bosonic Matsubara indices n >= 0 (nu_n = 2 n pi / beta)
    w_idx: np.ndarray    # [nw] fermionic Matsubara indices n >= 0 (w_n = (2n+1) pi / beta)
    ncont: int           # dense fermionic set n = 0 .. ncont-1 for continuation

    @property
    def ntau(self):
        return len(self.tau)

    @property
    def nnu(self):
        return len(self.nu_idx)

    @property
    def nw(self):
        return len(self.w_idx)

    @property
    def npole(self):
        return len(self.poles)


def tau_grid_gl_log(beta, ntau, tau_min=1e-3):
    """Gauss-Legendre nodes in ln(tau) on [tau_min, beta/2], mirrored to beta - tau."""
    assert ntau % 2 == 0
    h = ntau // 2
    x, w = np.polynomial.legendre.leggauss(h)
    a, b = math.log(tau_min), math.log(beta / 2.0)
    s = 0.5 * (b - a) * x + 0.5 * (b + a)
    ws = 0.5 * (b - a) * w
    t = np.exp(s)
    wt = ws * t
    tau = np.concatenate([t, beta - t[::-1]])
    wtau = np.concatenate([wt, wt[::-1]])
    return tau, wtau


def _kernel_f(tau, E, beta):
    """Fermionic Lehmann kernel exp(-E tau)/(1+exp(-beta E)), overflow-free (grid selection only)."""
    tau = np.asarray(tau, float)[:, None]
    E = np.asarray(E, float)[None, :]
    a = np.abs(E)
    den = 1.0 + np.exp(-beta * a)
    return np.where(E >= 0, np.exp(-a * tau), np.exp(-a * (beta - tau))) / den


def select_poles(tau, beta, lam, tol=1e-10, nfine=1500, emin=1e-6):
    """Column-pivoted QR of K(tau_i, E) over a fine log grid of +-E and 0; keep
    pivots with |R_jj| > tol |R_00| (at most len(tau))."""
    ef = np.geomspace(emin, lam, nfine)
    efine = np.concatenate([-ef[::-1], [0.0], ef])
    K = _kernel_f(tau, efine, beta)
    _, R, piv = _sl.qr(K, pivoting=True, mode="economic")
    d = np.abs(np.diag(R))
    r = int(np.sum(d > tol * d[0]))
    return np.sort(efine[piv[:r]])


def select_matsubara(poles, beta, nsel, fermionic, nmax):
    """Pivoted QR over n = 0..nmax of the Lehmann kernel's Matsubara transform
    columns; returns the first nsel pivots, sorted."""
    n = np.arange(nmax + 1)
    z = 1j * ((2 * n + 1) if fermionic else (2 * n)) * np.pi / beta
    E = np.asarray(poles)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        if fermionic:
            Kh = -1.0 / (z[:, None] - E)
        else:
            Kh = -np.tanh(0.5 * beta * E) / (z[:, None] - E)
            Kh = np.where((n[:, None] == 0) & (E == 0), 0.5 * beta, Kh)
    _, _, piv = _sl.qr(Kh.T, pivoting=True, mode="economic")
    nsel = min(nsel, len(piv))
    return np.sort(n[piv[:nsel]]).astype(np.int32)


def make_grid(beta, ntau, nnu, nw, ncont=128, tau_min=1e-3, lam=None, tol=1e-10):
    tau, wtau = tau_grid_gl_log(beta, ntau, tau_min)
    if lam is None:
        lam = 1.0 / tau_min
    poles = select_poles(tau, beta, lam, tol)
    nmax = int(math.ceil(2.0 * beta * lam / (2.0 * math.pi)))
    nu_idx = select_matsubara(poles, beta, nnu, False, nmax)
    w_idx = select_matsubara(poles, beta, nw, True, nmax)
    return Grid(beta=float(beta), tau=tau, wtau=wtau, poles=poles, nu_idx=nu_idx,
                w_idx=w_idx, ncont=int(ncont))


# ---------------------------------------------------------------------------
# Uniform power mesh (tau-domain screening, Sec. III.A / III.B.3)
# ---------------------------------------------------------------------------
def upm_grid(beta, p, m):
    """Uniform power mesh UPM(p, m) on [0, beta] (Sec. III.A, after Ku-Eguiluz and Stan et al.),
    2 p m + 1 points including 0 and beta. Reading of the paper's description: on [0, beta/2]
    the sub-interval ends are 0 and (beta/2) 2^(k - p), k = 1..p (widths beta 2^-p, beta 2^-p,
    beta 2^(1-p), ..., beta/4), each divided into m equal steps; the mesh is mirrored by
    tau -> beta - tau, so it is densest at both ends."""
    ends = [0.0] + [0.5 * beta * 2.0 ** (k - p) for k in range(1, p + 1)]
    half = []
    for a, b in zip(ends[:-1], ends[1:]):
        half.extend(a + (b - a) * np.arange(m) / m)
    half = np.array(half + [0.5 * beta])
    return np.concatenate([half, beta - half[-2::-1]])


def tau_pairs(tau, beta, rtol=1e-11):
    """The distinct differences d = (tau_p - tau_r) mod beta in [0, beta) of a mesh and, for every
    pair, the index of its difference: returns (d [ndiff], idx int [npts][npts]). Differences of
    0 and +-beta are all d = 0 (bosonic periodicity). Values equal up to rounding share one index."""
    tau = np.asarray(tau, float)
    d = tau[:, None] - tau[None, :]
    d = np.where(d < 0.0, d + beta, d)
    d = np.where(d >= beta * (1.0 - rtol), d - beta, d)
    d = np.where(np.abs(d) < beta * rtol, 0.0, d)
    key = np.round(d / (beta * rtol)).astype(np.int64)
    _, first, inv = np.unique(key.ravel(), return_index=True, return_inverse=True)
    return d.ravel()[first], inv.reshape(d.shape).astype(np.int32)


# Unit-cell volume Omega of 1/(Omega N_k) (Eqs. irpol, sigc): the paper's silicon cell,
# a = 5.43 Angstrom (Sec. IV), primitive fcc volume a^3 / 4 in bohr^3.
OMEGA_SI = (5.43 / 0.529177210903) ** 3 / 4.0

# ---------------------------------------------------------------------------
# Workload configurations (synthetic stand-ins for the paper's crystals)
# ---------------------------------------------------------------------------
CONFIGS = {
    # one q, Nk=8, Nb=16 (8 occ), NI=64, Ntau=16, beta=100
    "nk8_nb16": dict(seed=1001, nk=8, nb=16, nocc=8, ni=64, beta=100.0, ntau=16, nnu=16, nw=16,
               qlist=[1]),
    # Nk=64 (4x4x4), q on the same grid, Nb=64 (32 occ), NI=256, Ntau=48, beta=200
    "nk64_nb64": dict(seed=2001, nk=64, nb=64, nocc=32, ni=256, beta=200.0, ntau=48, nnu=48, nw=48,
               qlist=None),
    # Nk=216 (6x6x6), Nb=128 (48 occ), NI=512, Ntau=64, beta=400
    "nk216_nb128": dict(seed=3001, nk=216, nb=128, nocc=48, ni=512, beta=400.0, ntau=64, nnu=64, nw=64,
               qlist=None),
}


def make_config(name, **over):
    c = dict(CONFIGS[name])
    c.update(over)
    cr = make_crystal(c["seed"], c["nk"], c["nb"], c["nocc"], c["ni"], c["beta"],
                      qlist=c["qlist"] if c["qlist"] is not None else list(range(c["nk"])))
    gr = make_grid(c["beta"], c["ntau"], c["nnu"], c["nw"], ncont=c.get("ncont", 128))
    return cr, gr


def batch_crystals(n=12, seed=4000, nb_choices=(32, 64, 96, 128), nk_choices=(8, 27), ntau_choices=(32, 48, 64),
                   beta_range=(100.0, 500.0), nb_max_at_nk27=64):
    """A seeded batch of heterogeneous synthetic crystals (the batched-launch workload): per
    crystal, Nb from nb_choices, NI = 4 Nb, Nb / 2 occupied, Nk from nk_choices (the larger
    k-mesh only up to Nb = nb_max_at_nk27, which bounds the M tensors to a few tens of GB in
    total), q on the k grid, Ntau = Nnu = Nw from ntau_choices, beta uniform in beta_range.
    Crystal i has seed `seed + 1 + i`. Returns a list of (Crystal, Grid)."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    out = []
    for i in range(n):
        nb = int(rng.choice(nb_choices))
        nks = [k for k in nk_choices if k == min(nk_choices) or nb <= nb_max_at_nk27]
        nk = int(rng.choice(nks))
        ntau = int(rng.choice(ntau_choices))
        beta = float(np.round(rng.uniform(*beta_range), 1))
        cr = make_crystal(seed + 1 + i, nk, nb, nb // 2, 4 * nb, beta, qlist=list(range(nk)))
        gr = make_grid(beta, ntau, ntau, ntau, ncont=128)
        out.append((cr, gr))
    return out
