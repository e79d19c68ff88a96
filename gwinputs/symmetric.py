"""A synthetic crystal with the cubic point group Oh (input generation only, no GW arithmetic).

Stand-in for the paper's use of crystal symmetry (Sec. III.C): 48 operations R (all signed
permutations of the three axes, no fractional translations) act on an n x n x n k mesh
(integer coordinates modulo n) and on a plane-wave product basis per q, {G : |q/n + G|^2 <= cut}
(q taken into (-n/2, n/2]), padded to NI with inert functions (M = 0) so that every q has NI
basis functions. Everything is built to obey the paper's transformation laws exactly:
    eps_b(R k) = eps_b(k),   v_{pi(I)}(R q) = v_I(q),
    M[R q][R k][pi_{R,q}(I)][a][b] = M[q][k][I][a][b],
with pi_{R,q} the basis map G -> R (q/n + G) - (R q)/n. M is drawn per orbit of (q, k) pairs,
averaged over the pair's stabiliser, and copied to the orbit.
"""
from __future__ import annotations

import itertools

import numpy as np


def oh_ops():
    """The 48 signed permutation matrices (integer 3 x 3), identity first."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), np.int64)
            for i in range(3):
                R[i, perm[i]] = signs[i]
            out.append(R)
    out.sort(key=lambda R: (not np.array_equal(R, np.eye(3, dtype=np.int64)),))
    return out


def _wrap(v, n):
    """Integer mesh vector -> its representative in (-n/2, n/2]."""
    return (np.asarray(v) + n // 2 - 1) % n - n // 2 + 1


def _basis(qw, n, cut):
    """Integer G with |qw/n + G|^2 <= cut, sorted by (norm, G)."""
    r = int(np.ceil(np.sqrt(cut))) + 1
    g = np.array(list(itertools.product(range(-r, r + 1), repeat=3)), np.int64)
    x = qw[None, :] / n + g
    nn = np.einsum("ij,ij->i", x, x)
    keep = nn <= cut + 1e-12
    g, nn = g[keep], nn[keep]
    order = sorted(range(len(g)), key=lambda i: (round(nn[i], 12), tuple(g[i])))
    return g[order], nn[order]


class SymmetricCrystal:
    """Fields: n, nk, nq (= nk, every mesh vector), nb, nocc, ni, beta, eps [nk][nb],
    v [nq][ni], kmq [nq][nk], M [nq][nk][ni][nb][nb] (complex), ops (48 matrices),
    kimg [48][nk] (index of R k), qimg [48][nq], ibz (representative q of each star, ascending),
    reps {q_ibz: [op indices mapping it to each distinct member of its star]}."""


def make_symmetric_crystal(n=2, nb=4, nocc=2, cut=1.6, beta=50.0, seed=5, ni=None):
    ops = oh_ops()
    nk = n ** 3
    kv = np.array(np.unravel_index(np.arange(nk), (n, n, n))).T          # [nk][3]
    kid = lambda v: int(np.ravel_multi_index(tuple(np.asarray(v) % n), (n, n, n)))  # noqa: E731
    kimg = np.array([[kid(R @ kv[k]) for k in range(nk)] for R in ops], np.int32)
    bases = [_basis(_wrap(kv[q], n), n, cut) for q in range(nk)]
    nmax = max(len(b[0]) for b in bases)
    ni = ni or 32 * ((nmax + 31) // 32)
    assert ni >= nmax
    # basis map pi[R][q][I] (index in the basis of R q); inert functions map in order
    pi = np.zeros((len(ops), nk, ni), np.int64)
    for r, R in enumerate(ops):
        for q in range(nk):
            qw, qr = _wrap(kv[q], n), kimg[r, q]
            gq, gr = bases[q][0], bases[qr][0]
            look = {tuple(g): i for i, g in enumerate(gr)}
            for i, g in enumerate(gq):
                x = R @ (qw + n * g) - _wrap(kv[qr], n)                 # n (R (q/n + G) - q'/n)
                assert np.all(x % n == 0)
                pi[r, q, i] = look[tuple(x // n)]
            pi[r, q, len(gq):] = np.arange(len(gq), ni)
    v = np.ones((nk, ni))
    for q in range(nk):
        v[q, :len(bases[q][1])] = 4.0 * np.pi / (0.05 + (2.0 * np.pi) ** 2 * bases[q][1])
    rng = np.random.default_rng(seed)
    base = np.concatenate([np.linspace(-1.0, -0.3, nocc), np.linspace(0.3, 1.0, nb - nocc)])
    hop = rng.uniform(-0.02, 0.02, nb)
    disp = np.cos(2.0 * np.pi * kv / n).sum(1)                           # invariant under Oh
    eps = base[None, :] + disp[:, None] * hop[None, :]
    kmq = np.array([[kid(kv[k] - kv[q]) for k in range(nk)] for q in range(nk)], np.int32)
    return _fill(ops, kimg, pi, bases, v, eps, kmq, n, nk, nb, nocc, ni, beta, rng)


def _fill(ops, kimg, pi, bases, v, eps, kmq, n, nk, nb, nocc, ni, beta, rng):
    nop = len(ops)
    M = np.zeros((nk, nk, ni, nb, nb), complex)
    done = np.zeros((nk, nk), bool)
    scale = np.sqrt(0.5 / nb)
    for q in range(nk):
        nq_basis = len(bases[q][0])
        for k in range(nk):
            if done[q, k]:
                continue
            m0 = np.zeros((ni, nb, nb), complex)
            m0[:nq_basis] = scale * (rng.standard_normal((nq_basis, nb, nb))
                                     + 1j * rng.standard_normal((nq_basis, nb, nb)))
            stab = [r for r in range(nop) if kimg[r, q] == q and kimg[r, k] == k]
            # average over the stabiliser: M[q][k][pi_S(I)] = M[q][k][I] for S in it
            ms = np.zeros_like(m0)
            for r in stab:
                ms[pi[r, q]] += m0
            ms /= len(stab)
            for r in range(nop):
                qr, kr = kimg[r, q], kimg[r, k]
                if not done[qr, kr]:
                    M[qr, kr][pi[r, q]] = ms
                    done[qr, kr] = True
    ibz, reps = [], {}
    seen = set()
    for q in range(nk):
        if q in seen:
            continue
        ibz.append(q)
        reps[q] = []
        for r in range(nop):
            if kimg[r, q] not in seen:
                seen.add(int(kimg[r, q]))
                reps[q].append(r)
    c = SymmetricCrystal()
    c.n, c.nk, c.nq, c.nb, c.nocc, c.ni, c.beta = n, nk, nk, nb, nocc, ni, float(beta)
    c.eps, c.v, c.kmq, c.M, c.ops, c.kimg, c.qimg = eps, v, kmq, M, ops, kimg, kimg
    c.ibz, c.reps, c.pi = ibz, reps, pi
    c.seed = 0
    return c


def restrict_q(c, qs):
    """The crystal seen by a context that holds only the q points qs (e.g. the irreducible
    ones): v, k - q rows and M of those q; seed 0 (M is passed explicitly)."""
    import copy
    r = copy.copy(c)
    qs = list(qs)
    r.nq = len(qs)
    r.v = np.ascontiguousarray(c.v[qs])
    r.kmq = np.ascontiguousarray(c.kmq[qs])
    r.M = np.ascontiguousarray(c.M[qs])
    r.qlist = qs
    return r


def star_kinv(c, q):
    """For each member R q of q's star (c.reps[q]): the index of R^-1 k for every k, [nrep][nk]."""
    out = []
    for r in c.reps[q]:
        inv = np.empty(c.nk, np.int32)
        inv[c.kimg[r]] = np.arange(c.nk, dtype=np.int32)
        out.append(inv)
    return np.array(out, np.int32)
