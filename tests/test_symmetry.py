"""Crystal-symmetry reduction (Sec. III.C) on a synthetic Oh crystal: the generator obeys the
paper's transformation laws, and the self-energy from the irreducible q points alone, each
q's contribution carried to the members of its star by k -> R^-1 k, equals the sum over all q
(the rearranged Eq. sigc), with the oracle throughout."""
import numpy as np

import gwinputs as gi
import oracle as orc
from gwinputs import symmetric as sy


def kinv_maps(c, q):
    """For each op of q's star: index of R^-1 k for every k."""
    out = []
    for r in c.reps[q]:
        inv = np.empty(c.nk, np.int32)
        inv[c.kimg[r]] = np.arange(c.nk)
        out.append(inv)
    return np.array(out)


def test_symmetric_crystal_obeys_the_laws():
    c = sy.make_symmetric_crystal(n=2, nb=4, nocc=2)
    assert sum(len(r) for r in c.reps.values()) == c.nq          # the stars tile the q mesh
    for r in range(len(c.ops)):
        for q in range(c.nk):
            qr = c.kimg[r, q]
            assert np.array_equal(c.v[qr][c.pi[r, q]], c.v[q])
            assert np.array_equal(c.kmq[qr][c.kimg[r]], c.kimg[r][c.kmq[q]])
            for k in range(c.nk):
                # equal up to the rounding of the stabiliser average
                assert np.allclose(c.M[qr, c.kimg[r, k]][c.pi[r, q]], c.M[q, k], rtol=0, atol=1e-15)
        assert np.allclose(c.eps[c.kimg[r]], c.eps, rtol=0, atol=1e-15)


def test_sigma_from_irreducible_q_equals_full_sum():
    c = sy.make_symmetric_crystal(n=2, nb=4, nocc=2, beta=50.0)
    gr = gi.make_grid(c.beta, 16, 16, 16, ncont=16)
    G, occ = orc.green_tau0(c.eps, gr.tau, gr.beta)
    contrib = {}
    for q in range(c.nq):
        P = orc.polarization(c.M[q], G, c.kmq[q], omega=2.0)
        # P of R q is P of q with rows and columns mapped (Sec. III.C)
        if q in c.reps:
            for r in c.reps[q]:
                qr = c.kimg[r, q]
                Pr = orc.polarization(c.M[qr], G, c.kmq[qr], omega=2.0)
                assert np.allclose(Pr[:, c.pi[r, q]][:, :, c.pi[r, q]], P, rtol=0, atol=1e-13 * np.abs(P).max())
        Wt = orc.nu_to_tau(orc.screen(orc.tau_to_nu(P, gr), c.v[q]), gr)
        sc, sx, _ = orc.selfenergy(c.M[q], G, Wt, c.v[q], c.kmq[q], occ, omega=2.0)
        contrib[q] = (sc, sx)
    full_c = sum(contrib[q][0] for q in range(c.nq))
    full_x = sum(contrib[q][1] for q in range(c.nq))
    red_c, red_x = np.zeros_like(full_c), np.zeros_like(full_x)
    for q in c.ibz:
        red_c += orc.symmetry.sigma_star(contrib[q][0], kinv_maps(c, q))
        red_x += orc.symmetry.sigma_star(contrib[q][1], kinv_maps(c, q))
    assert np.abs(red_c - full_c).max() < 1e-12 * np.abs(full_c).max()
    assert np.abs(red_x - full_x).max() < 1e-12 * np.abs(full_x).max()
    assert len(c.ibz) == 4 and c.nq == 8


def test_oh_stars_on_the_4x4x4_mesh():
    """Oh on the 4 x 4 x 4 mesh: 10 irreducible q whose stars (sizes 1, 1, 3, 3, 6, 6, 8, 12, 12,
    12, each dividing 48) tile all 64 q."""
    c = sy.make_symmetric_crystal(n=4, nb=4, nocc=2, cut=1.2)
    sizes = [len(c.reps[q]) for q in c.ibz]
    assert len(c.ibz) == 10 and sum(sizes) == 64
    assert all(48 % s == 0 for s in sizes)
    assert sorted(sizes) == [1, 1, 3, 3, 6, 6, 8, 12, 12, 12]
