"""Pins of the shared seeded input generators (no GW arithmetic here)."""
import os

import numpy as np
import pytest

import gwinputs as gi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_known_answers(row):
    c, k, want = row[:4], row[4:6], row[6:]
    out = gi.philox4x32_10(*[np.array([x], np.uint64) for x in c], *k)
    assert [int(o[0]) for o in out] == want


def test_m_statistics_and_determinism():
    M = gi.m_block(1234, 0, 0, 1, 64, 16)
    assert M.shape == (64, 16, 16)
    # E|M|^2 = 1/Nb, real and imaginary parts each N(0, 1/(2 Nb))
    assert abs(np.mean(np.abs(M) ** 2) * 16 - 1.0) < 0.05
    assert abs(np.mean(M.real)) < 0.02 and abs(np.mean(M.imag)) < 0.02
    assert np.array_equal(M, gi.m_block(1234, 0, 0, 1, 64, 16))
    assert not np.array_equal(M, gi.m_block(1235, 0, 0, 1, 64, 16))


def test_generator_elementary_functions():
    """The generator's own FP32 logarithm and turn sine / cosine are the functions they stand for:
    within a few FP32 ulps of the FP64 library values over the 24-bit uniform grid."""
    u = ((np.arange(1, 2 ** 24 + 1, 499, dtype=np.float64)) * 2.0 ** -24).astype(np.float32)
    ref = np.log(u.astype(np.float64))
    assert np.abs(gi.log_f32(u) - ref).max() < 4 * 2.0 ** -24 * (1.0 + np.abs(ref)).max()
    v = (np.arange(0, 2 ** 24, 487, dtype=np.float64) * 2.0 ** -24).astype(np.float32)
    c, s = gi.sincos_turn_f32(v)
    th = 2.0 * np.pi * v.astype(np.float64)
    assert np.abs(c - np.cos(th)).max() < 3e-7 and np.abs(s - np.sin(th)).max() < 3e-7
    assert np.abs(c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1.0).max() < 3e-7
    # the exact points: ln 1 = 0, and the quarter turns
    assert gi.log_f32(np.float32(1.0)) == 0.0
    c4, s4 = gi.sincos_turn_f32(np.array([0.0, 0.25, 0.5, 0.75], np.float32))
    assert np.array_equal(c4, [1, 0, -1, 0]) and np.array_equal(s4, [0, 1, 0, -1])


def test_crystal_spectrum():
    cr = gi.make_crystal(7, 8, 16, 8, 64, 100.0)
    assert np.allclose(cr.eps[:, 0], -1.0) and np.allclose(cr.eps[:, -1], 1.0)
    assert np.allclose(cr.eps[:, 7], -0.05) and np.allclose(cr.eps[:, 8], 0.05)
    assert np.all(np.diff(cr.eps, axis=1) >= 0)
    assert cr.v.min() > 4 * np.pi / 9.05 - 1e-12 and cr.v.max() < 4 * np.pi / 0.05
    # k - q table is a permutation for every q, and k - 0 = k
    assert all(sorted(r) == list(range(8)) for r in cr.kmq)
    assert np.array_equal(cr.kmq[0], np.arange(8))


def test_grid_structure():
    g = gi.make_grid(200.0, 48, 48, 48)
    assert np.allclose(g.tau + g.tau[::-1], g.beta)        # closed under beta - tau
    assert np.all(np.diff(g.tau) > 0) and g.tau[0] > 0
    # 24-point GL-in-log weights integrate 1 over [tau_min, beta - tau_min]
    assert abs(g.wtau.sum() - (g.beta - 2e-3)) < 1e-9
    assert len(set(g.nu_idx.tolist())) == len(g.nu_idx) and g.nu_idx.min() >= 0
    assert 1 <= g.npole <= g.ntau


def test_batch_crystals_respect_the_caps_and_are_reproducible():
    import gwinputs as gi
    a = gi.batch_crystals(n=5, seed=4200, nb_choices=(16, 32, 64), nk_choices=(8, 27), ntau_choices=(16, 24),
                          nb_max_at_nk27=16)
    b = gi.batch_crystals(n=5, seed=4200, nb_choices=(16, 32, 64), nk_choices=(8, 27), ntau_choices=(16, 24),
                          nb_max_at_nk27=16)
    for (cr, gr), (cr2, gr2) in zip(a, b):
        assert cr.nb in (16, 32, 64) and cr.ni == 4 * cr.nb and cr.nocc == cr.nb // 2
        assert cr.nk in (8, 27) and (cr.nk == 8 or cr.nb <= 16)
        assert cr.nq == cr.nk and len(gr.tau) in (16, 24) and 100.0 <= gr.beta <= 500.0
        assert (cr.eps == cr2.eps).all() and (cr.v == cr2.v).all() and gr.beta == gr2.beta
    assert len({cr.seed for cr, _ in a}) == 5
