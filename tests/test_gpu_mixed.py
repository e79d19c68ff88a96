"""Tensor-core (tcgen05, fp16 hi/lo split, FP32 TMEM accumulation) contractions
against the FP64 oracle and the FP64 GPU path, called through the C ABI.

Error bars of the split-precision path: each operand carries 22 significant
bits (two fp16 slices); the accumulation runs in FP32 in tensor memory over
K segments and is summed across segments with float-float (two-sum) accumulators. The expected max-norm
relative error is therefore ~sqrt(n_acc) * 2^-24 with n_acc the number of
FP32 accumulation steps per output (a few 1e-6 at the bench sizes); the
tolerances below are set from that bound.
"""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

pytestmark = pytest.mark.gpu

TOL_P = 2e-5
TOL_S = 2e-5
TOL_SX_FF = 1e-11  # float-float exchange sum: ~2^-44 per term, 256-term positive sums


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def zeros(shape, dtype="f8"):
    import torch
    return torch.zeros(shape, dtype={"f8": torch.float64, "c16": torch.complex128, "i4": torch.int32}[dtype],
                       device="cuda")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cases():
    yield "nk8_nb16", gi.make_config("nk8_nb16")
    yield "ragged", (gi.make_crystal(77, 3, 5, 2, 32, 30.0, qlist=[1, 2]), gi.make_grid(30.0, 8, 8, 8, ncont=24))
    yield "ni160", (gi.make_crystal(78, 8, 12, 5, 160, 50.0, qlist=[3]), gi.make_grid(50.0, 12, 12, 12, ncont=24))


@pytest.mark.parametrize("name,case", list(cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_polarization_tc(gw, name, case):
    cr, gr = case
    ctx = gw.GW(gr, cr, omega=1.0)
    G, _ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    for iq in range(cr.nq):
        P = zeros((gr.ntau, cr.ni, cr.ni), "c16")
        ctx.polarization(iq, dev(G), P, gw.GW_FP16X2)
        ctx.sync()
        ref = orc.polarization(gi.m_for_q(cr, iq), G, cr.kmq[iq])
        e = rel(host(P), ref)
        print(f"{name} q{iq}: P tensor-core rel err {e:.3e}")
        assert e < TOL_P
        Ph = host(P)
        assert np.abs(Ph - np.conj(np.swapaxes(Ph, 1, 2))).max() == 0.0


@pytest.mark.parametrize("name,case", list(cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_selfenergy_tc(gw, name, case):
    cr, gr = case
    ctx = gw.GW(gr, cr, omega=1.0)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(11)
    S = zeros((cr.nk, cr.nb, gr.ntau))
    Sx = zeros((cr.nk, cr.nb))
    Sref = np.zeros((cr.nk, cr.nb, gr.ntau))
    Sxref = np.zeros((cr.nk, cr.nb))
    for iq in range(cr.nq):
        X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
        W = -30.0 * (X @ np.conj(np.swapaxes(X, 1, 2))) / cr.ni
        ctx.selfenergy(iq, dev(G), dev(occ), dev(W), S, Sx, gw.GW_FP16X2)
        sc, sx, _ = orc.selfenergy(gi.m_for_q(cr, iq), G, W, cr.v[iq], cr.kmq[iq], occ)
        Sref += sc
        Sxref += sx
    ctx.sync()
    e = rel(host(S), Sref)
    ex = rel(host(Sx), Sxref)
    print(f"{name}: Sigma tensor-core rel err {e:.3e}; Sigma^x float-float rel err {ex:.3e}")
    assert e < TOL_S
    assert ex < TOL_SX_FF


def test_polarization_forms(gw):
    """Both covers of the Hermitian P, forced with GW_TUNE_POL_FORM on one context: the real
    matrix E = Re P + Im P (1) and Re P / Im P over the Hermitian half (2), at NI = 160 against the
    oracle, at NI = 256 and 384 against the FP64 GPU path, switching forms back and forth (the strip
    metadata is rebuilt for each); the default (0) takes E up to NI = 256."""
    cases_ = [("ni160", gi.make_crystal(78, 8, 12, 5, 160, 50.0, qlist=[3]), gi.make_grid(50.0, 12, 12, 12, ncont=24),
               True),
              ("ni256", *gi.make_config("nk64_nb64", nk=8, qlist=[3]), False),
              ("ni384", gi.make_crystal(79, 8, 24, 10, 384, 80.0, qlist=[2]), gi.make_grid(80.0, 16, 16, 16, ncont=24),
               False)]
    for name, cr, gr, with_oracle in cases_:
        ctx = gw.GW(gr, cr, omega=1.0)
        G, _ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
        Gd = dev(G)
        if with_oracle:
            ref = orc.polarization(gi.m_for_q(cr, 0), G, cr.kmq[0])
        else:
            P64 = zeros((gr.ntau, cr.ni, cr.ni), "c16")
            ctx.polarization(0, Gd, P64, gw.GW_FP64)
            ctx.sync()
            ref = host(P64)
        out = {}
        for form in (1, 2, 1, 0):
            ctx.set_tuning(gw.GW_TUNE_POL_FORM, form)
            P = zeros((gr.ntau, cr.ni, cr.ni), "c16")
            ctx.polarization(0, Gd, P, gw.GW_FP16X2)
            ctx.sync()
            Ph = host(P)
            e = rel(Ph, ref)
            print(f"{name} form {form}: P tensor-core rel err {e:.3e}")
            assert e < TOL_P
            assert np.abs(Ph - np.conj(np.swapaxes(Ph, 1, 2))).max() == 0.0
            if form in out:
                assert np.array_equal(out[form], Ph)  # the same form twice: the same bits
            out[form] = Ph
        assert np.array_equal(out[0], out[1] if cr.ni <= 256 else out[2])
        with pytest.raises(gw.GwError):
            ctx.set_tuning(gw.GW_TUNE_POL_FORM, 3)
        ctx.close()


def test_c2_full_size_tc_vs_fp64(gw):
    """Bench sizes (Nk = 64, Nb = 64, NI = 256, Ntau = 48), in the bench's launch configuration:
    tensor-core P and Sigma of one q against the FP64 GPU path everywhere, and against the oracle
    at sampled tau (P) and sampled (k, tau) (Sigma^c)."""
    cr, gr = gi.make_config("nk64_nb64", qlist=[7])
    ctx = gw.GW(gr, cr)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    Gd = dev(G)
    P64 = zeros((gr.ntau, cr.ni, cr.ni), "c16")
    P16 = zeros((gr.ntau, cr.ni, cr.ni), "c16")
    ctx.polarization(0, Gd, P64, gw.GW_FP64)
    ctx.polarization(0, Gd, P16, gw.GW_FP16X2)
    ctx.sync()
    e = rel(host(P16), host(P64))
    print(f"Nk=64: P tensor-core vs FP64 rel err {e:.3e}")
    assert e < TOL_P
    rng = np.random.default_rng(4)
    X = rng.standard_normal((gr.ntau, cr.ni, 16)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 16))
    W = dev(-(X @ np.conj(np.swapaxes(X, 1, 2))) * 5.0)
    S64 = zeros((cr.nk, cr.nb, gr.ntau))
    S16 = zeros((cr.nk, cr.nb, gr.ntau))
    Sx64 = zeros((cr.nk, cr.nb))
    Sx16 = zeros((cr.nk, cr.nb))
    ctx.selfenergy(0, Gd, dev(occ), W, S64, Sx64, gw.GW_FP64)
    ctx.selfenergy(0, Gd, dev(occ), W, S16, Sx16, gw.GW_FP16X2)
    ctx.sync()
    e = rel(host(S16), host(S64))
    ex = rel(host(Sx16), host(Sx64))
    print(f"Nk=64: Sigma tensor-core vs FP64 rel err {e:.3e}; Sigma^x float-float vs FP64 {ex:.3e}")
    assert e < TOL_S
    assert ex < TOL_SX_FF
    # against the oracle at sampled points
    its, ks = [0, 24, 47], [0, 63]
    M = gi.m_for_q(cr, 0)
    Pr = orc.polarization(M, G, cr.kmq[0], its=its)
    eP = rel(host(P16)[its], Pr)
    Wh = host(W)
    Sr, Sxr, _ = orc.selfenergy(M[ks], G, Wh, cr.v[0], cr.kmq[0], occ, ks=ks, its=its)
    S16h, Sx16h = host(S16), host(Sx16)
    eS = max(rel(S16h[k][:, its], Sr[k][:, its]) for k in ks)
    eX = max(rel(Sx16h[k], Sxr[k]) for k in ks)
    print(f"Nk=64 vs oracle: P tensor-core {eP:.3e}, Sigma^c tensor-core {eS:.3e}, Sigma^x float-float {eX:.3e}")
    assert eP < TOL_P and eS < TOL_S and eX < TOL_SX_FF


def test_chain_qp_gap_mixed_vs_fp64(gw):
    """Whole G0W0 chain (all q) with the Nk=64 crystal's shapes at Nk = 8 and the paper's silicon cell volume:
    quasiparticle energies and the band gap from the tensor-core path against the FP64 path,
    with Pade and with CPE continuation. Reported with the |Sigma| scale it was measured at."""
    from paper_1602_02313_gb300.driver import Chain
    cr, gr = gi.make_config("nk64_nb64", nk=8)
    res = {}
    # the mixed chain as the bench runs it (float-float dielectric solve, the default), and with the
    # plain FP32 solve
    runs = [("fp64", gw.GW_FP64, None, (gw.GW_PADE, gw.GW_CPE)), ("fp16x2", gw.GW_FP16X2, None, (gw.GW_PADE, gw.GW_CPE)),
            ("fp16x2_f32screen", gw.GW_FP16X2, gw.GW_F32, (gw.GW_CPE,))]
    for name, prec, sprec, conts in runs:
        for cont in conts:
            ctx = gw.GW(gr, cr, omega=gi.OMEGA_SI)
            ch = Chain(ctx, dev(cr.eps), prec=prec, qb=4, cont_method=cont, screen_prec=sprec)
            ch.step()
            ch.check()
            res[(name, cont)] = {"eqp": host(ch.eqp).reshape(cr.nk, cr.nb), "sx": host(ch.Sx), "S": host(ch.S),
                                 "ok": host(ch.qinfo) == 0}
            ctx.close()
    gap = lambda E: E[:, cr.nocc].min() - E[:, cr.nocc - 1].max()  # noqa: E731
    ha2mev = 27211.386
    for cont, cname in [(gw.GW_PADE, "pade"), (gw.GW_CPE, "cpe")]:
        a, b = res[("fp64", cont)], res[("fp16x2", cont)]
        dE = np.abs(a["eqp"] - b["eqp"]).max()
        dgap = abs(gap(a["eqp"]) - gap(b["eqp"]))
        eS = rel(b["S"], a["S"])
        print(f"chain nk=8 {cname}: |Sigma^x| {np.abs(a['sx']).max():.3e} Ha, |Sigma^c(tau)| {np.abs(a['S']).max():.3e} Ha;"
              f" Sigma^c rel err {eS:.3e}; max |dE_qp| {dE * ha2mev:.4f} meV; gap fp64 {gap(a['eqp']):.6f} Ha,"
              f" |dgap| {dgap * ha2mev:.4f} meV; QP roots found {a['ok'].mean():.3f}")
        assert eS < 1e-3
    a, b = res[("fp64", gw.GW_CPE)], res[("fp16x2", gw.GW_CPE)]
    assert abs(gap(a["eqp"]) - gap(b["eqp"])) * ha2mev < 1.0  # the 1 meV target, CPE continuation
    # the same with the dielectric solve in plain FP32 instead of float-float
    c = res[("fp16x2_f32screen", gw.GW_CPE)]
    dE, dgap = np.abs(a["eqp"] - c["eqp"]).max(), abs(gap(a["eqp"]) - gap(c["eqp"]))
    print(f"chain nk=8 cpe, FP32 screening: Sigma^c rel err {rel(c['S'], a['S']):.3e}; max |dE_qp| "
          f"{dE * ha2mev:.4f} meV; |dgap| {dgap * ha2mev:.4f} meV")
    assert rel(c["S"], a["S"]) < 1e-3
    assert dgap * ha2mev < 1.0


def test_ni512_shapes_tc_vs_fp64(gw):
    """The Nk=216 crystal's band and basis sizes (Nb = 128, NI = 512, Ntau = 64, beta = 400) at
    Nk = 8, one q: tensor-core P (K segments in two passes over the partial buffer) and Sigma
    (output columns in two parts of 256) against the FP64 GPU path; M generated per q on demand
    must equal M generated at context creation."""
    import torch
    cr, gr = gi.make_config("nk216_nb128", nk=8, qlist=[3])
    ctx = gw.GW(gr, cr, m_mode=2)
    ref = gw.GW(gr, cr, m_mode=1)
    a = torch.empty((2, cr.ni, cr.nb, cr.nb), dtype=torch.complex128, device="cuda")
    b = torch.empty_like(a)
    ctx.copy_m(0, 5, 2, a)
    ref.copy_m(0, 5, 2, b)
    ctx.sync()
    ref.sync()
    assert torch.equal(a, b)
    ref.close()
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    Gd = dev(G)
    P64 = zeros((gr.ntau, cr.ni, cr.ni), "c16")
    P16 = zeros((gr.ntau, cr.ni, cr.ni), "c16")
    ctx.polarization(0, Gd, P64, gw.GW_FP64)
    ctx.polarization(0, Gd, P16, gw.GW_FP16X2)
    ctx.sync()
    e = rel(host(P16), host(P64))
    print(f"NI=512: P tensor-core vs FP64 rel err {e:.3e}")
    assert e < TOL_P
    rng = np.random.default_rng(5)
    X = rng.standard_normal((gr.ntau, cr.ni, 16)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 16))
    W = dev(-(X @ np.conj(np.swapaxes(X, 1, 2))) * 5.0)
    S64 = zeros((cr.nk, cr.nb, gr.ntau))
    S16 = zeros((cr.nk, cr.nb, gr.ntau))
    ctx.selfenergy(0, Gd, dev(occ), W, S64, None, gw.GW_FP64)
    ctx.selfenergy(0, Gd, dev(occ), W, S16, None, gw.GW_FP16X2)
    ctx.sync()
    e = rel(host(S16), host(S64))
    print(f"NI=512: Sigma tensor-core vs FP64 rel err {e:.3e}")
    assert e < TOL_S


def test_c3_full_size_sigma_tc_sampled(gw):
    """The Nk=216 crystal at its full size (Nk = 216, Nb = 128, NI = 512, Ntau = 64; M generated per q
    on demand, as the bench's c3 run does), one q: the tensor-core Sigma^c (output columns in two
    parts) and the float-float Sigma^x against the oracle at sampled k and tau, with a Hermitian
    stand-in for W~(tau)."""
    cr, gr = gi.make_config("nk216_nb128", qlist=[7])
    ctx = gw.GW(gr, cr, m_mode=2)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((gr.ntau, cr.ni, 8)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 8))
    W = -30.0 * (X @ np.conj(np.swapaxes(X, 1, 2))) / 8
    S = zeros((cr.nk, cr.nb, gr.ntau))
    Sx = zeros((cr.nk, cr.nb))
    ctx.selfenergy(0, dev(G), dev(occ), dev(W), S, Sx, gw.GW_FP16X2)
    ctx.sync()
    ks, its = [0, 101, 215], [0, 37, 63]
    Sr, Sxr, _ = orc.selfenergy(gi.m_for_q(cr, 0, ks=ks), G, W, cr.v[0], cr.kmq[0], occ, ks=ks, its=its)
    Sh, Sxh = host(S), host(Sx)
    eS = max(rel(Sh[k][:, its], Sr[k][:, its]) for k in ks)
    eX = max(rel(Sxh[k], Sxr[k]) for k in ks)
    print(f"Nk=216 vs oracle: Sigma^c tensor-core {eS:.3e}, Sigma^x float-float {eX:.3e}")
    assert eS < TOL_S and eX < TOL_SX_FF
    ctx.close()
