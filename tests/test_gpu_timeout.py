"""Failure detection in the tensor-core pipelines, tested without faulting the GPU.

Every pipeline wait of k_pol_tc and k_sig_tc is bounded (GW_TUNE_WAIT_CYCLES). Here the stall
is injected from the host: GW_TUNE_FAULT_STALL makes the MMA-issuing thread of every block first
wait on a barrier that nothing arrives on, with a budget of about a millisecond. The wait runs
out; the block stops, lets the copies and MMAs it already issued finish, frees its tensor memory
and returns; gw_sync reports GW_ETIMEOUT once and clears it. Restoring the knobs, the same
context gives the healthy results again (bit for bit: the kernels are deterministic).
"""
import numpy as np
import pytest

import gwinputs as gi
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def test_wait_runs_out_reports_timeout_and_context_recovers(gw):
    import torch
    cr, gr = gi.make_config("nk8_nb16")
    ctx = gw.GW(gr, cr, omega=1.0)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    Gd, occd = torch.from_numpy(G).cuda(), torch.from_numpy(occ).cuda()
    rng = np.random.default_rng(5)
    X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
    Wd = torch.from_numpy(-30.0 * (X @ np.conj(np.swapaxes(X, 1, 2))) / cr.ni).cuda()

    def run():
        P = torch.zeros((gr.ntau, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
        S = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
        ctx.polarization(0, Gd, P, gw.GW_FP16X2)
        ctx.selfenergy(0, Gd, occd, Wd, S, None, gw.GW_FP16X2)
        return P, S

    P0, S0 = run()
    ctx.sync()
    # the knobs are checked on the host
    for key, bad in [(gw.GW_TUNE_WAIT_CYCLES, 10), (gw.GW_TUNE_FAULT_STALL, 2)]:
        with pytest.raises(gw.GwError, match="GW_EINVAL"):
            ctx.set_tuning(key, bad)
    # stalled: each contraction's wait runs out after ~1 ms (2e6 cycles)
    ctx.set_tuning(gw.GW_TUNE_WAIT_CYCLES, 2_000_000)
    ctx.set_tuning(gw.GW_TUNE_FAULT_STALL, 1)
    for call in ("polarization", "selfenergy"):
        P = torch.zeros((gr.ntau, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
        S = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
        if call == "polarization":
            ctx.polarization(0, Gd, P, gw.GW_FP16X2)
        else:
            ctx.selfenergy(0, Gd, occd, Wd, S, None, gw.GW_FP16X2)
        with pytest.raises(gw.GwError, match="GW_ETIMEOUT"):
            ctx.sync()
        ctx.sync()  # reported once, then cleared
    # healthy again: the same results as before the stall
    ctx.set_tuning(gw.GW_TUNE_FAULT_STALL, 0)
    ctx.set_tuning(gw.GW_TUNE_WAIT_CYCLES, 4_000_000_000)
    P1, S1 = run()
    ctx.sync()
    assert torch.equal(P1, P0) and torch.equal(S1, S0)
    Pr = orc.polarization(gi.m_for_q(cr, 0), G, cr.kmq[0])
    assert np.abs(P1.cpu().numpy() - Pr).max() < 2e-5 * np.abs(Pr).max()
    ctx.close()
