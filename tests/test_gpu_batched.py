"""Several heterogeneous crystals in one CUDA graph (batched.Batch): the graph replay must give
exactly what the same chains give when launched call by call, crystal after crystal."""
import numpy as np
import pytest

import gwinputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def test_batch_graph_matches_sequential(gw):
    import torch

    from paper_1602_02313_gb300.batched import Batch
    systems = gi.batch_crystals(n=4, seed=4100, nb_choices=(16, 32), nk_choices=(8,), ntau_choices=(16, 24))
    batch = Batch(systems, omega=gi.OMEGA_SI, qb=2)
    with pytest.raises(gw.GwError):
        batch.ctxs[0].set_tuning(gw.GW_TUNE_POL_SEG_CHUNKS, 33)  # beyond the FP32 accumulation bound
    with pytest.raises(gw.GwError):
        batch.ctxs[0].set_tuning(gw.GW_TUNE_POL_PART_MB, 0)
    tuning = batch.tune_kernels(seg_choices=(32, 8), part_mb_choices=(64, 1))
    assert all(v["seg_chunks"] in (32, 8) for v in tuning.values())
    ms = batch.time_crystals()
    assert len(ms) == 4 and min(ms) > 0
    batch.run_sequential()
    torch.cuda.synchronize()
    batch.check()
    ref = [(ch.S.cpu().numpy().copy(), ch.Sx.cpu().numpy().copy(), ch.eqp.cpu().numpy().copy())
           for ch in batch.chains]
    for ch in batch.chains:  # the replay must rewrite every output
        ch.S.fill_(np.nan)
        ch.eqp.fill_(np.nan)
    res = batch.tune_schedule(branch_choices=(1, 2, 4))
    assert set(res) == {1, 2, 4} and batch.nbranch in res
    batch.replay()
    torch.cuda.synchronize()
    batch.check()
    for ch, (S, Sx, E) in zip(batch.chains, ref):
        assert np.array_equal(ch.S.cpu().numpy(), S)
        assert np.array_equal(ch.Sx.cpu().numpy(), Sx)
        assert np.array_equal(ch.eqp.cpu().numpy(), E)
    print(f"batch of 4: sequential crystals {['%.2f' % m for m in ms]} ms, graph by branches "
          f"{ {k: round(v, 2) for k, v in res.items()} } ms")
    batch.close()


def test_polarization_queue_matches_per_crystal(gw):
    """gw_polarization_many (one persistent launch whose blocks pull (crystal, K segment, strip, tau)
    units from a device counter) gives each crystal's gw_polarization bit for bit, and agrees with
    the oracle; a context given twice is refused on the host."""
    import torch

    import oracle as orc
    systems = gi.batch_crystals(n=3, seed=4200, nb_choices=(16, 32), nk_choices=(8,), ntau_choices=(16, 24))
    ctxs, Gs, refs, outs = [], [], [], []
    for cr, gr in systems:
        ctx = gw.GW(gr, cr, omega=1.0)
        G, _ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
        Gd = torch.from_numpy(G).cuda()
        P = torch.zeros((gr.ntau, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
        ctx.polarization(1, Gd, P, gw.GW_FP16X2)
        ctxs.append(ctx)
        Gs.append(Gd)
        refs.append(P)
        outs.append(torch.full_like(P, float("nan")))
    torch.cuda.synchronize()
    gw.polarization_many(ctxs, [1, 1, 1], Gs, outs)
    ctxs[0].sync()
    for (cr, gr), P, Pq in zip(systems, refs, outs):
        assert torch.equal(P, Pq)
        Pr = orc.polarization(gi.m_for_q(cr, 1), orc.green_tau0(cr.eps, gr.tau, gr.beta)[0], cr.kmq[1], its=[0, 5])
        assert np.abs(Pq.cpu().numpy()[[0, 5]] - Pr).max() < 2e-5 * np.abs(Pr).max()
    with pytest.raises(gw.GwError, match="GW_EINVAL"):
        gw.polarization_many([ctxs[0], ctxs[0]], [1, 2], Gs[:2], outs[:2])
    for ctx in ctxs:
        ctx.close()


def test_queued_batch_graph_matches_sequential(gw):
    """The batch on one stream, q index by q index with one queued polarization launch per index,
    eagerly and as one captured CUDA graph, equals the per-crystal chains bit for bit."""
    import torch

    from paper_1602_02313_gb300.batched import Batch
    systems = gi.batch_crystals(n=4, seed=4300, nb_choices=(16, 32), nk_choices=(8,), ntau_choices=(16, 24))
    batch = Batch(systems, omega=gi.OMEGA_SI, qb=2)
    batch.run_sequential()
    torch.cuda.synchronize()
    batch.check()
    ref = [(ch.S.cpu().numpy().copy(), ch.Sx.cpu().numpy().copy(), ch.eqp.cpu().numpy().copy())
           for ch in batch.chains]
    batch.step_queued()
    torch.cuda.synchronize()
    batch.check()
    for ch, (S, Sx, E) in zip(batch.chains, ref):
        assert np.array_equal(ch.S.cpu().numpy(), S) and np.array_equal(ch.eqp.cpu().numpy(), E)
    g = batch.capture_queued()
    for ch in batch.chains:
        ch.S.fill_(np.nan)
        ch.eqp.fill_(np.nan)
    with torch.cuda.stream(batch.s0):
        g.replay()
    torch.cuda.synchronize()
    batch.check()
    for ch, (S, Sx, E) in zip(batch.chains, ref):
        assert np.array_equal(ch.S.cpu().numpy(), S)
        assert np.array_equal(ch.Sx.cpu().numpy(), Sx)
        assert np.array_equal(ch.eqp.cpu().numpy(), E)
    batch.close()
