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
