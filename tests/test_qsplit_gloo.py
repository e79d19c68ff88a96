"""The multi-rank form of one iteration on CPU: q blocks per rank and the sum-all-reduce of the
partial self-energies (gloo, world size 2). Each rank computes its q points' contributions
with the FP64 oracle; the reduced arrays must equal the serial sum over all q."""
import os
import socket

import numpy as np
import pytest

from paper_1602_02313_gb300.qsplit import q_range


@pytest.mark.parametrize("nq,world", [(1, 1), (8, 2), (7, 2), (64, 8), (5, 8), (0, 3), (13, 4)])
def test_q_range_partitions(nq, world):
    seen = []
    for r in range(world):
        q0, n = q_range(nq, r, world)
        assert n >= 0 and 0 <= q0 <= nq
        seen += list(range(q0, q0 + n))
    assert seen == list(range(nq))  # disjoint, in order, complete


def test_q_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        q_range(4, 2, 2)


def _case():
    import gwinputs as gi
    import oracle as orc
    cr = gi.make_crystal(515, 8, 4, 2, 8, 30.0, qlist=list(range(8)))
    gr = gi.make_grid(cr.beta, 8, 8, 8)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(9)
    Wt = []
    for _ in range(cr.nq):
        X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
        Wt.append(0.5 * (X + np.conj(np.swapaxes(X, 1, 2))))  # Hermitian W~(tau)
    return cr, G, occ, Wt


def _partial(cr, G, occ, Wt, iqs):
    import gwinputs as gi
    import oracle as orc
    S = np.zeros((cr.nk, cr.nb, len(G[0, 0])))
    Sx = np.zeros((cr.nk, cr.nb))
    for iq in iqs:
        s, x, _ = orc.selfenergy(gi.m_for_q(cr, iq), G, Wt[iq], cr.v[iq], cr.kmq[iq], occ, omega=2.0)
        S += s
        Sx += x
    return S, Sx


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_1602_02313_gb300.qsplit import allreduce_sigma
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cr, G, occ, Wt = _case()
        q0, n = q_range(cr.nq, rank, world)
        S, Sx = _partial(cr, G, occ, Wt, range(q0, q0 + n))
        St, Sxt = torch.from_numpy(S), torch.from_numpy(Sx)
        allreduce_sigma(St, Sxt)
        np.savez(out.format(rank), S=St.numpy(), Sx=Sxt.numpy(), q0=q0, n=n)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_sigma_reduction(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "rank{}.npz")
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    cr, G, occ, Wt = _case()
    S, Sx = _partial(cr, G, occ, Wt, range(cr.nq))
    blocks = []
    for r in range(world):
        d = np.load(out.format(r))
        blocks.append((int(d["q0"]), int(d["n"])))
        # every rank holds the full sum after the reduction
        assert np.allclose(d["S"], S, rtol=1e-13, atol=1e-13 * np.abs(S).max())
        assert np.allclose(d["Sx"], Sx, rtol=1e-13, atol=1e-13 * np.abs(Sx).max())
    assert blocks == [(0, 4), (4, 4)]
