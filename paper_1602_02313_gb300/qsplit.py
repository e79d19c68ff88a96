"""Sharding of one GW iteration over ranks (one process per GPU).

The self-energy is a sum over q of independent per-q contributions (Eqs. sigc, sigx):
every step from P_q(tau) to the q-th term of Sigma touches only that q. Ranks therefore
take contiguous blocks of q points, accumulate their partial Sigma^c(tau) and Sigma^x on
their own GPU, and one sum-all-reduce of those two arrays is the only exchange; the
Matsubara transform, Dyson update and continuation that follow are then identical on
every rank.
"""
from __future__ import annotations


def q_range(nq: int, rank: int, world: int) -> tuple[int, int]:
    """(first q, count) of `rank`: blocks of ceil(nq / world), the last ones possibly short
    or empty. The blocks are disjoint and cover 0 .. nq - 1."""
    if nq < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("q_range: need nq >= 0 and 0 <= rank < world")
    per = (nq + world - 1) // world
    q0 = min(rank * per, nq)
    return q0, max(0, min(per, nq - q0))


def allreduce_sigma(S, Sx, group=None):
    """Sum the ranks' partial Sigma^c(tau) and Sigma^x in place (no-op on one rank)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    dist.all_reduce(S, group=group)
    dist.all_reduce(Sx, group=group)
