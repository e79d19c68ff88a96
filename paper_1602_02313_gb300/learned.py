"""Learned seed of the continuous-pole expansion (not in the paper): training data from
G0W0 chains of synthetic crystals, training on the GPU, and the seeded continuation.

All arithmetic runs in libgw kernels (features, network, loss, Adam, seed, CPE); this
module only orders the calls.
"""
from __future__ import annotations

import torch

from . import GW, GW_CPE, GW_FP16X2, MLP
from .driver import Chain

NFIT = 64  # Matsubara points fed to the network: 2 x 64 = 128 inputs


def chain_samples(make_crystal_grid, seeds, omega, prec=GW_FP16X2, qb=4):
    """Network inputs x [N][2 NFIT] (float32, device) from the Sigma^c(i w) of G0W0 chains,
    one crystal per seed (make_crystal_grid(seed) -> (crystal, grid))."""
    xs = []
    A = None
    for s in seeds:
        cr, gr = make_crystal_grid(s)
        ctx = GW(gr, cr, omega=omega)
        ch = Chain(ctx, torch.from_numpy(cr.eps).cuda(), prec=prec, qb=qb, cont_method=GW_CPE)
        ch.start_g0()
        ch.sigma()
        ch.finish()
        nprob = cr.nk * cr.nb
        x = torch.zeros(nprob, 2 * NFIT, dtype=torch.float32, device="cuda")
        scale = torch.zeros(nprob, dtype=torch.float64, device="cuda")
        ctx.cpe_features(ch.Siwc, NFIT, x, scale)
        if A is None:
            A = torch.zeros(2 * NFIT, len(ch.cpe_x) - 2, dtype=torch.float32, device="cuda")
            ctx.cpe_fit_matrix(NFIT, A)
        ctx.sync()
        xs.append(x)
        ctx.close()
    return torch.cat(xs), A


def train(mlp, x, A, steps=400, batch=512, lr=1e-3, seed=0):
    """Adam on L = (1/B) sum ||A b_hat - x||^2 over random mini-batches; returns the losses."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0] - x.shape[0] % batch
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for it in range(steps):
        idx = torch.randint(0, x.shape[0], (batch,), generator=g).cuda()
        xb = x[idx].contiguous()
        mlp.train_step(xb, A, lr, loss)
        if it % 50 == 0 or it == steps - 1:
            hist.append(float(loss.item()))
    return hist


def seeded_cpe(ctx, mlp, chain):
    """Continuation of a chain's Sigma^c with the network's seed: features -> network ->
    warm start -> gw_continue(GW_CPE). Returns the Lawson-Hanson iteration counts."""
    nprob = chain.nk * chain.nb
    pad = (nprob + 127) // 128 * 128
    x = torch.zeros(pad, 2 * NFIT, dtype=torch.float32, device="cuda")
    scale = torch.ones(nprob, dtype=torch.float64, device="cuda")
    ctx.cpe_features(chain.Siwc, NFIT, x[:nprob], scale)
    out = torch.zeros(pad, mlp.nout, dtype=torch.float32, device="cuda")
    mlp.forward(x, out)
    ctx.cpe_seed(out[:nprob], scale)
    vxc = chain.Sx
    ctx.continue_(GW_CPE, chain.Siwc, chain.eps.reshape(-1), chain.Sx.reshape(-1), vxc.reshape(-1), None, None,
                  chain.eqp, chain.qinfo)
    iters = torch.zeros(nprob, dtype=torch.int32, device="cuda")
    ctx.cpe_iterations(iters)
    return iters


def trained_seed(omega, seeds=(9001, 9002, 9003), steps=400, device=0):
    """A network trained on the G0W0 chains of crystals with the Nk=64 crystal's band and basis sizes (Nk = 8) and the given
    seeds (kept apart from the benchmarked crystal's seed)."""
    import gwinputs as gi
    x, A = chain_samples(lambda s: gi.make_config("nk64_nb64", nk=8, seed=s), list(seeds), omega)
    net = MLP(seed=17, device=device)
    hist = train(net, x, A, steps=steps, batch=512, lr=1e-3)
    return net, hist


def continuation_gain(ctx, mlp, chain, reps=3):
    """On one chain's Sigma^c: QP energies and timing of the plain CPE fit, the CPE fit seeded by the
    network, and Pade, all through gw_continue. Returns a dict of host arrays and timings (ms, the
    best of reps; the seeded time includes the features, the network and the seed)."""
    from . import GW_PADE
    nprob = chain.nk * chain.nb
    vxc = chain.Sx.reshape(-1)
    eps, sx = chain.eps.reshape(-1), chain.Sx.reshape(-1)
    st = ctx.stream
    out = {}

    def timed(fn):
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    def plain():
        ctx.continue_(GW_CPE, chain.Siwc, eps, sx, vxc, None, None, chain.eqp, chain.qinfo)

    out["ms_plain"] = timed(plain)
    it = torch.zeros(nprob, dtype=torch.int32, device="cuda")
    ctx.cpe_iterations(it)
    out["iters_plain"] = it.cpu().numpy()
    out["e_plain"] = chain.eqp.cpu().numpy().copy()
    out["ms_seeded"] = timed(lambda: seeded_cpe(ctx, mlp, chain))
    ctx.cpe_iterations(it)
    out["iters_seeded"] = it.cpu().numpy()
    out["e_seeded"] = chain.eqp.cpu().numpy().copy()
    out["ms_pade"] = timed(lambda: ctx.continue_(GW_PADE, chain.Siwc, eps, sx, vxc, None, None, chain.eqp,
                                                 chain.qinfo))
    out["e_pade"] = chain.eqp.cpu().numpy().copy()
    return out
