"""Learned CPE seed (not in the paper): the network's tensor-core gradients against the
FP64 oracle, training on G0W0 chains of synthetic crystals, and what the trained seed gains
over the plain CPE fit (fewer Lawson-Hanson iterations for the same continuation)."""
import numpy as np
import pytest

import gwinputs as gi
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_1602_02313_gb300 import build as b
    b.build()
    import paper_1602_02313_gb300 as pkg
    return pkg


def test_mlp_gradients_vs_oracle(gw):
    """Loss and gradients of the tensor-core network against the FP64 oracle network. The weights,
    the inputs and the CPE matrix are made exactly representable in fp16, so that the operand
    rounding of the first products is exact; what remains is the fp16 rounding of the hidden
    activations the kernels keep for the next product (2^-11 relative) and FP32 accumulation."""
    import torch
    net = gw.MLP(seed=3)
    rng = np.random.default_rng(7)
    f16 = lambda a: np.asarray(a, np.float32).astype(np.float16).astype(np.float32)  # noqa: E731
    net.set_params(f16(net.get_params()))
    x = f16(0.5 * rng.standard_normal((256, 128)))
    A = f16(0.05 * rng.standard_normal((128, 128)))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grads = torch.zeros(net.num_params(), dtype=torch.float32, device="cuda")
    net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(A).cuda(), loss, grads)
    torch.cuda.synchronize()
    p = net.get_params().astype(np.float64)
    sizes = [128, 256, 256, 256, 128]
    params, off = [], 0
    for din, dout in zip(sizes[:-1], sizes[1:]):
        W = p[off:off + din * dout].reshape(dout, din)
        off += din * dout
        params.append((W, p[off:off + dout]))
        off += dout
    ref_loss, ref = omlp.loss_and_grad(params, x.astype(np.float64), A.astype(np.float64))
    g = grads.cpu().numpy().astype(np.float64)
    eL = abs(float(loss.item()) - ref_loss) / ref_loss
    print(f"loss rel err {eL:.2e}")
    assert eL < 1e-3
    off = 0
    for l, (gW, gb) in enumerate(ref):
        GW_ = g[off:off + gW.size].reshape(gW.shape)
        off += gW.size
        Gb = g[off:off + gb.size]
        off += gb.size
        eW = np.linalg.norm(GW_ - gW) / np.linalg.norm(gW)
        eb = np.linalg.norm(Gb - gb) / max(np.linalg.norm(gb), 1e-30)
        print(f"layer {l}: |dW| rel err {eW:.2e}, |db| rel err {eb:.2e}")
        # fp16 hidden activations (11-bit significand) with FP32 accumulation
        assert eW < 1e-3 and eb < 1e-3
    net.close()


def test_training_and_seed_gain(gw):
    import torch

    from paper_1602_02313_gb300 import learned
    from paper_1602_02313_gb300.driver import Chain
    mk = lambda s: gi.make_config("nk64_nb64", nk=8, seed=s)  # noqa: E731
    x, A = learned.chain_samples(mk, [5001, 5002, 5003], gi.OMEGA_SI)
    net = gw.MLP(seed=11)
    hist = learned.train(net, x, A, steps=400, batch=512, lr=1e-3)
    print(f"training loss: {hist[0]:.4e} -> {hist[-1]:.4e} over 400 steps, {x.shape[0]} samples")
    assert hist[-1] < 0.2 * hist[0]
    # held-out crystal: plain CPE against the seeded CPE on the same Sigma
    cr, gr = mk(5101)
    ctx = gw.GW(gr, cr, omega=gi.OMEGA_SI)
    ch = Chain(ctx, torch.from_numpy(cr.eps).cuda(), prec=gw.GW_FP16X2, qb=4, cont_method=gw.GW_CPE)
    ch.start_g0()
    ch.sigma()
    ch.finish()
    it_cold = torch.zeros(cr.nk * cr.nb, dtype=torch.int32, device="cuda")
    ctx.cpe_iterations(it_cold)
    e_cold = ch.eqp.clone()
    b_cold = torch.zeros(cr.nk * cr.nb, len(ch.cpe_x) - 2, dtype=torch.float64, device="cuda")
    ctx.cpe_coeffs(b_cold)
    it_seed = learned.seeded_cpe(ctx, net, ch)
    b_seed = torch.zeros_like(b_cold)
    ctx.cpe_coeffs(b_seed)
    ctx.sync()
    ic, isd = it_cold.cpu().numpy(), it_seed.cpu().numpy()
    dE = (ch.eqp - e_cold).abs().max().item()
    print(f"Lawson-Hanson outer iterations: plain {ic.mean():.1f} (max {ic.max()}), seeded {isd.mean():.1f} "
          f"(max {isd.max()}); max |dE_qp| seeded vs plain {dE * 27211.386:.4f} meV")
    assert isd.mean() < ic.mean()
    assert dE * 27211.386 < 1.0
    ctx.close()
    net.close()
