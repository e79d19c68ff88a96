"""One GW iteration through the libgw C ABI (host orchestration only; every
step runs in libgw's kernels).

Order of the steps follows the paper's cycle (Sec. III.B): G(tau) -> for every
q: P(tau) [Eq. irpol] -> P(i nu) -> W~(i nu) [Eq. tildeW, solved in i nu] ->
W~(tau) -> Sigma^c(tau) += [Eq. sigc], Sigma^x += [Eq. sigx]; then
Sigma^c(i w) [Eq. trans] on the sparse set (Dyson) and on the dense set
(continuation), the diagonal Dyson update of G [Eqs. dysongf-zcjk] and the
analytic continuation with quasiparticle energies (Sec. III.B.6).
Screening runs for a batch of q at once (one thread block per (q, nu) system).
"""
from __future__ import annotations

import torch

from . import (GW_BOSE, GW_CPE, GW_F32, GW_F32X2, GW_FERMI, GW_FP16X2, GW_FP64, GW_IW_TO_TAU, GW_PADE, GW_TAU_TO_IW,
               GW_TAU_TO_IW_CONT, GwError)


def cpe_grid(nhat=128, xmin=0.01, xmax=50.0):
    """Real-frequency nodes of the continuous-pole expansion: +-geomspace(xmin, xmax, nhat/2)
    and two end nodes where the hats vanish (same construction as the oracle's)."""
    import numpy as np
    h = nhat // 2
    g = np.geomspace(xmin, xmax, h)
    r = g[1] / g[0]
    return np.concatenate([[-xmax * r], -g[::-1], g, [xmax * r]])


def contraction_flops(nk, nb, ni, ntau):
    """Algorithmic real flops of one q (8 per complex multiply-add; the Hermitian half of P):
    P: 4 NI^2 Nb^2 per (k, tau); Sigma^c: 8 NI^2 Nb^2 + 8 NI Nb^2 per (k, tau)."""
    p = 4.0 * ni * ni * nb * nb * nk * ntau
    s = (8.0 * ni * ni * nb * nb + 8.0 * ni * nb * nb) * nk * ntau
    return p, s


class Chain:
    """Buffers and call sequence of one GW iteration on a libgw context."""

    def __init__(self, ctx, eps, prec=GW_FP16X2, qb=8, iqs=None, cont_method=GW_PADE, cpe_ridge=1e-3, mlp=None,
                 nfit=64, screen_prec=None, keep_w=False, star=None):
        self.ctx = ctx
        g, cr = ctx.grid, ctx.cr
        self.nk, self.nb, self.ni, self.ntau = cr.nk, cr.nb, cr.ni, len(g.tau)
        self.nnu, self.nw, self.ncont = len(g.nu_idx), len(g.w_idx), g.ncont
        self.prec = prec
        # the dielectric solve: native FP64 on the FP64 chain, float-float (FP64-grade, ~44-bit
        # significand) on the mixed one; screen_prec=GW_F32 selects plain FP32. The bosonic
        # transforms: FP64 on the FP64 chain, float-float on the mixed one.
        if screen_prec is None:
            screen_prec = GW_FP64 if prec == GW_FP64 or ctx.cr.ni % 32 else GW_F32X2
        self.screen_prec = screen_prec
        # crystal symmetry (Sec. III.C): iqs are the irreducible q points and star[j] the
        # device int32 [nrep][nk] map k -> R^-1 k of each member of iqs[j]'s star; every q's
        # self-energy goes to T buffers first and is carried to its star (gw_sigma_star)
        self.star = star
        self.bose_prec = GW_FP64 if screen_prec == GW_FP64 else GW_F32X2
        self.iqs = list(range(cr.nq)) if iqs is None else list(iqs)
        self.qb = max(1, min(qb, len(self.iqs)))
        self.cont_method = cont_method
        d = dict(device="cuda")
        f8, c16 = torch.float64, torch.complex128
        self.eps = eps
        nk, nb, ni, nt = self.nk, self.nb, self.ni, self.ntau
        self.G = torch.zeros(nk, nb, nt, dtype=f8, **d)
        self.occ = torch.zeros(nk, nb, dtype=f8, **d)
        self.S = torch.zeros(nk, nb, nt, dtype=f8, **d)
        self.Sx = torch.zeros(nk, nb, dtype=f8, **d)
        if star is not None:
            self.Tc = torch.zeros(nk, nb, nt, dtype=f8, **d)
            self.Tx = torch.zeros(nk, nb, dtype=f8, **d)
        self.P = torch.zeros(self.qb, nt, ni, ni, dtype=c16, **d)
        self.Piv = torch.zeros(self.qb, self.nnu, ni, ni, dtype=c16, **d)
        self.Wiv = torch.zeros(self.qb, self.nnu, ni, ni, dtype=c16, **d)
        self.Wt = torch.zeros(self.qb, nt, ni, ni, dtype=c16, **d)
        self.info = torch.zeros(self.qb, self.nnu, dtype=torch.int32, **d)
        self.Siw = torch.zeros(nk, nb, self.nw, dtype=c16, **d)
        self.Siwc = torch.zeros(nk, nb, self.ncont, dtype=c16, **d)
        # GW0 (Sec. III.B, after Eq. dysong): W~(tau) of every q kept from the first pass
        self.Wkeep = torch.zeros(len(self.iqs), nt, ni, ni, dtype=c16, **d) if keep_w else None
        self.G1 = torch.zeros_like(self.G)
        self.occ1 = torch.zeros_like(self.occ)
        self.eqp = torch.zeros(nk * nb, dtype=f8, **d)
        self.qinfo = torch.zeros(nk * nb, dtype=torch.int32, **d)
        self.vxc = None
        self.timers = None
        self.mlp = mlp
        if cont_method == GW_CPE:
            # ridge 1e-3 (relative to ||A||_F): above the noise of the mixed chain's Sigma(i w), so
            # that the fit, and the QP root it leads to, do not jump with rounding-level changes
            self.cpe_x = cpe_grid()
            ctx.cpe_setup(self.cpe_x, cpe_ridge)
        if mlp is not None:
            # learned seed of the CPE fit: network input / output buffers (rows padded to 128)
            nprob = nk * nb
            pad = (nprob + 127) // 128 * 128
            self.nfit = nfit
            self.feat = torch.zeros(pad, 2 * nfit, dtype=torch.float32, **d)
            self.scale = torch.ones(nprob, dtype=f8, **d)
            self.bhat = torch.zeros(pad, mlp.nout, dtype=torch.float32, **d)

    def _timed(self, key, fn):
        if self.timers is None:
            fn()
            return
        s = self.ctx.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        self.timers.setdefault(key, []).append((e0, e1))

    def start_g0(self):
        """Reference G0 from the band energies (Sec. III.B.1)."""
        self.ctx.green_tau(self.eps, self.G, self.occ)

    def sigma(self, G=None, occ=None):
        """Sigma^c(tau), Sigma^x of the context's q points (accumulated from zero)."""
        ctx = self.ctx
        G = self.G if G is None else G
        occ = self.occ if occ is None else occ
        self.S.zero_()
        self.Sx.zero_()
        ni = self.ni
        for b0 in range(0, len(self.iqs), self.qb):
            batch = self.iqs[b0:b0 + self.qb]
            nb_ = len(batch)
            for j, iq in enumerate(batch):
                self._timed("polarization", lambda: ctx.polarization(iq, G, self.P[j], self.prec))
            # the block's q points in one grid per direction
            ctx.tau_to_freq_many(GW_BOSE, GW_TAU_TO_IW, nb_, ni * ni, self.P, self.Piv, self.bose_prec)
            ctx.screen(batch[0], nb_, self.Piv[:nb_], self.Wiv[:nb_], self.info[:nb_], self.screen_prec)
            ctx.tau_to_freq_many(GW_BOSE, GW_IW_TO_TAU, nb_, ni, self.Wiv, self.Wt, self.bose_prec)
            for j, iq in enumerate(batch):
                if self.Wkeep is not None:
                    self.Wkeep[b0 + j].copy_(self.Wt[j])
                self._timed("selfenergy", lambda: self._sigma_q(b0 + j, iq, G, occ, self.Wt[j]))

    def sigma_fixed_w(self, G, occ):
        """Sigma^c(tau), Sigma^x from G with the W~(tau) kept by the first pass (GW0)."""
        self.S.zero_()
        self.Sx.zero_()
        for j, iq in enumerate(self.iqs):
            self._sigma_q(j, iq, G, occ, self.Wkeep[j])

    def _sigma_q(self, pos, iq, G, occ, Wt):
        """Sigma^c, Sigma^x += the contribution of q (and of its star, with symmetry)."""
        if self.star is None:
            self.ctx.selfenergy(iq, G, occ, Wt, self.S, self.Sx, self.prec)
            return
        self.Tc.zero_()
        self.Tx.zero_()
        self.ctx.selfenergy(iq, G, occ, Wt, self.Tc, self.Tx, self.prec)
        self.ctx.sigma_star(self.star[pos], self.Tc, self.S)
        self.ctx.sigma_star(self.star[pos], self.Tx, self.Sx)

    def finish(self, vxc=None):
        """Sigma(i w), Dyson update, continuation and QP energies from the summed Sigma."""
        ctx = self.ctx
        nkb = self.nk * self.nb
        if vxc is None:
            vxc = self.Sx  # reference xc potential = Sigma^x[G0] (G0W0 keeps eps~ = eps)
        ctx.tau_to_freq(GW_FERMI, GW_TAU_TO_IW, nkb, self.S, self.Siw)
        ctx.tau_to_freq(GW_FERMI, GW_TAU_TO_IW_CONT, nkb, self.S, self.Siwc)
        ctx.green_tau(self.eps, self.G1, self.occ1, self.Sx, vxc, self.Siw)
        if self.mlp is not None and self.cont_method == GW_CPE:
            nprob = nkb
            ctx.cpe_features(self.Siwc, self.nfit, self.feat[:nprob], self.scale)
            self.mlp.forward(self.feat, self.bhat)
            ctx.cpe_seed(self.bhat[:nprob], self.scale)
        ctx.continue_(self.cont_method, self.Siwc, self.eps.reshape(-1), self.Sx.reshape(-1),
                      vxc.reshape(-1), None, None, self.eqp, self.qinfo)

    def step(self):
        """One G0W0 pass: every row of the hot path over all q of the context."""
        self.start_g0()
        self.sigma()
        self.finish()
        self.vxc = self.Sx.clone()  # Sigma_0 = Sigma^x[G0], kept fixed by the later passes
        self.G_in = None

    def iterate(self, n, gw0=False, mix=1.0):
        """n self-consistent passes after step(): P, W~ and Sigma from the previous pass's
        dressed G (Eqs. dysongf-zcjk solved in i w), the Dyson update from the band energies
        with the new Sigma and the fixed reference potential. gw0=True keeps W~ of the first
        pass (the chain must be built with keep_w=True) and updates only G and Sigma.
        mix < 1 feeds each pass the linear mixture G_in = mix G_out + (1 - mix) G_in(previous)
        of the dressed G and of its occupations (the first pass's G_in(previous) is G0); the
        paper's passes are mix = 1."""
        if self.vxc is None:
            raise GwError("Chain.iterate: run step() first")
        if gw0 and self.Wkeep is None:
            raise GwError("Chain.iterate: GW0 needs a chain built with keep_w=True")
        if not hasattr(self, "G_in") or self.G_in is None:
            self.G_in, self.occ_in = self.G.clone(), self.occ.clone()
        for _ in range(n):
            if mix == 1.0:
                G, occ = self.G1.clone(), self.occ1.clone()
            else:
                G = self.G_in.mul_(1.0 - mix).add_(self.G1, alpha=mix).clone()
                occ = self.occ_in.mul_(1.0 - mix).add_(self.occ1, alpha=mix).clone()
            if gw0:
                self.sigma_fixed_w(G, occ)
            else:
                self.sigma(G, occ)
            self.finish(self.vxc)

    def check(self):
        ctx = self.ctx
        ctx.sync()
        if int(self.info.abs().sum()):
            raise GwError("zero pivot in a dielectric solve")
