"""Many heterogeneous crystals in one CUDA-graph launch, with a small autotuner.

Each crystal has its own libgw context and chain (driver.Chain). One GW iteration of every
crystal is captured into a single CUDA graph: the crystals are dealt to a number of branches
(streams forked from the capture stream and joined back at the end), each branch running its
crystals' chains one after another; replaying the graph is then one launch for the whole batch,
and the branches let small crystals fill the GPU beside large ones. Host work (argument
checking, the launch sequence) is paid once at capture.

The autotuner picks, per crystal shape, the polarization's K-segment length and partial-buffer
size (gw_set_tuning) from timed trial calls, and, for the batch, the number of branches: crystals
go to branches longest-first onto the least-loaded branch (their measured single-crystal times),
each candidate graph is captured and timed, and the fastest is kept.

The queued schedule (step_queued, capture_queued) runs the batch on one stream instead: for each
q index, the polarizations of every crystal that has that q go to one persistent launch whose
blocks pull (crystal, K segment, strip, tau) units from a device counter
(gw_polarization_many); each crystal's transforms, screening and self-energy of that q follow.
Its results equal the per-crystal chains' bit for bit.
"""
from __future__ import annotations

import json
import os

import torch

from . import (GW, GW_BOSE, GW_CPE, GW_FP16X2, GW_IW_TO_TAU, GW_TAU_TO_IW, GW_TUNE_POL_PART_MB,
               GW_TUNE_POL_SEG_CHUNKS, polarization_many)
from .driver import Chain, contraction_flops


def _shape_key(cr, gr):
    return f"nk{cr.nk}_nb{cr.nb}_ni{cr.ni}_nt{len(gr.tau)}"


class Batch:
    """A batch of (crystal, grid) systems on one GPU."""

    def __init__(self, systems, omega, prec=GW_FP16X2, qb=2, cont_method=GW_CPE, device=0):
        self.systems = list(systems)
        self.device = device
        self.s0 = torch.cuda.Stream(device)
        self.ctxs, self.chains, self.cstreams = [], [], []
        for cr, gr in self.systems:
            s = torch.cuda.Stream(device)
            self.cstreams.append(s)
            ctx = GW(gr, cr, omega=omega, device=device, stream=s, m_mode=1)
            eps = torch.from_numpy(cr.eps).to(f"cuda:{device}")
            self.ctxs.append(ctx)
            self.chains.append(Chain(ctx, eps, prec=prec, qb=qb, cont_method=cont_method))
        self.flops = sum(sum(contraction_flops(cr.nk, cr.nb, cr.ni, len(gr.tau))) * cr.nq
                         for cr, gr in self.systems)
        self.tuning = {}
        self.graph = None
        self.nbranch = None
        self.crystal_ms = None

    # ------------------------------------------------------------------ eager runs
    def _step(self, i):
        self.chains[i].step()

    def run_sequential(self):
        """Every crystal's iteration in turn on one stream, launched call by call (no graph)."""
        with torch.cuda.stream(self.s0):
            for i, ctx in enumerate(self.ctxs):
                ctx.set_stream(self.s0)
                self._step(i)

    def time_sequential(self, reps=1):
        self.run_sequential()
        torch.cuda.synchronize(self.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.s0)
        for _ in range(reps):
            self.run_sequential()
        e1.record(self.s0)
        torch.cuda.synchronize(self.device)
        return e0.elapsed_time(e1) / reps

    def time_crystals(self):
        """Single-crystal iteration times (ms), eager, on the capture stream."""
        out = []
        with torch.cuda.stream(self.s0):
            for i, ctx in enumerate(self.ctxs):
                ctx.set_stream(self.s0)
                self._step(i)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.s0)
                self._step(i)
                e1.record(self.s0)
                torch.cuda.synchronize(self.device)
                out.append(e0.elapsed_time(e1))
        self.crystal_ms = out
        return out

    # ------------------------------------------------------------------ tuning
    def tune_kernels(self, seg_choices=(32, 16), part_mb_choices=(2048, 512), cache=None):
        """Per crystal shape, time the polarization of the first q under each (segment chunks,
        partial MiB) pair and keep the fastest; `cache` (a JSON file path) stores the choices."""
        saved = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                saved = json.load(f)
        for i, (cr, gr) in enumerate(self.systems):
            key = _shape_key(cr, gr)
            ctx, ch = self.ctxs[i], self.chains[i]
            ctx.set_stream(self.s0)
            if key not in saved:
                best = None
                with torch.cuda.stream(self.s0):
                    ch.start_g0()
                    for seg in seg_choices:
                        for mb in part_mb_choices:
                            ctx.set_tuning(GW_TUNE_POL_SEG_CHUNKS, seg)
                            ctx.set_tuning(GW_TUNE_POL_PART_MB, mb)
                            ctx.polarization(ch.iqs[0], ch.G, ch.P[0], ch.prec)  # allocation, warm-up
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            e0.record(self.s0)
                            ctx.polarization(ch.iqs[0], ch.G, ch.P[0], ch.prec)
                            e1.record(self.s0)
                            torch.cuda.synchronize(self.device)
                            t = e0.elapsed_time(e1)
                            if best is None or t < best[0]:
                                best = (t, seg, mb)
                saved[key] = {"seg_chunks": best[1], "part_mb": best[2], "pol_ms": best[0]}
            ctx.set_tuning(GW_TUNE_POL_SEG_CHUNKS, saved[key]["seg_chunks"])
            ctx.set_tuning(GW_TUNE_POL_PART_MB, saved[key]["part_mb"])
            self.tuning[key] = saved[key]
        if cache:
            with open(cache, "w") as f:
                json.dump(saved, f, indent=1)
        return self.tuning

    @staticmethod
    def assign(ms, nbranch):
        """Longest first onto the least-loaded branch; returns a list of crystal-index lists."""
        loads = [0.0] * nbranch
        groups = [[] for _ in range(nbranch)]
        for i in sorted(range(len(ms)), key=lambda j: -ms[j]):
            b = min(range(nbranch), key=lambda j: loads[j])
            groups[b].append(i)
            loads[b] += ms[i]
        return [g for g in groups if g]

    # ------------------------------------------------------------------ graph
    def capture(self, groups):
        """One CUDA graph holding one iteration of every crystal; `groups` gives the crystals
        of each branch. Every chain must have run once eagerly (workspaces allocated)."""
        streams = [torch.cuda.Stream(self.device) for _ in groups]
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g, stream=self.s0):
            for s, grp in zip(streams, groups):
                s.wait_stream(self.s0)
                with torch.cuda.stream(s):
                    for i in grp:
                        self.ctxs[i].set_stream(s)
                        self._step(i)
            for s in streams:
                self.s0.wait_stream(s)
        self._keep = streams
        return g

    def time_graph(self, g, reps=2):
        """Device time of one replay (ms); replays are launched on the capture stream."""
        with torch.cuda.stream(self.s0):
            g.replay()
            torch.cuda.synchronize(self.device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.s0)
            for _ in range(reps):
                g.replay()
            e1.record(self.s0)
        torch.cuda.synchronize(self.device)
        return e0.elapsed_time(e1) / reps

    def tune_schedule(self, branch_choices=(1, 2, 4, 6, 12), reps=1):
        """Capture a graph for each branch count (crystals dealt by their measured times), time
        one replay each, keep the fastest. Returns {branches: ms}."""
        if self.crystal_ms is None:
            self.time_crystals()
        res, best = {}, None
        for nb in sorted(set(min(b, len(self.systems)) for b in branch_choices)):
            groups = self.assign(self.crystal_ms, nb)
            g = self.capture(groups)
            t = self.time_graph(g, reps)
            res[nb] = t
            if best is None or t < best[0]:
                best = (t, nb, g, groups)
            else:
                del g
        self.graph, self.nbranch, self.groups = best[2], best[1], best[3]
        return res

    # ------------------------------------------------------------------ device-queue schedule
    def step_queued(self):
        """One GW iteration of every crystal, the q indices in blocks of the chains' q-block size:
        on the capture stream, per q index one gw_polarization_many over all crystals that have it
        (at most 16 per call); then each crystal's bosonic transforms and screening of the block's
        q points and their self-energies on the crystal's own stream (forked from and joined back
        to the capture stream by events, so that the crystals' post-polarization work overlaps and
        the next block's polarizations wait for it)."""
        s0 = self.s0
        qb = min(ch.qb for ch in self.chains)
        with torch.cuda.stream(s0):
            for ctx, ch in zip(self.ctxs, self.chains):
                ctx.set_stream(s0)
                ch.start_g0()
                ch.S.zero_()
                ch.Sx.zero_()
            for j0 in range(0, max(len(ch.iqs) for ch in self.chains), qb):
                for j in range(j0, j0 + qb):
                    jobs = [i for i, ch in enumerate(self.chains) if j < len(ch.iqs)]
                    for g0 in range(0, len(jobs), 16):
                        grp = jobs[g0:g0 + 16]
                        polarization_many([self.ctxs[i] for i in grp], [self.chains[i].iqs[j] for i in grp],
                                          [self.chains[i].G for i in grp],
                                          [self.chains[i].P[j - j0] for i in grp], self.chains[grp[0]].prec)
                fork = torch.cuda.Event()
                fork.record(s0)
                joins = []
                for ctx, ch, st in zip(self.ctxs, self.chains, self.cstreams):
                    js = list(range(j0, min(j0 + qb, len(ch.iqs))))
                    if not js:
                        continue
                    st.wait_event(fork)
                    ctx.set_stream(st)
                    with torch.cuda.stream(st):
                        nb_, ni = len(js), ch.ni
                        ctx.tau_to_freq_many(GW_BOSE, GW_TAU_TO_IW, nb_, ni * ni, ch.P, ch.Piv, ch.bose_prec)
                        ctx.screen(ch.iqs[j0], nb_, ch.Piv[:nb_], ch.Wiv[:nb_], ch.info[:nb_], ch.screen_prec)
                        ctx.tau_to_freq_many(GW_BOSE, GW_IW_TO_TAU, nb_, ni, ch.Wiv, ch.Wt, ch.bose_prec)
                        for jj, j in enumerate(js):
                            ch._sigma_q(j, ch.iqs[j], ch.G, ch.occ, ch.Wt[jj])
                        ev = torch.cuda.Event()
                        ev.record(st)
                        joins.append(ev)
                    ctx.set_stream(s0)
                for ev in joins:
                    s0.wait_event(ev)
            for ch in self.chains:
                ch.finish()

    def capture_queued(self):
        """The queued schedule as one CUDA graph (run step_queued once eagerly first)."""
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g, stream=self.s0):
            self.step_queued()
        self.graph_queued = g
        return g

    def replay(self):
        with torch.cuda.stream(self.s0):
            self.graph.replay()

    def check(self):
        for ch in self.chains:
            ch.check()

    def close(self):
        self.graph = None
        for ctx in self.ctxs:
            ctx.close()
