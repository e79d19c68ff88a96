"""Benchmark of one GW iteration (G0W0 pass) of the Matsubara-time GW hot path.

Workload: synthetic crystal shaped like the paper's (Nk = 64 on a 4x4x4 grid, q on
the same grid, Nb = 64 with 32 occupied, NI = 256, Ntau = 48 Gauss-Legendre-in-log
nodes, 48 bosonic / fermionic Matsubara nodes, beta = 200 / Ha). One step = every
row of the hot path over all 64 q: G0, P(tau) (tensor cores), tau -> i nu, screening,
i nu -> tau, Sigma^c(tau) + Sigma^x (tensor cores), Sigma(i w) on the sparse and the
continuation sets, Dyson update, Pade continuation and QP energies.

metric / value: P + Sigma contraction throughput over the whole iteration, in
algorithmic TFLOP/s (8 real flops per complex multiply-add, Hermitian half of P);
ms_per_step is the GW iteration time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp16x2|fp64]
       python bench.py --impl reference ...   (the FP64 CPU oracle on a bounded sample)
Multi-GPU (torchrun, one rank per GPU): the q points are split over the ranks, each
rank computes its Sigma contributions and one all-reduce sums Sigma^c(tau), Sigma^x.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GW iteration time & P/Sigma contraction TFLOP/s, mixed vs FP64, at <=1 meV gap error"
FALLBACK_TENSOR_SUSTAINED = 1700.0   # TFLOP/s, profiling-recipe fallback (no MEASURED_PEAKS.json)
FALLBACK_TENSOR_BURST = 1900.0
FALLBACK_HBM = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return {"tensor_sustained": float(d.get("bf16_tflops_sustained", d.get("bf16_tflops"))),
                    "tensor_burst": float(d.get("bf16_tflops")), "hbm": float(d.get("hbm_gbs")),
                    "sm_mhz": (d.get("clocks_under_load") or {}).get("sm_mhz_median"),
                    "source": "measured (MEASURED_PEAKS.json)"}
        except Exception:
            pass
    return {"tensor_sustained": FALLBACK_TENSOR_SUSTAINED, "tensor_burst": FALLBACK_TENSOR_BURST,
            "hbm": FALLBACK_HBM, "sm_mhz": None, "source": "fallback (profiling recipe; MEASURED_PEAKS.json absent)"}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken
    on the current source of the kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_1602_02313_gb300", "csrc", "tc_mixed.cu")
    try:
        d = json.load(open(p)).get(kernel)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if d and d.get("src_sha") == sha:
            return d["bytes_per_launch"]
    except Exception:
        pass
    return None


def cpu_sample(cr, gr, omega, its=(0, 11, 23, 35), ks=(0, 9, 17, 26, 33, 41, 50, 60)):
    """The FP64 oracle on a bounded sample of the workload: P of one q at len(its) tau
    values (all k), and Sigma^c of one q at len(ks) k points x len(its) tau values.
    Returns (flops, seconds, description); the M tensor of the q is generated before timing."""
    import gwinputs as gi
    import oracle as orc
    M = gi.m_for_q(cr, 0)
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((gr.ntau, cr.ni, 8)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 8))
    W = -(X @ np.conj(np.swapaxes(X, 1, 2)))
    t0 = time.perf_counter()
    orc.polarization(M, G, cr.kmq[0], omega, its=list(its))
    orc.selfenergy(M[list(ks)], G, W, cr.v[0], cr.kmq[0], occ, omega, ks=list(ks), its=list(its))
    dt = time.perf_counter() - t0
    from paper_1602_02313_gb300.driver import contraction_flops
    fp, fs = contraction_flops(cr.nk, cr.nb, cr.ni, 1)
    flops = fp * len(its) + fs / cr.nk * len(ks) * len(its)
    desc = (f"oracle P of 1 q at {len(its)} tau (all {cr.nk} k) + Sigma^c of 1 q at {len(ks)} k x {len(its)} tau, "
            f"numpy/BLAS FP64")
    return flops, dt, desc


def run_reference(args, cfg):
    import gwinputs as gi
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cr, gr = gi.make_config(cfg)
    cores = os.cpu_count()
    for _ in range(args.warmup):
        cpu_sample(cr, gr, args.omega)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t, desc = cpu_sample(cr, gr, args.omega)
        tot_f += f
        tot_t += t
    value = tot_f / tot_t / 1e12
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(cfg, args, "oracle"),
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _gap_record(cfg, args, prec):
    """The committed measurement of the QP-gap error of this chain against the FP64 chain
    (`--config gapcheck`, profiles/gap_<cfg>.json), if it was taken on the current source of the
    tensor-core kernels; else {}."""
    p = os.path.join(ROOT, "profiles", f"gap_{cfg}.json")
    src = os.path.join(ROOT, "paper_1602_02313_gb300", "csrc", "tc_mixed.cu")
    if prec in ("fp64", "oracle") or not os.path.exists(p):
        return {}
    try:
        d = json.load(open(p))
        if d.get("src_sha") != hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]:
            return {}
        chain = "mixed_" + getattr(args, "screen", "f32x2")
        return {"gap_err_mev": {"cpe_ridge_1e-3": d["gap_err_mev"][chain + "/cpe_0.001"],
                                "pade": d["gap_err_mev"][chain + "/pade"]},
                "fp64_iteration_s": d["fp64_iteration_s"],
                "gap_source": f"profiles/gap_{cfg}.json ({d['command']}, all {cfg} q)"}
    except Exception:
        return {}


def _config(cfg, args, prec):
    import gwinputs as gi
    c = gi.CONFIGS[cfg]
    return {**_gap_record(cfg, args, prec), "workload": f"synthetic crystal {cfg}: Nk={c['nk']} (q on the same grid), Nb={c['nb']} "
                        f"({c['nocc']} occ), NI={c['ni']}, Ntau={c['ntau']}, Nnu=Nw={c['nnu']}, beta={c['beta']}",
            "precision": prec, "omega": args.omega, "continuation": getattr(args, "cont", "pade"),
            "screening": getattr(args, "screen", "f32x2") if prec != "fp64" else "fp64",
            "parallelism": f"q-split over {args.gpus} GPU(s)",
            "l2": "inputs larger than L2 (M tensor %.1f GB per q, P(tau) and W~(tau) %.0f MB per q each)" % (
                c["nk"] * c["ni"] * c["nb"] ** 2 * 16 / 1e9, c["ntau"] * c["ni"] ** 2 * 16 / 1e6)}


def _dtype(args):
    """The arithmetic of each step of the benchmarked chain."""
    if args.prec == "fp64":
        return "f64 (every step)"
    scr = "f32x2 (float-float)" if args.screen == "f32x2" else "f32"
    return (f"P and Sigma^c: fp16x2 split on tensor cores, fp32 accumulation, f32x2 segment sums; "
            f"dielectric solve: {scr}; bosonic transforms and Sigma^x: f32x2 (float-float); "
            f"G, Dyson, fermionic transforms, continuation: f64")


def run_batch(args, prec):
    """Twelve heterogeneous crystals (gwinputs.batch_crystals): one GW iteration of all of them
    launched call by call, crystal after crystal, against one replay of the autotuned CUDA graph of
    per-crystal branches and one replay of the queued graph (per q index, one persistent
    polarization launch whose blocks pull units of every crystal from a device counter). Not the
    headline workload; one GPU."""
    import torch

    import gwinputs as gi
    from paper_1602_02313_gb300.batched import Batch
    systems = gi.batch_crystals()
    batch = Batch(systems, omega=args.omega, prec=prec, qb=2)
    tuning = batch.tune_kernels()
    crystal_ms = batch.time_crystals()
    for _ in range(max(0, args.warmup - 1)):
        batch.run_sequential()
    seq_ms = batch.time_sequential(reps=args.steps)
    sched = batch.tune_schedule(branch_choices=(1, 2, 3, 4, 6, 12), reps=1)
    graph_ms = batch.time_graph(batch.graph, reps=args.steps)
    batch.check()
    # the queued schedule: per q index one persistent polarization launch over all crystals
    batch.step_queued()
    batch.check()
    gq = batch.capture_queued()
    queued_ms = batch.time_graph(gq, reps=args.steps)
    batch.check()
    best_ms = min(graph_ms, queued_ms)
    shapes = [f"Nk={cr.nk} Nb={cr.nb} NI={cr.ni} Ntau={len(gr.tau)} beta={gr.beta}" for cr, gr in systems]
    out = {"metric": METRIC + " (batch of 12 crystals)", "value": batch.flops / (best_ms * 1e-3) / 1e12,
           "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best_ms,
           "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": _dtype(args),
           "data": "synthetic",
           "config": {"workload": "batch of 12 heterogeneous synthetic crystals: " + "; ".join(shapes),
                      "sequential_ms": seq_ms, "graph_ms": graph_ms, "queued_graph_ms": queued_ms,
                      "speedup_vs_sequential": seq_ms / best_ms,
                      "branches": batch.nbranch, "graph_ms_by_branches": sched,
                      "crystal_ms": crystal_ms, "pol_tuning": tuning, "continuation": "cpe",
                      "l2": "inputs larger than L2"},
           "gpu_launches": None, "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out))
    batch.close()
    torch.cuda.synchronize()


def run_tau_screen(args):
    """The paper's tau-domain form of Eq. (tildeW) (gw_screen_tau) on the Nk=8 crystal's basis
    (NI = 64, beta = 100) and the uniform power mesh UPM(4, 2) (17 points): one dense solve of
    1088 unknowns with 64 right-hand sides. A cross-check of the i nu route, not a step of the
    benchmarked iteration; timed alone, one GPU."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    b.build()
    cr, gr = gi.make_config("nk8_nb16")
    p_, m_ = 4, 2
    tau = gi.upm_grid(gr.beta, p_, m_)
    npts, ni = len(tau), cr.ni
    # synthetic polarization at every mesh difference: four bosonic modes with random Hermitian
    # negative semidefinite weights (P(i nu) = -sum_s B_s B_s^+ 2 E_s / (nu^2 + E_s^2))
    d, idx = gi.tau_pairs(tau, gr.beta)
    rng = np.random.default_rng(20260)
    P = np.zeros((len(d), ni, ni), complex)
    for E in (0.3, 0.7, 1.2, 2.0):
        B = (rng.standard_normal((ni, 8)) + 1j * rng.standard_normal((ni, 8))) * (0.02 / np.sqrt(ni))
        shape = np.cosh(E * (d - 0.5 * gr.beta)) / np.sinh(0.5 * E * gr.beta)
        P -= shape[:, None, None] * (B @ B.conj().T)[None]
    Pp = np.ascontiguousarray(P[idx])
    ctx = gw.GW(gr, cr, omega=args.omega)
    Pd = torch.from_numpy(Pp).cuda()
    W = torch.zeros((npts, ni, ni), dtype=torch.complex128, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    ctx.set_stream(s)
    for _ in range(args.warmup):
        ctx.screen_tau(0, tau, Pd, W, info)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed solves only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        ctx.screen_tau(0, tau, Pd, W, info)
    e1.record(s)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - launches0
    assert int(info.item()) == 0
    N, L = npts * ni, npts * ni + ni
    macs = float(sum(N * (L - k) for k in range(N)))  # complex multiply-adds of the elimination
    fp64_tf, _ = gw.measure_alu(0)
    ach = 8.0 * macs / (ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "k_tsys_step (all N pivot steps of one solve, CUDA events around the call)",
            "achieved": ach, "peak": fp64_tf, "unit": "TFLOP/s FP64", "frac": ach / fp64_tf,
            "peak_source": "measured FP64 FMA rate of this GPU (gw_measure_alu, this run)",
            "flops_per_solve": 8.0 * macs}
    cpu = None
    if not args.no_cpu:
        import oracle as orc
        t0 = time.perf_counter()
        ref = orc.screen_tau.screen_tau(Pp, cr.v[0], tau)
        tc = time.perf_counter() - t0
        err = float(np.abs(W.cpu().numpy() - ref).max() / np.abs(ref).max())
        cpu = {"value": tc * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "the whole solve (oracle: numpy/LAPACK zgesv on the same system)", "max_rel_diff_vs_gpu": err}
    out = {"metric": "tau-domain W~ solve time (Eq. tildeW on the uniform power mesh)", "value": ms, "unit": "ms",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"tau-domain screening: NI={ni} (nk8_nb16 basis), beta={gr.beta}, UPM({p_},{m_}) "
                                  f"= {npts} points, {N} unknowns x {ni} right-hand sides",
                      "l2": "system (2 x 20 MB) resident in L2 between pivot steps"},
           "gpu_launches": int(launches), "roofline_alu": roof, "roofline": None, "cpu_baseline": cpu, "e2e": None}
    print(json.dumps(out))
    ctx.close()


def run_dyson_tau(args):
    """The paper's tau-domain Dyson equation (gw_dyson_tau) for every state of the benchmarked
    crystal (Nk = 64, Nb = 64: 4096 states) at beta = 100 on UPM(4, 8) (129 uniform points): one
    dense 129-unknown solve per state, one block per state. A cross-check of the i w Dyson
    update, not a step of the benchmarked iteration; timed alone, one GPU."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    b.build()
    cr, gr = gi.make_config("nk64_nb64")
    beta, p_, m_ = 100.0, 4, 8
    tu = gi.upm_grid(beta, p_, m_)
    h = tu[1] - tu[0]
    n = int(round(beta / h))
    eps = cr.eps.reshape(-1).copy()
    nprob = len(eps)
    rng = np.random.default_rng(20261)
    s = rng.uniform(-0.2, 0.2, nprob)
    # synthetic Sigma^c(tau): three poles per state, Sigma^c(i w) = sum c^2 / (i w - E)
    sig = np.zeros((nprob, len(tu)))
    for _ in range(3):
        c2, E = rng.uniform(0.01, 0.1, nprob), rng.uniform(-1.5, 1.5, nprob)
        x = -np.where(E[:, None] >= 0, np.exp(-np.outer(E, tu)) / (1.0 + np.exp(-beta * E))[:, None],
                      np.exp(np.outer(E, beta - tu)) / (1.0 + np.exp(beta * E))[:, None])
        sig += c2[:, None] * x
    ctx = gw.GW(gr, cr, omega=args.omega, m_mode=2)
    d_eps, d_s, d_sig = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (eps, s, sig))
    G = torch.zeros((nprob, n + 1), dtype=torch.float64, device="cuda")
    info = torch.zeros(nprob, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    ctx.set_stream(st)
    for _ in range(args.warmup):
        ctx.dyson_tau(tu, d_eps, d_s, d_sig, G, info)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    torch.cuda.profiler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.dyson_tau(tu, d_eps, d_s, d_sig, G, info)
    e1.record(st)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - launches0
    assert int((info != 0).sum().item()) == 0
    np1 = n + 1
    # FP64 multiply-adds per state: the Z^c sum (np1^3) and the elimination (sum_k np1 (np1 + 1 - k))
    fmas = float(np1) ** 3 + float(sum(np1 * (np1 + 1 - k) for k in range(np1)))
    fp64_tf, _ = gw.measure_alu(0)
    ach = 2.0 * fmas * nprob / (ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "k_dyson_tau (one block per state; CUDA events around the call)",
            "achieved": ach, "peak": fp64_tf, "unit": "TFLOP/s FP64", "frac": ach / fp64_tf,
            "peak_source": "measured FP64 FMA rate of this GPU (gw_measure_alu, this run)",
            "flops_per_state": 2.0 * fmas}
    cpu = None
    if not args.no_cpu:
        import time

        import oracle as orc
        nsamp = 256
        t0 = time.perf_counter()
        ref = np.stack([orc.dyson_tau.dyson_tau(eps[i], s[i], sig[i], tu)[0] for i in range(nsamp)])
        tc = time.perf_counter() - t0
        err = float(np.abs(G[:nsamp].cpu().numpy() - ref).max() / np.abs(ref).max())
        cpu = {"value": tc * 1e3 * nprob / nsamp, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the first {nsamp} of the {nprob} states (numpy/LAPACK), scaled to all states",
               "max_rel_diff_vs_gpu": err}
    out = {"metric": "tau-domain Dyson solve time, all states (Eqs. dysongf-dysong)", "value": ms, "unit": "ms",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"tau-domain Dyson: {nprob} states (nk64_nb64 band energies), beta={beta}, "
                                  f"Sigma^c on UPM({p_},{m_}) = {len(tu)} points, spline to {np1} uniform points",
                      "l2": "per-state systems (133 KB each) written and solved by one block"},
           "gpu_launches": int(launches), "roofline_alu": roof, "roofline": None, "cpu_baseline": cpu, "e2e": None}
    print(json.dumps(out))
    ctx.close()


def run_sym(args, prec):
    """Crystal-symmetry reduction (Sec. III.C) on a synthetic Oh crystal (4 x 4 x 4 mesh, Nb = 32,
    plane-wave product basis padded to NI = 64): one G0W0 iteration of the mixed chain over all
    64 q against the same over the 10 irreducible q (each q's self-energy carried to its star).
    Not the headline workload; one GPU."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from gwinputs import symmetric as sy
    from paper_1602_02313_gb300 import build as b
    from paper_1602_02313_gb300.driver import Chain, contraction_flops
    b.build()
    c = sy.make_symmetric_crystal(n=4, nb=32, nocc=16, cut=4.6, beta=100.0, seed=17)
    gr = gi.make_grid(c.beta, 32, 32, 32, ncont=64)
    eps = torch.from_numpy(c.eps).cuda()
    st = torch.cuda.current_stream()
    res = {}
    for name, qs in (("full", list(range(c.nq))), ("irreducible", list(c.ibz))):
        cq = sy.restrict_q(c, qs)
        M = torch.from_numpy(cq.M).cuda()
        ctx = gw.GW(gr, cq, omega=args.omega, M=M, stream=st)
        star = None if name == "full" else [torch.from_numpy(sy.star_kinv(c, q)).cuda() for q in qs]
        ch = Chain(ctx, eps, prec=prec, qb=len(qs), cont_method=gw.GW_CPE, star=star)
        for _ in range(args.warmup):
            ch.step()
        ch.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            ch.step()
        e1.record(st)
        torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1) / args.steps, ch.S.cpu().numpy().copy(), ch.eqp.cpu().numpy().copy())
        ctx.close()
        del M, ch
        torch.cuda.empty_cache()
    fp, fs = contraction_flops(c.nk, c.nb, c.ni, len(gr.tau))
    ms_full, S_full, E_full = res["full"]
    ms_red, S_red, E_red = res["irreducible"]
    out = {"metric": "symmetry-reduced G0W0 iteration time (Sec. III.C)", "value": ms_red, "unit": "ms",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_red, "higher_is_better": False,
           "scaling": "strong", "vs_baseline": None, "dtype": _dtype(args), "data": "synthetic",
           "config": {"workload": f"synthetic Oh crystal: 4x4x4 mesh, Nb={c.nb} ({c.nocc} occ), NI={c.ni}, "
                                  f"Ntau={len(gr.tau)}, beta={c.beta}; {len(c.ibz)} irreducible of {c.nq} q",
                      "full_mesh_ms": ms_full, "speedup": ms_full / ms_red,
                      "effective_tflops": (fp + fs) * c.nq / (ms_red * 1e-3) / 1e12,
                      "max_rel_diff_sigma_c": float(np.abs(S_red - S_full).max() / np.abs(S_full).max()),
                      "max_abs_diff_qp_ha": float(np.abs(E_red - E_full).max()), "continuation": "cpe"},
           "gpu_launches": None, "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out))


def run_offdiag(args):
    """Off-diagonal self-energy (gw_selfenergy_offdiag, FP64) of one q of a synthetic crystal with
    Nk = 64, Nb = 32, NI = 128, Ntau = 32; timed alone against the measured FP64 rate."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    b.build()
    cr = gi.make_crystal(seed=2101, nk=64, nb=32, nocc=16, ni=128, beta=100.0, qlist=[5])
    gr = gi.make_grid(100.0, 32, 32, 32, ncont=64)
    ctx = gw.GW(gr, cr, omega=args.omega)
    rng = np.random.default_rng(2102)
    X = rng.standard_normal((gr.ntau, cr.ni, cr.ni)) + 1j * rng.standard_normal((gr.ntau, cr.ni, cr.ni))
    W = torch.from_numpy(-(X @ np.conj(np.swapaxes(X, 1, 2))) / cr.ni).cuda()
    G = torch.from_numpy(np.ascontiguousarray(np.repeat(-np.exp(-np.abs(cr.eps))[:, :, None], gr.ntau, 2))).cuda()
    occ = torch.from_numpy((cr.eps < 0).astype(np.float64)).cuda()
    S = torch.zeros((cr.nk, cr.nb, cr.nb, gr.ntau), dtype=torch.complex128, device="cuda")
    Sx = torch.zeros((cr.nk, cr.nb, cr.nb), dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream()
    ctx.set_stream(st)
    for _ in range(args.warmup):
        ctx.selfenergy_offdiag(0, G, occ, W, S, Sx)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.selfenergy_offdiag(0, G, occ, W, S, Sx)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    nk, nb, ni, nt = cr.nk, cr.nb, cr.ni, gr.ntau
    macs = float(nk) * nt * nb * (ni * ni * nb + ni * nb * nb) + float(nk) * nb ** 3 * ni
    fp64_tf, _ = gw.measure_alu(0)
    ach = 8.0 * macs / (ms * 1e-3) / 1e12
    out = {"metric": "off-diagonal self-energy time, one q (Eqs. sigc, sigx as band matrices)", "value": ms,
           "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"one q: Nk={nk}, Nb={nb}, NI={ni}, Ntau={nt}"},
           "gpu_launches": 2 * args.steps,
           "roofline_alu": {"bound": "alu", "kernel": "k_sigma_offdiag + k_sigx_offdiag", "achieved": ach,
                            "peak": fp64_tf, "unit": "TFLOP/s FP64", "frac": ach / fp64_tf,
                            "peak_source": "measured FP64 FMA rate of this GPU (gw_measure_alu, this run)"},
           "roofline": None, "cpu_baseline": None, "e2e": None}
    print(json.dumps(out))
    ctx.close()


def run_gap_check(args):
    """The metric's accuracy claim on the benchmarked crystal (nk64_nb64, all 64 q): one G0W0 iteration
    in FP64 (every step FP64) and in the mixed form (tensor-core P and Sigma^c, float-float or FP32
    dielectric solve), the same continuation applied to both: CPE at ridges 1e-3, 1e-4, 1e-5 and Pade.
    Reports each chain's quasiparticle gap, the gap differences and the largest QP-energy difference
    (meV), the |Sigma| scale and the FP64 iteration time. A measurement run, not a bench line."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    from paper_1602_02313_gb300.driver import Chain, cpe_grid
    b.build()
    cr, gr = gi.make_config(args.gap_config)
    if args.nq > 0:
        cr = gi.subset_q(cr, 0, min(args.nq, cr.nq))
    ctx = gw.GW(gr, cr, omega=args.omega)
    eps = torch.from_numpy(cr.eps).cuda()
    HA_MEV = 27211.386245988
    ridges = (1e-3, 1e-4, 1e-5)
    variants = [("fp64", gw.GW_FP64, gw.GW_FP64), ("mixed_f32x2", gw.GW_FP16X2, gw.GW_F32X2),
                ("mixed_f32", gw.GW_FP16X2, gw.GW_F32)]
    res, eq = {}, {}
    for name, prec, sprec in variants:
        ch = Chain(ctx, eps, prec=prec, qb=min(64, cr.nq), cont_method=gw.GW_CPE, screen_prec=sprec)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ch.step()
        e1.record(st)
        ch.check()
        r = {"iteration_ms": e0.elapsed_time(e1), "sigx_max_abs_ha": float(ch.Sx.abs().max()),
             "sigc_iw0_max_abs_ha": float(ch.Siwc[:, :, 0].abs().max())}
        for ridge in ridges:
            ctx.cpe_setup(cpe_grid(), ridge)
            ch.cont_method = gw.GW_CPE
            ch.finish(ch.vxc)
            ch.check()
            e = ch.eqp.cpu().numpy().reshape(cr.nk, cr.nb).copy()
            eq[(name, f"cpe_{ridge:g}")] = e
            r[f"gap_cpe_{ridge:g}_ha"] = float(e[:, cr.nocc].min() - e[:, cr.nocc - 1].max())
        ch.cont_method = gw.GW_PADE
        ch.finish(ch.vxc)
        ch.check()
        e = ch.eqp.cpu().numpy().reshape(cr.nk, cr.nb).copy()
        eq[(name, "pade")] = e
        r["gap_pade_ha"] = float(e[:, cr.nocc].min() - e[:, cr.nocc - 1].max())
        res[name] = r
        del ch
        torch.cuda.empty_cache()
    diffs = {}
    for name in ("mixed_f32x2", "mixed_f32"):
        for cont in [f"cpe_{x:g}" for x in ridges] + ["pade"]:
            g_m, g_f = res[name][f"gap_{cont}_ha"], res["fp64"][f"gap_{cont}_ha"]
            d = eq[(name, cont)] - eq[("fp64", cont)]
            diffs[f"{name}/{cont}"] = {"gap_err_mev": (g_m - g_f) * HA_MEV,
                                       "max_abs_qp_err_mev": float(np.abs(d).max() * HA_MEV),
                                       "median_abs_qp_err_mev": float(np.median(np.abs(d)) * HA_MEV)}
    out = {"metric": "quasiparticle gap, mixed vs FP64 chain (one G0W0 iteration)", "config": args.gap_config,
           "nq": cr.nq, "omega": args.omega, "vxc": "Sigma^x[G0]", "chains": res, "differences": diffs}
    print(json.dumps(out))
    ctx.close()


def run_mlp(args):
    """The learned CPE seed at its stated scale: ~2e5 band-diagonal Sigma^c(i w) samples from the G0W0
    chains of 48 synthetic crystals shaped like the benchmarked one (Nk = 64, Nb = 64, NI = 256,
    Ntau = 48; seeds apart from it), GPU training (tensor-core forward, backward and Adam), then on two
    held-out crystals of the same shape the QP energies of the seeded CPE fit against the plain CPE
    fit and Pade, with the Lawson-Hanson iterations and the continuation time. A measurement run."""
    import torch

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    from paper_1602_02313_gb300 import learned
    from paper_1602_02313_gb300.driver import Chain
    b.build()
    HA_MEV = 27211.386245988
    mk = lambda s: gi.make_config("nk64_nb64", seed=s)  # noqa: E731
    t0 = time.perf_counter()
    x, A = learned.chain_samples(mk, list(range(9101, 9101 + args.mlp_crystals)), args.omega, qb=64)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = gw.MLP(seed=17)
    t0 = time.perf_counter()
    hist = learned.train(net, x, A, steps=args.mlp_steps, batch=1024, lr=3e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    held = []
    for s in (9301, 9302):
        cr, gr = mk(s)
        ctx = gw.GW(gr, cr, omega=args.omega)
        ch = Chain(ctx, torch.from_numpy(cr.eps).cuda(), prec=gw.GW_FP16X2, qb=64, cont_method=gw.GW_CPE)
        ch.start_g0()
        ch.sigma()
        ch.finish()
        ch.check()
        r = learned.continuation_gain(ctx, net, ch)
        bsol = torch.zeros(cr.nk * cr.nb, len(ch.cpe_x) - 2, dtype=torch.float64, device="cuda")
        ctx.cpe_coeffs(bsol)
        supp = (bsol > 0).sum(1).float()
        ds = np.abs(r["e_seeded"] - r["e_plain"]) * HA_MEV
        dp = np.abs(r["e_pade"] - r["e_plain"]) * HA_MEV
        dsp = np.abs(r["e_seeded"] - r["e_pade"]) * HA_MEV
        gap = lambda e: float((e.reshape(cr.nk, cr.nb)[:, cr.nocc].min()  # noqa: E731
                               - e.reshape(cr.nk, cr.nb)[:, cr.nocc - 1].max()) * HA_MEV)
        held.append({"seed": s, "solution_support_mean": float(supp.mean()),
                     "nnls_iterations_plain_mean": float(r["iters_plain"].mean()),
                     "nnls_iterations_seeded_mean": float(r["iters_seeded"].mean()),
                     "continuation_ms_plain": r["ms_plain"], "continuation_ms_seeded": r["ms_seeded"],
                     "continuation_ms_pade": r["ms_pade"],
                     "qp_seeded_vs_plain_cpe_mev": {"max": float(ds.max()), "median": float(np.median(ds))},
                     "qp_pade_vs_plain_cpe_mev": {"max": float(dp.max()), "median": float(np.median(dp))},
                     "qp_seeded_vs_pade_mev": {"max": float(dsp.max()), "median": float(np.median(dsp))},
                     "gap_mev": {"plain_cpe": gap(r["e_plain"]), "seeded_cpe": gap(r["e_seeded"]),
                                 "pade": gap(r["e_pade"])}})
        ctx.close()
    out = {"metric": "learned CPE seed: training at scale and its gain over the plain continuation",
           "samples": int(x.shape[0]), "crystals": args.mlp_crystals, "data_s": t_data, "train_s": t_train,
           "train_steps": args.mlp_steps, "batch": 1024, "lr": 3e-4, "loss_first": hist[0], "loss_last": hist[-1],
           "loss_history_every_50": hist, "held_out": held}
    print(json.dumps(out))
    net.close()


def run_c3(args):
    """The nk216_nb128 workload as a whole: all 216 q of the Nk = 216 (6x6x6), Nb = 128 (48
    occupied), NI = 512, Ntau = Nnu = Nw = 64, beta = 400 crystal, mixed precision (tensor-core P and
    Sigma^c, float-float screening and bosonic transforms), one G0W0 iteration and args.c3_passes
    self-consistent passes (P, W~ and Sigma from the previous pass's dressed G), CPE continuation.
    Prints one JSON line per pass (time, gap, the change of G) and, first, per-quantity errors of
    this precision at sampled points: P of one q at two tau and Sigma^c of that q at sampled (k, tau)
    (with a Hermitian stand-in for W~(tau)) against the FP64 oracle, and the float-float dielectric
    solve of that q against the FP64 one on the GPU. A measurement run."""
    import torch

    import gwinputs as gi
    import oracle as orc
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300 import build as b
    from paper_1602_02313_gb300.driver import Chain, contraction_flops
    b.build()
    HA_MEV = 27211.386245988
    cr, gr = gi.make_config("nk216_nb128")
    if args.nq > 0:
        cr = gi.subset_q(cr, 0, min(args.nq, cr.nq))
    ctx = gw.GW(gr, cr, omega=args.omega)
    eps = torch.from_numpy(cr.eps).cuda()
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    # ---- per-quantity errors at sampled points, one q
    iq = 7 % cr.nq
    its, ks = [0, 37], [0, 215 % cr.nk]
    G, occ = orc.green_tau0(cr.eps, gr.tau, gr.beta)
    P = torch.zeros((gr.ntau, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
    ctx.polarization(iq, d(G), P, gw.GW_FP16X2)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((gr.ntau, cr.ni, 8)) + 1j * rng.standard_normal((gr.ntau, cr.ni, 8))
    Wst = -30.0 * (X @ np.conj(np.swapaxes(X, 1, 2))) / 8
    S1 = torch.zeros((cr.nk, cr.nb, gr.ntau), dtype=torch.float64, device="cuda")
    ctx.selfenergy(iq, d(G), d(occ), d(Wst), S1, None, gw.GW_FP16X2)
    Piv = torch.zeros((1, gr.nnu, cr.ni, cr.ni), dtype=torch.complex128, device="cuda")
    ctx.tau_to_freq_many(gw.GW_BOSE, gw.GW_TAU_TO_IW, 1, cr.ni * cr.ni, P, Piv, gw.GW_F32X2)
    Wff, W64 = torch.zeros_like(Piv), torch.zeros_like(Piv)
    inf = torch.zeros((1, gr.nnu), dtype=torch.int32, device="cuda")
    ctx.screen(iq, 1, Piv, Wff, inf, gw.GW_F32X2)
    ctx.screen(iq, 1, Piv, W64, inf, gw.GW_FP64)
    ctx.sync()
    t0 = time.perf_counter()
    # the oracle's P of q at the tau indices its_p, its sum over k taken in chunks of 8 k (M of all
    # 216 k would take 29 GB of host memory): each chunk is the oracle's polarization of those k
    # (their G rows first, then all rows for k - q), weighted by chunk size / Nk
    its_p = its[1:]
    Pr = 0.0
    for k0 in range(0, cr.nk, 8):
        kk = list(range(k0, min(cr.nk, k0 + 8)))
        Mk = gi.m_for_q(cr, iq, ks=kk)
        Gx = np.concatenate([G[kk], G])
        Pr = Pr + orc.polarization(Mk, Gx, cr.kmq[iq][kk] + len(kk), omega=args.omega, its=its_p) * (len(kk) / cr.nk)
    Mk = gi.m_for_q(cr, iq, ks=ks)
    Sr, _, _ = orc.selfenergy(Mk, G, Wst, cr.v[iq], cr.kmq[iq], occ, omega=args.omega, ks=ks, its=its)
    t_orc = time.perf_counter() - t0
    rel = lambda a, b_: float(np.abs(a - b_).max() / np.abs(b_).max())  # noqa: E731
    Sg = S1.cpu().numpy()
    errs = {"P_tc_vs_oracle": rel(P.cpu().numpy()[its_p], Pr),
            "Sigma_c_tc_vs_oracle": max(rel(Sg[k][:, its], Sr[k][:, its]) for k in ks),
            "W_f32x2_vs_fp64_gpu": rel(Wff.cpu().numpy(), W64.cpu().numpy()),
            "sample": f"q {iq}; P at tau index {its_p}; Sigma^c at k {ks} x tau {its} with a Hermitian stand-in "
                      f"for W~(tau); the dielectric solve at all {gr.nnu} nu of q {iq}", "oracle_s": t_orc}
    print(json.dumps({"c3": "errors", **errs}), flush=True)
    del P, Piv, Wff, W64, S1
    torch.cuda.empty_cache()
    # ---- the chain
    ch = Chain(ctx, eps, prec=gw.GW_FP16X2, qb=32, cont_method=gw.GW_CPE)
    fp, fs = contraction_flops(cr.nk, cr.nb, cr.ni, gr.ntau)
    flops = (fp + fs) * cr.nq
    st = torch.cuda.current_stream()

    def gap(e):
        e = e.cpu().numpy().reshape(cr.nk, cr.nb)
        return float((e[:, cr.nocc].min() - e[:, cr.nocc - 1].max()) * HA_MEV)

    Gprev = None
    for it in range(args.c3_passes + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        if it == 0:
            ch.step()
        else:
            ch.iterate(1)
        e1.record(st)
        ch.check()
        ms = e0.elapsed_time(e1)
        dG = None if Gprev is None else float((ch.G1 - Gprev).abs().max() / ch.G1.abs().max())
        Gprev = ch.G1.clone()
        print(json.dumps({"c3": "pass", "pass": it, "kind": "G0W0" if it == 0 else "scGW", "ms": ms,
                          "tflops_algorithmic": flops / (ms * 1e-3) / 1e12, "gap_mev": gap(ch.eqp),
                          "max_rel_change_G": dG, "sigx_max_abs_ha": float(ch.Sx.abs().max()),
                          "qp_not_converged": int((ch.qinfo != 0).sum())}), flush=True)
    ctx.close()


def run_dyson_matrix(args):
    """Full-matrix Dyson update (gw_dyson_matrix, FP64) at the nk64_nb64 band and grid sizes: Nk = 64,
    Nb = 64, Ntau = Nw = 48, beta = 200; a Hermitian static part and a Hermitian Sigma^c(tau) made of
    three matrix poles per k. Timed alone against the measured FP64 rate; the oracle on 4 of the 64 k."""
    import torch

    import gwinputs as gi
    import oracle as orc
    import paper_1602_02313_gb300 as gw
    from oracle import offdiag as od
    from paper_1602_02313_gb300 import build as b
    b.build()
    cr, gr = gi.make_config("nk64_nb64", qlist=[0])
    nk, nb, nt, nw = cr.nk, cr.nb, gr.ntau, gr.nw
    ctx = gw.GW(gr, cr, omega=args.omega, m_mode=2)
    rng = np.random.default_rng(2201)

    def herm(s):
        X = rng.standard_normal((nk, nb, nb)) + 1j * rng.standard_normal((nk, nb, nb))
        return s * (X + np.conj(np.swapaxes(X, 1, 2))) / 2

    Sx, vxc = herm(0.2), herm(0.05)
    E = rng.uniform(-1.5, 1.5, 3)
    C = 0.2 * (rng.standard_normal((nk, nb, 3)) + 1j * rng.standard_normal((nk, nb, 3)))
    g0, _ = orc.green_tau0(E[None, :], gr.tau, gr.beta)
    Sc = np.einsum("knp,pt,kmp->knmt", C, g0[0], np.conj(C))
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    eps_d, Sx_d, vxc_d, Sc_d = d(cr.eps), d(Sx), d(vxc), d(Sc)
    G = torch.zeros((nk, nb, nb, nt), dtype=torch.complex128, device="cuda")
    occ = torch.zeros((nk, nb, nb), dtype=torch.complex128, device="cuda")
    info = torch.zeros(nk, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    ctx.set_stream(st)
    for _ in range(args.warmup):
        ctx.dyson_matrix(eps_d, Sx_d, vxc_d, Sc_d, G, occ, info)
    ctx.sync()
    launches0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        ctx.dyson_matrix(eps_d, Sx_d, vxc_d, Sc_d, G, occ, info)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.launch_count() - launches0
    assert int(info.abs().sum()) == 0
    # algorithmic FP64 flops (8 per complex multiply-add): forward map nk nb^2 nw nt, inversion nb^3
    # and matrix tail nb^3 per (k, w), tau maps nk nb^2 (nt + 1) (nb + nw / 2)
    macs = nk * nb * nb * nw * nt + 2.0 * nk * nw * nb ** 3 + nk * nb * nb * (nt + 1) * (nb + nw / 2.0)
    fp64_tf, _ = gw.measure_alu(0)
    ach = 8.0 * macs / (ms * 1e-3) / 1e12
    # the oracle on 4 of the 64 k, scaled to all of them
    ks = [0, 21, 42, 63]
    siw = orc.sigma_tau_to_iw(Sc[ks], gr)
    t0 = time.perf_counter()
    Gr, occr = od.dyson_matrix_iw(cr.eps[ks], Sx[ks], vxc[ks], siw, gr)
    cpu_s = (time.perf_counter() - t0) * nk / len(ks)
    err = max(np.abs(G.cpu().numpy()[ks] - Gr).max() / np.abs(Gr).max(),
              np.abs(occ.cpu().numpy()[ks] - occr).max() / np.abs(occr).max())
    out = {"metric": "full-matrix Dyson update time (Eq. dysonGF as band matrices, i w with exact matrix tail)",
           "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"Nk={nk}, Nb={nb}, Ntau={nt}, Nw={nw}, beta={gr.beta}; Hermitian static part "
                                  f"and three-pole Sigma^c(tau)", "max_rel_err_vs_oracle_4k": err},
           "gpu_launches": int(launches),
           "roofline_alu": {"bound": "alu", "kernel": "gw_dyson_matrix (k_dm_fwd, k_dm_eig, k_dm_inv, k_dm_g0tab, "
                                                      "k_dm_tau)", "achieved": ach, "peak": fp64_tf,
                            "unit": "TFLOP/s FP64", "frac": ach / fp64_tf,
                            "peak_source": "measured FP64 FMA rate of this GPU (gw_measure_alu, this run)"},
           "roofline": None,
           "cpu_baseline": {"value": cpu_s * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"oracle.offdiag.dyson_matrix_iw on {len(ks)} of {nk} k, scaled by {nk // len(ks)}"},
           "e2e": None}
    print(json.dumps(out))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gw", choices=["gw", "reference"])
    ap.add_argument("--prec", default="fp16x2", choices=["fp16x2", "fp64"])
    ap.add_argument("--screen", default="f32x2", choices=["f32x2", "f32"],
                    help="arithmetic of the dielectric solve on the mixed chain: float-float (FP64-grade, the "
                         "default) or plain FP32")
    ap.add_argument("--config", default="nk64_nb64")
    ap.add_argument("--omega", type=float, default=None,
                    help="unit-cell volume in 1/(Omega Nk); default: the paper's Si cell, 270.1 bohr^3")
    ap.add_argument("--nq", type=int, default=0, help="limit q points (profiling / exploration only; not a bench line)")
    ap.add_argument("--nk", type=int, default=0, help="override Nk (profiling small cases only; not a bench line)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cont", default="cpe_mlp", choices=["cpe_mlp", "cpe", "pade"],
                    help="continuation: CPE warm-started by the learned seed (default), plain CPE, or Pade")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--gap-config", default="nk64_nb64", help="crystal of --config gapcheck")
    ap.add_argument("--mlp-crystals", type=int, default=48, help="training crystals of --config mlp")
    ap.add_argument("--c3-passes", type=int, default=8, help="self-consistent passes of --config c3run")
    ap.add_argument("--mlp-steps", type=int, default=4000, help="training steps of --config mlp")
    args = ap.parse_args()
    if args.omega is None:
        import gwinputs as gi
        args.omega = gi.OMEGA_SI
    if args.impl == "reference":
        return run_reference(args, args.config)
    if args.config == "tau_screen":
        return run_tau_screen(args)
    if args.config == "dyson_tau":
        return run_dyson_tau(args)
    if args.config == "offdiag":
        return run_offdiag(args)
    if args.config == "dyson_matrix":
        return run_dyson_matrix(args)
    if args.config == "gapcheck":
        return run_gap_check(args)
    if args.config == "mlp":
        return run_mlp(args)
    if args.config == "c3run":
        return run_c3(args)
    if args.config == "sym":
        import paper_1602_02313_gb300 as gw
        return run_sym(args, gw.PREC[args.prec])

    import torch
    import torch.distributed as dist

    import gwinputs as gi
    import paper_1602_02313_gb300 as gw
    from paper_1602_02313_gb300.driver import Chain, contraction_flops
    from paper_1602_02313_gb300.qsplit import allreduce_sigma, q_range

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1602_02313_gb300 import build as b
    if rank == 0:
        b.build()
    if world > 1:
        dist.barrier()
    prec = gw.PREC[args.prec]
    if args.config == "batch12":
        return run_batch(args, prec)
    full, gr = gi.make_config(args.config, **({"nk": args.nk} if args.nk > 0 else {}))
    nq = full.nq if args.nq <= 0 else min(args.nq, full.nq)
    q0, cnt = q_range(nq, rank, world)
    cr = gi.subset_q(full, q0, max(cnt, 1))
    stream = torch.cuda.current_stream()
    cont = gw.GW_PADE if args.cont == "pade" else gw.GW_CPE
    mlp, mlp_hist = None, None
    if args.cont == "cpe_mlp":
        # learned CPE seed, trained (untimed) on chains of three other crystals
        from paper_1602_02313_gb300 import learned
        mlp, mlp_hist = learned.trained_seed(args.omega, device=local)
    ctx = gw.GW(gr, cr, omega=args.omega, device=local, stream=stream, q0=q0)
    eps = torch.from_numpy(cr.eps).cuda()
    sprec = None if prec == gw.GW_FP64 else {"f32x2": gw.GW_F32X2, "f32": gw.GW_F32}[args.screen]
    chain = Chain(ctx, eps, prec=prec, qb=min(max(cnt, 1), 64), iqs=list(range(cnt)), cont_method=cont, mlp=mlp,
                  screen_prec=sprec)
    fp, fs = contraction_flops(cr.nk, cr.nb, cr.ni, gr.ntau)
    flops_step = (fp + fs) * nq

    def one_step():
        chain.start_g0()
        chain.sigma()
        allreduce_sigma(chain.S, chain.Sx)
        chain.finish()

    for _ in range(args.warmup):
        one_step()
    chain.check()
    # ---------------------------------------------------------------- timed region
    smi_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if "CUDA_VISIBLE_DEVICES" in os.environ else local
    sampler = ClockSampler(smi_index)
    chain.timers = {}
    ctx.kernel_timing(True)  # CUDA events around each tensor-core / screening launch, on the context's stream
    launches0 = ctx.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    torch.cuda.profiler.start()  # a profiler started with --profile-from-start off sees the timed steps only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = ctx.launch_count() - launches0
    chain.check()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = flops_step / (ms * 1e-3) / 1e12
    # per-call timings of the two contractions
    kt = {}
    for key, evs in chain.timers.items():
        d = [a.elapsed_time(b_) for a, b_ in evs]
        kt[key] = float(np.mean(d))
    chain.timers = None
    kern = {}
    for name in ("k_pol_tc", "k_sig_tc", "k_screen_inv"):
        tot, n = ctx.kernel_time(name)
        if n:
            kern[name] = {"launches": n, "total_ms": tot, "avg_ms": tot / n}
    ctx.kernel_timing(False)
    per_launch_flops = {"polarization": fp, "selfenergy": fs, "k_pol_tc": fp, "k_sig_tc": fs}
    # tensor-core MMA flops per algorithmic flop: 3 split products times the cover of P's strips;
    # Sigma runs 4 real GEMMs over the upper triangle of W~, (nkc + 1) / (2 nkc) of the columns,
    # against 4 NI^2 MACs counted
    ni_ = cr.ni
    # P up to NI = 256: E = Re P + Im P in strips of 128 rows over all NI columns (rows padded to
    # 128); above: Re P and Im P over strips of the Hermitian half
    if ni_ <= 256:
        strip_cover = 128 * ((ni_ + 127) // 128) / float(ni_)
    else:
        strip_cover = sum(128 * (ni_ - 128 * i) for i in range((ni_ + 127) // 128)) / (ni_ * ni_ / 2.0)
    nkc_ = ni_ // 32
    mma_factor = {"k_pol_tc": 3.0 * strip_cover, "k_sig_tc": 3.0 * (nkc_ + 1) / (2.0 * nkc_)}
    peaks = _peaks()
    peak = peaks["tensor_sustained"]
    tc = {k: v for k, v in kern.items() if k in ("k_pol_tc", "k_sig_tc")}
    if tc and prec != gw.GW_FP64:
        kname = max(tc, key=lambda k: tc[k]["total_ms"])
        # one call per q and step (a call may hold several launches: P runs its K segments
        # in passes when their partials exceed 8 GiB)
        calls = len(chain.iqs) * args.steps
        achieved = per_launch_flops[kname] * calls / (tc[kname]["total_ms"] * 1e-3) / 1e12
        label = kname + " (CUDA events around each launch)"
    else:
        dom = max(kt, key=lambda k: kt[k]) if kt else "selfenergy"
        kname = dom
        achieved = per_launch_flops[dom] / (kt[dom] * 1e-3) / 1e12 if dom in kt else None
        label = "gw_" + dom + " (whole call)"
    # the screening against the measured rate of the FP32 pipes: NI^3 complex multiply-adds per
    # (q, nu) system (in-place Gauss-Jordan inverse); a float-float complex multiply-add is 48
    # FP32-pipe operations, an FP32 one 4 FMAs
    roof_alu = None
    if "k_screen_inv" in kern and prec != gw.GW_FP64:
        fp64_tf, fp32_tf = gw.measure_alu(local)
        macs = float(cr.ni) ** 3 * len(chain.iqs) * len(gr.nu_idx) * args.steps
        ach = macs / (kern["k_screen_inv"]["total_ms"] * 1e-3) / 1e9
        ops = 48.0 if args.screen == "f32x2" else 4.0
        arith_name = "float-float" if args.screen == "f32x2" else "FP32"
        peak_ff = fp32_tf * 1e3 / (2.0 * ops)  # 2 flops per FP32-pipe operation
        roof_alu = {"bound": "alu", "kernel": f"k_screen_inv<{arith_name}> (CUDA events around each launch)",
                    "achieved": ach, "peak": peak_ff, "unit": f"G complex {arith_name} MAC/s", "frac": ach / peak_ff,
                    "peak_source": f"measured FP32 FMA rate of this GPU (gw_measure_alu, this run) / {ops:.0f} "
                                   f"operations per {arith_name} complex multiply-add",
                    "measured_fp64_tflops": fp64_tf, "measured_fp32_tflops": fp32_tf}
    roof = {"bound": "tensor" if prec != gw.GW_FP64 else "alu", "kernel": label,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": _traffic(kname),
            "peak_source": peaks["source"] + ", sustained bf16/fp16 dense",
            "mma_flops_per_algorithmic_flop": mma_factor.get(kname),
            "kernels": kern, "per_call_ms": kt, "flops_per_launch": {"k_pol_tc": fp, "k_sig_tc": fs}}
    # the same fraction in issued MMA work, and both at the clock this run saw: the sustained
    # peak was measured at the median SM clock of its own loop, a tensor-bound kernel scales with it
    if roof["frac"] is not None and mma_factor.get(kname):
        roof["frac_issued"] = roof["frac"] * mma_factor[kname]
        if peaks.get("sm_mhz") and clocks.get("sm_mhz"):
            r = clocks["sm_mhz"] / float(peaks["sm_mhz"])
            roof["peak_clock_mhz"] = float(peaks["sm_mhz"])
            roof["frac_at_run_clock"] = roof["frac"] / r
            roof["frac_issued_at_run_clock"] = roof["frac_issued"] / r

    # ---------------------------------------------------------------- end to end through the public API
    e2e = None
    if args.e2e_steps > 0:
        eps_h = torch.from_numpy(cr.eps).pin_memory()
        out_h = torch.empty(cr.nk * cr.nb, dtype=torch.float64).pin_memory()
        sx_h = torch.empty(cr.nk * cr.nb, dtype=torch.float64).pin_memory()
        ctx.close()
        del chain
        torch.cuda.empty_cache()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx2 = gw.GW(gr, cr, omega=args.omega, device=local, stream=stream, q0=q0)   # M generated from the seed
            eps_d = eps_h.to("cuda", non_blocking=True)
            ch = Chain(ctx2, eps_d, prec=prec, qb=min(max(cnt, 1), 64), iqs=list(range(cnt)), cont_method=cont, mlp=mlp,
                       screen_prec=sprec)
            ch.start_g0()
            ch.sigma()
            allreduce_sigma(ch.S, ch.Sx)
            ch.finish()
            out_h.copy_(ch.eqp, non_blocking=True)
            sx_h.copy_(ch.Sx.reshape(-1), non_blocking=True)
            torch.cuda.synchronize()
            ctx2.close()
            del ch
        dt = (time.perf_counter() - t0) / args.e2e_steps
        if world > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": flops_step / dt / 1e12, "unit": "TFLOP/s", "ms_per_step": dt * 1e3,
               "h2d_bytes_per_step": int(eps_h.numel() * 8 + cr.v.nbytes + cr.kmq.nbytes + gr.tau.nbytes),
               "d2h_bytes_per_step": int(out_h.numel() * 8 + sx_h.numel() * 8),
               "includes": "gw_create (transform matrices; M generated on the GPU from the seed on a low-priority stream, q by q ahead of its first use), H2D of eps, "
                           "the iteration, D2H of QP energies and Sigma^x, gw_destroy"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        f, t, desc = cpu_sample(full, gr, args.omega)
        cpu = {"value": f / t / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
               "vs_baseline": None, "dtype": _dtype(args),
               "data": "synthetic", "config": _config(args.config, args, args.prec) | {"nq": nq, "nk": cr.nk},
               "gpu_launches": int(launches), "clocks": clocks, "roofline": roof, "roofline_alu": roof_alu, "e2e": e2e,
               "cpu_baseline": cpu}
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
