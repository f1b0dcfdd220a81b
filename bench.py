"""Benchmark of the Laplace-transform AO-direct J/K hot path on GB300.

One step = one Laplace J/K request on the 200-AO chain (10 heavy 3s2p1d + 10 H
2s1p, 35 occupied, 3 transition pairs x 16 Laplace points = 48 non-symmetric
densities, Schwarz 1e-12): Laplace quadrature (host, cached per range), the
pseudo-densities D_q on the device, and J[D_q], K[D_q] with ERIs recomputed on
the fly.  The context (shell pairs, Schwarz factors, work lists) is built once
per geometry and reused, as a resident per-molecule cache.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_05622_gb300 import workloads as W  # noqa: E402

HBM_L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

METRIC = "Laplace J/K builds/s (200-AO chain, 48 densities)"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# Nominal FP64 / FP32 FMA peaks from unit counts and clocks (context only):
# per SM per clock 128 FP32 FMA lanes and 2 FP64 FMA.
def alu_peaks(sm_mhz, nsm=152):
    f = sm_mhz * 1e6
    return {"fp32_tflops": nsm * 128 * 2 * f / 1e12, "fp64_tflops": nsm * 2 * 2 * f / 1e12}


def measure_alu_peaks(ltjk, torch, stream, reps=5):
    """Arithmetic throughput on this GPU (ltjk_alu_peak: independent FMA chains
    over 4 CTAs x 256 threads per SM), best of `reps` launches timed with CUDA
    events, in TFLOP/s: binary32 FMA, binary64 FMA, double-float FMA (2 flops
    each) and the digestion's double-float dot-product accumulation."""
    out = {}
    for kind, name in [(ltjk.ALU_FP32, "fp32_fma"), (ltjk.ALU_FP64, "fp64_fma"),
                       (ltjk.ALU_DFLOAT_FMA, "dfloat_fma"), (ltjk.ALU_DFLOAT_DOT, "dfloat_dot")]:
        ltjk.alu_peak(kind, stream)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = ltjk.alu_peak(kind, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        out[name + "_tflops"] = fl / best / 1e12
    return out


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"ltjk_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, device_index=0):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        rows = [r for r in rows if len(r) >= 9 and r[0] == str(device_index)]
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("LTJK_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_sample(w, budget_s=20.0, nblocks=None):
    """Time the oracle (as it stands) on a bounded sample of the workload: J and K
    blocks of randomly chosen shell pairs for all densities, each block summing
    over every ordered ket (J) or (b,d) (K) shell pair of the full molecule,
    unscreened.  The full build is extrapolated by shell-quartet evaluations."""
    from oracle import oracle as O
    O.build()
    mol = w.mol
    ns = mol.nshells
    nd = w.ndens
    rng = np.random.default_rng(0)
    D = rng.standard_normal((nd, mol.nao, mol.nao))
    t0 = time.perf_counter()
    evals = 0
    done = 0
    while True:
        a, b = int(rng.integers(ns)), int(rng.integers(ns))
        O.j_block(mol, D, a, b)
        O.k_block(mol, D, a, b)
        evals += 2 * ns * ns
        done += 1
        el = time.perf_counter() - t0
        if (nblocks and done >= nblocks) or (not nblocks and el > budget_s):
            break
    el = time.perf_counter() - t0
    rate = evals / el  # shell quartets (with all densities) per second
    unique = ns * (ns + 1) // 2
    unique = unique * (unique + 1) // 2
    build_s = unique / rate
    return {"value": nd / build_s, "unit": "builds/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{done} J+K shell-pair blocks x {nd} densities ({evals} ordered shell "
                      f"quartets in {el:.1f} s), extrapolated to {unique} unique quartets, unscreened",
            "seconds": el, "evals": evals, "blocks": done}


def bench_config(w, precision):
    """The workload description both arms print."""
    return {"workload": w.name, "precision": precision, "schwarz_tau": w.schwarz_tau,
            "mixed_tau": 1e-6 if precision == "mixed" else None, "nao": w.mol.nao, "ndens": w.ndens,
            "laplace_points": w.nlap, "l2": "flushed between timed steps (512 MB write)"}


def run_reference(args, world, rank):
    """The oracle as it stands, on the host cores: each step is a time-bounded
    sample of the same workload (J and K blocks of random shell pairs,
    extrapolated to the whole unscreened build); the value is the mean rate
    over the timed steps."""
    if rank != 0:
        return
    w = W.config2()
    times, rates, evals, blocks = [], [], 0, 0
    cores = None
    for step in range(args.warmup + args.steps):
        timed = step >= args.warmup
        r = cpu_oracle_sample(w, budget_s=args.ref_seconds if timed else 1.0)
        cores = r["cores"]
        if timed:
            times.append(r["seconds"])
            rates.append(r["value"])
            evals += r["evals"]
            blocks += r["blocks"]
    val = statistics.mean(rates)
    cfg = bench_config(w, args.precision)
    cfg["parallelism"] = "host cores (oracle)"
    line = {"impl": "reference", "metric": METRIC,
            "value": val, "unit": "builds/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": "builds/s", "cores": cores, "kind": "oracle",
                             "sample": f"{blocks} J+K shell-pair blocks x {w.ndens} densities over "
                                       f"{args.steps} steps of ~{args.ref_seconds:.0f} s ({evals} ordered "
                                       f"shell quartets), extrapolated to the unscreened build; the oracle "
                                       f"computes in FP64"},
            "e2e": {"value": val, "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU path
def _event_ms(torch, stream, fn, reps):
    """Mean device time of fn() over reps calls, CUDA events on `stream`."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def mixed_peak(parts):
    """Harmonic mix of peaks weighted by flop share: parts = [(flops, peak), ...];
    the time-weighted peak of a path whose flops split over several units."""
    tot = sum(f for f, _ in parts)
    t = sum(f / p for f, p in parts if f > 0)
    return tot / t if t > 0 else None


def measure_gradient(ltjk, torch, dev, local, stream, prec, peaks, reps=3):
    """ERI-derivative contraction (Eq. jkderiv) on the 200-AO chain geometry with
    16 separable symmetric terms: gradients/s, quartets/s, the error against an
    IEEE FP64 gradient on the same GPU, and its roofline: algorithmic flops per
    gradient = the derivative-recurrence flop model + per kept Cartesian
    integral 2R (Gamma formation, R terms) + 18 (nine derivative components),
    against the measured peaks of the units they run on (derivative
    recurrences double-float, or binary32 in mixed mode; Gamma and the
    contraction binary64)."""
    wl = W.config4()
    ctx = ltjk.Context(wl.mol, schwarz_tau=wl.schwarz_tau, mixed_tau=1e-6, precision=prec, device=local)
    P = torch.from_numpy(wl.P).to(dev)
    Q = torch.from_numpy(wl.Q).to(dev)
    g = torch.empty((wl.mol.natoms, 3), dtype=torch.float64, device=dev)
    ctx.jk_grad(P, Q, wl.cJ, wl.cK, grad=g)
    ms = _event_ms(torch, stream, lambda: ctx.jk_grad(P, Q, wl.cJ, wl.cK, grad=g), reps)
    c64 = ltjk.Context(wl.mol, schwarz_tau=wl.schwarz_tau, precision=ltjk.FP64_NATIVE, device=local)
    g64 = c64.jk_grad(P, Q, wl.cJ, wl.cK)
    torch.cuda.synchronize()
    gmax = float(g64.abs().max())
    err = float((g - g64).abs().max())
    st = ctx.stats()
    R = int(P.shape[0])
    f_gamma = st["cart_integrals_kept"] * (2.0 * R + 18.0)
    f_d64 = st["grad_eri_flops_fp64"]
    f_d32 = st["grad_eri_flops"] - f_d64
    if prec == ltjk.FP64_NATIVE:
        parts = [(f_d64 + f_d32, peaks["fp64_fma_tflops"]), (f_gamma, peaks["fp64_fma_tflops"])]
    else:
        parts = [(f_d64, peaks["dfloat_fma_tflops"]), (f_d32, peaks["fp32_fma_tflops"]),
                 (f_gamma, peaks["fp64_fma_tflops"])]
    flops = f_gamma + f_d64 + f_d32
    peak = mixed_peak(parts)
    ach = flops / (ms / 1e3) / 1e12
    return {"workload": wl.name, "terms": R, "cJ": wl.cJ, "cK": wl.cK,
            "grad_ms": ms, "gradients_per_s": 1e3 / ms,
            "quartets_per_s": st["quartets_kept"] / (ms / 1e3),
            "max_abs_vs_fp64": err, "rel_to_max_vs_fp64": err / gmax,
            "sum_over_atoms_rel": float(g.sum(0).abs().max()) / gmax,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "algorithmic_flops": flops,
                         "flops_split": {"derivative_recurrences_fp64_class": f_d64,
                                         "derivative_recurrences_fp32": f_d32,
                                         "gamma_and_contraction_binary64": f_gamma},
                         "peak_source": "harmonic mix by flop share of the peaks measured in this run"}}


def measure_config1(ltjk, torch, dev, local, stream, reps=20):
    """The plain-FP64 single request of the 25-AO water-like molecule (8
    pseudo-densities): builds/s in IEEE FP64 and FP64 class, and their
    difference (relative to max)."""
    w = W.config1()
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    t, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
    out = {"workload": w.name, "nao": w.mol.nao, "ndens": w.ndens, "schwarz_tau": w.schwarz_tau}
    res = {}
    for name, prec in [("fp64_native", ltjk.FP64_NATIVE), ("fp64_class", ltjk.FP64)]:
        ctx = ltjk.Context(w.mol, schwarz_tau=w.schwarz_tau, precision=prec, device=local)
        D = ctx.pseudo_densities(torch.from_numpy(w.C_occ).to(dev), torch.from_numpy(w.C_vir).to(dev),
                                 torch.from_numpy(w.eps_occ).to(dev), torch.from_numpy(w.eps_vir).to(dev),
                                 torch.from_numpy(np.ascontiguousarray(w.X)).to(dev), t)
        J, K = ctx.jk_build(D)
        times = []
        for _ in range(reps):
            times.append(_event_ms(torch, stream, lambda: ctx.jk_build(D, J, K), 1))
        ms = statistics.median(times)
        res[name] = (J, K)
        out[name] = {"build_ms": ms, "builds_per_s": w.ndens / (ms / 1e3), "quartets_kept": ctx.stats()["quartets_kept"]}
    (J1, K1), (J2, K2) = res["fp64_native"], res["fp64_class"]
    out["fp64_class_vs_native"] = {"J_max_rel_to_max": float((J2 - J1).abs().max() / J1.abs().max()),
                                   "K_max_rel_to_max": float((K2 - K1).abs().max() / K1.abs().max())}
    return out


def measure_serving(ltjk, torch, dev, nreq=32, nao_hi=300):
    """A short stream of the serving workload's shape (chain molecules with
    AO counts log-uniform from 25 up to nao_hi, 8-16 Laplace points, 70 % J/K
    and 30 % gradients, mixed precision, 150 GB budget) through the
    continuous-batching service: p50/p99 latency at 0.8 of the measured
    capacity, and the saturated throughput (every request at t = 0), each
    against sequential plain FP64 on the same request list."""
    import serving_bench as SB
    paced = SB.run_stream(ltjk, torch, dev, nreq=nreq, nao_hi=nao_hi, load=0.8)
    sat = SB.run_stream(ltjk, torch, dev, nreq=nreq, nao_hi=nao_hi, saturated=True)
    return {"paced": paced, "saturated": sat}


def measure_macrocycle(ltjk, torch, dev, local, stream, reps=2):
    """Mixed-precision J/K of 128 pseudo-densities on the 445-AO macrocycle
    (FP64 for quartets with Q_ab Q_cd > 1e-6): builds/s and the per-element
    error against the FP64-class build on the same GPU (itself parity-tested
    against the oracle)."""
    w = W.config3()
    mol = w.mol
    t0 = time.perf_counter()
    cm = ltjk.Context(mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=ltjk.MIXED, device=local)
    setup_s = time.perf_counter() - t0
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    tq, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
    D = cm.pseudo_densities(torch.from_numpy(w.C_occ).to(dev), torch.from_numpy(w.C_vir).to(dev),
                            torch.from_numpy(w.eps_occ).to(dev), torch.from_numpy(w.eps_vir).to(dev),
                            torch.from_numpy(np.ascontiguousarray(w.X)).to(dev), tq)
    J, K = cm.jk_build(D)
    ms = _event_ms(torch, stream, lambda: cm.jk_build(D, J, K), reps)
    c64 = ltjk.Context(mol, schwarz_tau=w.schwarz_tau, precision=ltjk.FP64, device=local)
    J64, K64 = c64.jk_build(D)
    ms64 = _event_ms(torch, stream, lambda: c64.jk_build(D, J64, K64), 1)
    dj = float((J - J64).abs().max())
    dk = float((K - K64).abs().max())
    st = cm.stats()
    out = {"workload": w.name, "nao": mol.nao, "ndens": int(D.shape[0]), "precision": "mixed",
           "mixed_tau": 1e-6, "build_ms": ms, "builds_per_s": D.shape[0] / (ms / 1e3),
           "fp64_class_builds_per_s": D.shape[0] / (ms64 / 1e3),
           "quartets_kept": st["quartets_kept"], "quartets_fp64": st["quartets_fp64"],
           "quartets_per_s": st["quartets_kept"] / (ms / 1e3), "setup_ms": 1e3 * setup_s,
           "error_vs_fp64_class": {"J_max_abs": dj, "K_max_abs": dk,
                                   "J_max_rel_to_max": dj / float(J64.abs().max()),
                                   "K_max_rel_to_max": dk / float(K64.abs().max())}}
    del cm, c64, D, J, K, J64, K64
    return out


def measure_fshell(ltjk, torch, dev, local, stream, reps=3):
    """J/K of 48 pseudo-densities on the 200-AO f-shell chain (4 heavy atoms
    4s3p2d1f, 4 H 3s2p1d; every class up to (ff|ff)): builds/s in the FP64
    class, mixed and IEEE FP64 modes, and the FP64-class and mixed error
    against the IEEE FP64 build on the same GPU (all three parity-tested
    against the oracle on the smaller f-shell molecules)."""
    w = W.config_fshell()
    mol = w.mol
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    tq, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
    out = {"workload": w.name, "nao": mol.nao, "ndens": w.ndens}
    res = {}
    for name, prec, r in (("fp64_class", ltjk.FP64, reps), ("mixed", ltjk.MIXED, reps),
                          ("fp64_native", ltjk.FP64_NATIVE, 1)):
        t0 = time.perf_counter()
        c = ltjk.Context(mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=prec, device=local)
        setup_s = time.perf_counter() - t0
        D = c.pseudo_densities(torch.from_numpy(w.C_occ).to(dev), torch.from_numpy(w.C_vir).to(dev),
                               torch.from_numpy(w.eps_occ).to(dev), torch.from_numpy(w.eps_vir).to(dev),
                               torch.from_numpy(np.ascontiguousarray(w.X)).to(dev), tq)
        J, K = c.jk_build(D)
        ms = _event_ms(torch, stream, lambda: c.jk_build(D, J, K), r)
        st = c.stats()
        out[name] = {"build_ms": ms, "builds_per_s": w.ndens / (ms / 1e3), "setup_ms": 1e3 * setup_s,
                     "quartets_kept": st["quartets_kept"], "quartets_fp64": st["quartets_fp64"],
                     "quartets_per_s": st["quartets_kept"] / (ms / 1e3)}
        res[name] = (J, K)
        del c, D
    J64, K64 = res["fp64_native"]
    for name in ("fp64_class", "mixed"):
        J, K = res[name]
        out[name]["error_vs_fp64"] = {"J_max_rel_to_max": float((J - J64).abs().max() / J64.abs().max()),
                                      "K_max_rel_to_max": float((K - K64).abs().max() / K64.abs().max())}
    del res, J64, K64
    return out


def measure_next_rows(ltjk, torch, stream, ctx, w, J, K, Co, Cv, xmin, xmax, peaks, reps=5):
    """The rows either side of the build: the Laplace-Fock back-transform of the
    48 J/K pairs to the occupied-virtual block (Eq. laplacefock; FP64 GEMMs on
    the FP64 pipe) and the host-side minimax grid (Eq. laplace, Remez)."""
    nd, N = J.shape[0], J.shape[1]
    no, nv = Co.shape[1], Cv.shape[1]
    F = torch.empty((nd, no, nv), dtype=torch.float64, device=J.device)
    ctx.laplace_fock(J, K, Co, Cv, 2.0, -1.0, F=F)
    ms = _event_ms(torch, stream, lambda: ctx.laplace_fock(J, K, Co, Cv, 2.0, -1.0, F=F), reps)
    flops = nd * (3.0 * N * N + 2.0 * N * N * nv + 2.0 * N * no * nv)
    peak = peaks["fp64_fma_tflops"]
    t0 = time.perf_counter()
    tm, wm, em, conv = ltjk.laplace_minimax(xmin, xmax, w.nlap)
    mm_ms = 1e3 * (time.perf_counter() - t0)
    _, _, els = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
    return {"laplace_fock": {"densities": nd, "ms": ms, "tflops": flops / (ms / 1e3) / 1e12,
                             "fp64_pipe_frac": flops / (ms / 1e3) / 1e12 / peak,
                             "algorithmic_flops": flops},
            "laplace_minimax": {"points": w.nlap, "host_ms": mm_ms, "max_rel_err": em,
                                "converged": conv, "least_squares_max_rel_err": els}}


def measure_cd(ltjk, torch, stream, ctx, w, D, J, K, Co, Cv, eo, ev, X, t, peaks, delta=1e-9, reps=2):
    """The Cholesky-factorised route on the same request (Eqs. cdfact, cdj,
    cdknonsym): factor set-up time and vectors, the J/K of the 48 pseudo-densities
    from their rank-nocc factors, FP64 pipe fraction, and the difference from the
    direct build (bounded by the residual diagonal times sum|D|)."""
    N = ctx.nao
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B, naux, res = ctx.cd_factor(delta, 20 * N)
    torch.cuda.synchronize()
    factor_s = time.perf_counter() - t0
    U, V = ctx.pseudo_density_factors(Co, Cv, eo, ev, X, t)
    U = U[:1].contiguous()  # C_occ: one left factor for every pseudo-density
    Jc, Kc = ctx.cd_jk(B, U, V)
    ms = _event_ms(torch, stream, lambda: ctx.cd_jk(B, U, V, J=Jc, K=Kc), reps)
    nd, r = V.shape[0], V.shape[2]
    # B U once; per density B V_q, sum_Q (B_Q U)(B_Q V_q)^T, gamma and J
    flops = 2.0 * naux * N * N * r + nd * (4.0 * naux * N * N * r + 2.0 * naux * N * r + 2.0 * naux * N * N)
    native = ctx.precision == ltjk.FP64_NATIVE
    peak = peaks["fp64_fma_tflops"] if native else peaks["dfloat_fma_tflops"]
    dj = float((Jc - J).abs().max())
    dk = float((Kc - K).abs().max())
    bound = res * float(D.abs().sum(dim=(1, 2)).max())
    out = {"delta": delta, "naux": naux, "max_residual": res, "factor_s": factor_s,
           "jk_ms": ms, "builds_per_s": nd / (ms / 1e3), "rank": r,
           "tflops": flops / (ms / 1e3) / 1e12, "peak_tflops": peak, "frac": flops / (ms / 1e3) / 1e12 / peak,
           "arithmetic": "IEEE FP64" if native else "double-float GEMMs on the FP32 pipe",
           "vs_direct": {"J_max_abs": dj, "K_max_abs": dk, "bound_res_x_sum_abs_D": bound,
                         "J_max_rel_to_max": dj / float(J.abs().max()),
                         "K_max_rel_to_max": dk / float(K.abs().max())}}
    del B, U, V, Jc, Kc
    return out


def run_gpu(args, world, rank, local):
    import torch
    from paper_2607_05622_gb300 import ltjk
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w = W.config2()
    mol = w.mol
    N, nd = mol.nao, w.ndens
    prec = {"mixed": ltjk.MIXED, "fp64": ltjk.FP64, "fp64-native": ltjk.FP64_NATIVE}[args.precision]
    t0 = time.perf_counter()
    ctx = ltjk.Context(mol, schwarz_tau=w.schwarz_tau, mixed_tau=1e-6, precision=prec, device=local)
    setup_s = time.perf_counter() - t0
    st = ctx.stats()
    xmin = 2.0 * (w.eps_vir.min() - w.eps_occ.max())
    xmax = 2.0 * (w.eps_vir.max() - w.eps_occ.min())
    tq, wq, lap_err = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
    Co, Cv = torch.from_numpy(w.C_occ).to(dev), torch.from_numpy(w.C_vir).to(dev)
    eo, ev = torch.from_numpy(w.eps_occ).to(dev), torch.from_numpy(w.eps_vir).to(dev)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).to(dev)
    D = torch.empty((nd, N, N), dtype=torch.float64, device=dev)
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    flush = torch.empty(HBM_L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        t, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
        ctx.pseudo_densities(Co, Cv, eo, ev, X, t, D=D)
        ctx.jk_build(D, J, K)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # device-timed steps, L2 flushed between steps (outside the timed events)
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    l0 = ltjk.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with Clocks() as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev_s[i].record(stream)
            t, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
            ctx.pseudo_densities(Co, Cv, eo, ev, X, t, D=D)
            ev_k0[i].record(stream)
            ctx.jk_build(D, J, K)
            ev_e[i].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = ltjk.launch_count() - l0
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(args.steps)]
    jk_ms = [ev_k0[i].elapsed_time(ev_e[i]) for i in range(args.steps)]
    total_s = reduce_max(sum(step_ms) / 1e3, world)
    value = world * nd * args.steps / total_s
    # end to end: pinned host inputs -> device -> D -> J, K -> pinned host outputs
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hC, hV, he, hv, hX = pin(w.C_occ), pin(w.C_vir), pin(w.eps_occ), pin(w.eps_vir), pin(w.X)
    hJ = torch.empty((nd, N, N), dtype=torch.float64).pin_memory()
    hK = torch.empty((nd, N, N), dtype=torch.float64).pin_memory()  # (empty_like would not pin)
    h2d = sum(x.numel() * 8 for x in (hC, hV, he, hv, hX))
    d2h = 2 * nd * N * N * 8

    def e2e_step():
        t, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
        dC, dV = hC.to(dev, non_blocking=True), hV.to(dev, non_blocking=True)
        de, dv, dX = he.to(dev, non_blocking=True), hv.to(dev, non_blocking=True), hX.to(dev, non_blocking=True)
        Dd = ctx.pseudo_densities(dC, dV, de, dv, dX, t)
        Jd, Kd = ctx.jk_build(Dd)
        hJ.copy_(Jd, non_blocking=True)
        hK.copy_(Kd, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e_s, e_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ne = max(2, min(args.steps, 5))
    barrier(world)
    torch.cuda.synchronize()
    e_s.record(stream)
    for _ in range(ne):
        e2e_step()
    e_e.record(stream)
    torch.cuda.synchronize()
    e2e_s = reduce_max(e_s.elapsed_time(e_e) / 1e3, world)
    e2e_val = world * nd * ne / e2e_s
    # error of this precision against a plain FP64 build on the same GPU
    err = {}
    if prec != ltjk.FP64_NATIVE:
        c64 = ltjk.Context(mol, schwarz_tau=w.schwarz_tau, precision=ltjk.FP64_NATIVE, device=local)
        J64, K64 = c64.jk_build(D)
        torch.cuda.synchronize()
        e64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e64[0].record(stream)
        c64.jk_build(D, J64, K64)
        e64[1].record(stream)
        torch.cuda.synchronize()
        fp64_ms = e64[0].elapsed_time(e64[1])
        dj = (J - J64).abs().max().item()
        dk = (K - K64).abs().max().item()
        err = {"vs": "IEEE FP64 build on the same GPU (itself parity-tested against the oracle)",
               "J_max_abs": dj, "K_max_abs": dk,
               "J_max_rel_to_max": dj / J64.abs().max().item(), "K_max_rel_to_max": dk / K64.abs().max().item(),
               "fp64_single_request_builds_per_s": nd / (fp64_ms / 1e3)}
        del c64
    # roofline of the dominant kernel (the J/K quartet kernels of one build,
    # 21 class launches, > 99 % of the step), against arithmetic peaks
    # measured on this GPU in this run
    clocks = clk.summary(local)
    peaks = measure_alu_peaks(ltjk, torch, stream)
    jk_s = statistics.mean(jk_ms) / 1e3
    dig = 20.0 * st["cart_integrals_kept"] * nd
    dig64 = 20.0 * st["cart_integrals_fp64"] * nd
    eri, eri64 = st["eri_flops_per_build"], st["eri_flops_fp64"]
    flops = eri + dig
    if prec == ltjk.FP64_NATIVE:
        parts = [(flops, peaks["fp64_fma_tflops"])]
        pipe = "fp64 FMA pipe (IEEE binary64 throughout)"
    else:
        parts = [(eri64, peaks["dfloat_fma_tflops"]), (dig64, peaks["dfloat_dot_tflops"]),
                 (eri - eri64, peaks["fp32_fma_tflops"]), (dig - dig64, peaks["fp32_fma_tflops"])]
        pipe = (f"fp32 pipe: {100 * (eri64 + dig64) / flops:.0f}% of the flops double-float "
                f"(recurrences as FMAs, digestion as dot-product accumulation), the rest binary32")
    peak = mixed_peak(parts)
    roof = {"bound": "alu", "pipe": pipe,
            "achieved": flops / jk_s / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": flops / jk_s / 1e12 / peak, "traffic": None,
            "traffic_note": ("not captured for this kernel version: the working set (density copies and "
                             "accumulators, 56 nd N^2 bytes = 108 MB here) is L2-resident, so DRAM counts "
                             "only first-touch traffic of an arithmetic-bound path"),
            "algorithmic_bytes_per_build": 3 * nd * N * N * 8,
            "algorithmic_flops_per_build": flops,
            "flops_split": {"eri_fp64_class": eri64, "digestion_fp64_class": dig64,
                            "eri_fp32": eri - eri64, "digestion_fp32": dig - dig64},
            "peak_source": ("harmonic mix by flop share of arithmetic peaks measured in this run "
                            "(ltjk_alu_peak, CUDA events, best of 5); of measured"),
            "measured_peaks_tflops": peaks,
            "nominal_peaks_tflops": alu_peaks(2070.0, torch.cuda.get_device_properties(local).multi_processor_count)}
    extras = {}
    legs = set() if args.no_extras else set(args.legs.split(","))
    if rank == 0:
        if "next_rows" in legs:
            extras["next_rows"] = measure_next_rows(ltjk, torch, stream, ctx, w, J, K, Co, Cv, xmin, xmax, peaks)
            tq, _, _ = ltjk.laplace_quadrature(xmin, xmax, w.nlap)
            extras["next_rows"]["cholesky_jk"] = measure_cd(ltjk, torch, stream, ctx, w, D, J, K, Co, Cv, eo, ev,
                                                            X, tq, peaks)
        if "gradient" in legs:
            extras["gradient"] = measure_gradient(ltjk, torch, dev, local, stream, prec, peaks)
        if "macrocycle" in legs:
            extras["macrocycle_445"] = measure_macrocycle(ltjk, torch, dev, local, stream)
        if "water" in legs:
            extras["water_fp64_single_request"] = measure_config1(ltjk, torch, dev, local, stream)
        if "fshell" in legs:
            extras["fshell_chain_200"] = measure_fshell(ltjk, torch, dev, local, stream)
        if "serving" in legs:
            extras["serving"] = measure_serving(ltjk, torch, dev)
            pc = extras["serving"]["paced"]
            extras["latency"] = {"p50_ms": pc["p50_ms"], "p99_ms": pc["p99_ms"],
                                 "what": "serving stream, 0.8 x capacity, mixed precision (see serving.paced)"}
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_sample(w, budget_s=args.cpu_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    cfg = bench_config(w, args.precision)
    cfg.update({"laplace_max_rel_err": lap_err, "parallelism": f"replicas x{world}"})
    line = {
        "metric": METRIC,
        "value": value, "unit": "builds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {ltjk.FP64_NATIVE: "f64", ltjk.FP64: "f64-class (f32 pairs + f64)",
                  ltjk.MIXED: "f32 + f64-class"}[prec],
        "data": "synthetic",
        "config": cfg,
        "quartets_per_s": world * st["quartets_kept"] * args.steps / total_s,
        "prim_quartets_per_s": world * st["prim_quartets_kept"] * args.steps / total_s,
        "jk_build_ms": statistics.mean(jk_ms),
        "setup_ms": 1e3 * setup_s,
        "work": {k: st[k] for k in ("quartets_total", "quartets_kept", "quartets_fp64",
                                    "prim_quartets_kept", "cart_integrals_kept", "eri_flops_per_build")},
        "error_vs_fp64": err or None,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "builds/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extras)
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp64-native"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-seconds", type=float, default=4.0,
                    help="oracle seconds per timed step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="next_rows,gradient,macrocycle,water,fshell,serving",
                    help="comma-separated measurements beside the headline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements beside the headline (gradient, 445-AO macrocycle, "
                         "next rows, 25-AO FP64 request, 200-AO f-shell chain, serving stream)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
