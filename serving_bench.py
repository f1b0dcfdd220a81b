"""Serving benchmark: a Poisson stream of J/K and gradient requests on one GB300.

Request stream (paper_2607_05622_gb300.workloads.serving_requests): chain
molecules with AO counts log-uniform in [25, 730], 8-16 Laplace points, 1-3
transition pairs, 70 % J/K builds and 30 % gradients (8 terms), mixed
precision, admitted under a 150 GB HBM budget by the continuous-batching
service.  Reported against the same request list run one at a time in plain
IEEE FP64 on the same GPU:

  1. sequential FP64 pass: per request, context + pseudo-densities + build,
     service time, and 4096 sampled result elements kept as the reference;
  2. mixed-precision single-request pass (service time only) to measure the
     capacity; the arrival rate is set to 0.8 x that capacity;
  3. the stream replayed in real time into the service by a pool of frontend
     threads that build each request's context and densities on arrival;
     latency = completion time - arrival time (context creation and density
     formation included); with --saturated every request arrives at once, so
     the throughput is the service's capacity.

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_05622_gb300 import workloads as W  # noqa: E402


def prepare(L, req, precision, dev, torch):
    """Context and device inputs of one request (timed as part of its service)."""
    inp = W.request_inputs(req)
    mol = req["mol"]
    ctx = L.Context(mol, schwarz_tau=1e-12, mixed_tau=1e-6, precision=precision)
    if req["kind"] == "jk":
        xmin = 2.0 * (inp["eps_vir"].min() - inp["eps_occ"].max())
        xmax = 2.0 * (inp["eps_vir"].max() - inp["eps_occ"].min())
        t, _, _ = L.laplace_quadrature(xmin, xmax, req["nlap"])
        C = inp["C"]
        Co = torch.from_numpy(np.ascontiguousarray(C[:, :inp["nocc"]])).to(dev)
        Cv = torch.from_numpy(np.ascontiguousarray(C[:, inp["nocc"]:])).to(dev)
        D = ctx.pseudo_densities(Co, Cv, torch.from_numpy(inp["eps_occ"]).to(dev),
                                 torch.from_numpy(inp["eps_vir"]).to(dev),
                                 torch.from_numpy(np.ascontiguousarray(inp["X"])).to(dev), t)
        return ctx, {"D": D}
    P = torch.from_numpy(inp["P"]).to(dev)
    Q = torch.from_numpy(inp["Q"]).to(dev)
    return ctx, {"P": P, "Q": Q}


def sample_index(n, k, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=min(k, n))


def run_stream(L, torch, dev, nreq=256, nao_hi=730, budget_gb=150.0, load=0.8, frontend_threads=4,
               seed=5, saturated=False):
    """The three passes above on one request list; returns the result dict.
    saturated: every request arrives at time 0 (offered load above capacity),
    so the throughput measured is the service's capacity, not the arrival rate."""
    reqs = W.serving_requests(nreq, seed=seed, nao_hi=nao_hi, rate_hz=1.0)
    # untimed warm-up over the whole list: load every kernel and table the
    # passes below use (first launches would otherwise land in pass 1)
    for prec in (L.FP64_NATIVE, L.MIXED):
        for r in reqs:
            ctx, inp = prepare(L, r, prec, dev, torch)
            if r["kind"] == "jk":
                ctx.jk_build(inp["D"])
            else:
                ctx.jk_grad(inp["P"], inp["Q"], 1.0, 0.0)
            torch.cuda.synchronize()
            ctx.close()
    ref = []
    seq_fp64 = []
    # 1. sequential plain FP64
    for r in reqs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx, inp = prepare(L, r, L.FP64_NATIVE, dev, torch)
        if r["kind"] == "jk":
            J, K = ctx.jk_build(inp["D"])
            torch.cuda.synchronize()
            idx = sample_index(J.numel(), 4096, r["seed"])
            ref.append((J.flatten()[idx].cpu().numpy(), K.flatten()[idx].cpu().numpy(),
                        float(J.abs().max()), float(K.abs().max()), idx))
        else:
            g = ctx.jk_grad(inp["P"], inp["Q"], 1.0, 0.0)
            torch.cuda.synchronize()
            ref.append((g.cpu().numpy(),))
        seq_fp64.append(time.perf_counter() - t0)
        ctx.close()
        del inp
    # 2. mixed single-request service times (capacity)
    seq_mixed = []
    for r in reqs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx, inp = prepare(L, r, L.MIXED, dev, torch)
        if r["kind"] == "jk":
            ctx.jk_build(inp["D"])
        else:
            ctx.jk_grad(inp["P"], inp["Q"], 1.0, 0.0)
        torch.cuda.synchronize()
        seq_mixed.append(time.perf_counter() - t0)
        ctx.close()
        del inp
    capacity = len(reqs) / sum(seq_mixed)
    rate = load * capacity
    # arrival times rescaled to the chosen rate (same Poisson draws)
    base = np.array([r["arrival"] for r in reqs])
    arrivals = np.zeros(len(reqs)) if saturated else base * (1.0 / rate) / (base[-1] / len(reqs))
    # 3. served stream: a pool of host threads (a serving frontend) builds each
    # request's context and densities when it arrives and submits it; the main
    # thread collects completions.  Latency = completion - arrival.
    import concurrent.futures as cf
    import threading
    svc = L.Service(int(budget_gb * (1 << 30)))
    pending = {}
    lock = threading.Lock()
    lat, slow, errs_j, errs_k, errs_g, per_req = [], [], [], [], [], []
    t_sub = {}
    t_start = time.perf_counter()

    def arrive(i):
        dt = arrivals[i] - (time.perf_counter() - t_start)
        if dt > 0:
            time.sleep(dt)
        r = reqs[i]
        s_ = torch.cuda.Stream(priority=-1)  # the frontend's work ahead of queued bulk steps
        with torch.cuda.stream(s_):
            ctx, inp = prepare(L, r, L.MIXED, dev, torch)
            if r["kind"] == "jk":
                tk, J, K = svc.submit_jk(ctx, inp["D"])
                out = (J, K)
            else:
                tk, g = svc.submit_grad(ctx, inp["P"], inp["Q"], 1.0, 0.0)
                out = (g,)
        with lock:
            pending[tk] = (i, ctx, inp, out, arrivals[i])
            t_sub[i] = time.perf_counter() - t_start

    done_list = []

    def harvest():
        # completion times only: the checks against the FP64 results (device
        # gathers and copies that would queue behind the running work and
        # delay the next timestamps) run after the stream
        with lock:
            items = list(pending.items())
        for tk, (i, ctx, inp, out, t_arr) in items:
            done, rc = svc.poll(tk)
            if not done:
                continue
            t_done = time.perf_counter() - t_start
            L._check(rc)
            lat.append(t_done - t_arr)
            slow.append((t_done - t_arr) / seq_mixed[i])
            per_req.append((slow[-1], i, t_arr, t_done))
            done_list.append((i, ctx, out))
            with lock:
                del pending[tk]

    with cf.ThreadPoolExecutor(max_workers=frontend_threads) as pool:
        futs = [pool.submit(arrive, i) for i in range(len(reqs))]
        while len(lat) < len(reqs):
            harvest()
            for f in futs:
                if f.done() and f.exception():
                    raise f.exception()
            time.sleep(0.001)
    span = time.perf_counter() - t_start
    st = svc.stats()
    svc.close()
    torch.cuda.synchronize()
    for i, ctx, out in done_list:
        if reqs[i]["kind"] == "jk":
            J, K = out
            rj, rk, mj, mk, idx = ref[i]
            errs_j.append(float(np.abs(J.flatten()[idx].cpu().numpy() - rj).max()) / mj)
            errs_k.append(float(np.abs(K.flatten()[idx].cpu().numpy() - rk).max()) / mk)
        else:
            g = out[0].cpu().numpy()
            errs_g.append(float(np.abs(g - ref[i][0]).max() / np.abs(ref[i][0]).max()))
        ctx.close()
    lat_ms = sorted(1e3 * x for x in lat)
    pct = lambda p: lat_ms[min(len(lat_ms) - 1, int(round(p * (len(lat_ms) - 1))))]  # noqa: E731
    slow_s = sorted(slow)
    spct = lambda p: slow_s[min(len(slow_s) - 1, int(round(p * (len(slow_s) - 1))))]  # noqa: E731
    nao = [r["mol"].nao for r in reqs]
    return {
        "metric": "serving: p50/p99 latency and throughput, mixed precision, continuous batching",
        "requests": len(reqs), "jk": sum(r["kind"] == "jk" for r in reqs),
        "grad": sum(r["kind"] == "grad" for r in reqs),
        "nao_min": min(nao), "nao_median": int(np.median(nao)), "nao_max": max(nao),
        "arrivals": "all at t = 0 (saturated)" if saturated else f"Poisson at {load} x capacity",
        "arrival_rate_hz": None if saturated else rate, "offered_load": None if saturated else load,
        "p50_ms": pct(0.5), "p99_ms": pct(0.99), "mean_ms": statistics.mean(lat_ms),
        "slowdown_p50": spct(0.5), "slowdown_p99": spct(0.99),
        "slowdown_what": "latency / the request's stand-alone mixed service time (same list, one at a time)",
        "worst_slowdowns": [{"nao": reqs[i]["mol"].nao, "kind": reqs[i]["kind"], "arrival_s": round(ta, 3),
                             "latency_ms": round(1e3 * (td - ta), 1), "alone_ms": round(1e3 * seq_mixed[i], 1),
                             "frontend_ms": round(1e3 * (t_sub[i] - ta), 1)}
                            for sl, i, ta, td in sorted(per_req, key=lambda x: -x[0])[:5]],
        "throughput_rps": len(reqs) / span, "span_s": span,
        "sequential_fp64": {"throughput_rps": len(reqs) / sum(seq_fp64),
                            "p50_service_ms": 1e3 * float(np.median(seq_fp64)),
                            "total_s": sum(seq_fp64)},
        "sequential_mixed": {"throughput_rps": capacity, "total_s": sum(seq_mixed)},
        "error_vs_fp64": {"J_max_rel_to_max": max(errs_j) if errs_j else None,
                          "K_max_rel_to_max": max(errs_k) if errs_k else None,
                          "grad_max_rel_to_max": max(errs_g) if errs_g else None,
                          "how": "4096 sampled elements per J/K result, full gradient"},
        "service": {k2: st[k2] for k2 in ("steps", "launches", "bytes_peak", "budget", "completed",
                                          "p50_ms", "p99_ms")},
        "service_latency_what": "service p50/p99: submission to completion inside the service (without "
                                "the frontend's context creation and density formation)",
        "budget_gb": budget_gb, "frontend_threads": frontend_threads,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--nao-max", type=int, default=730)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--saturated", action="store_true", help="every request arrives at time 0")
    ap.add_argument("--frontend-threads", type=int, default=4)
    args = ap.parse_args()
    import torch
    from paper_2607_05622_gb300 import ltjk as L
    out = run_stream(L, torch, torch.device("cuda:0"), args.requests, args.nao_max, args.budget_gb, args.load,
                     args.frontend_threads, saturated=args.saturated)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
