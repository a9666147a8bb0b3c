"""Serving a mix of resident problems (config 5): the 512x512 channel problem
(two levels), the 1024x1024 three-level problem (log-uniform coefficient per
8x8 block) and the 2048x2048 three-level problem on 4096 Voronoi cells, all
set up once and kept on the device, each fed by its own seeded Poisson stream
of requests of 1-64 N(0,1) right-hand sides (at least one request per
problem in the window), served at once by one server
(continuous batching, three engines per problem and precision) that admits
requests by an HBM budget.

Usage: ``python -m paper_0911_5730_gb300.serve_mix [--load 0.8] [--seconds 3]
[--precisions fp32,fp64] [--problems channels,blocks,voronoi]``.
The offered rate of each problem is `load` times its share of the GPU: its
own closed-loop rate (one solve of 96 right-hand sides, measured first in the
same precision) divided by the number of problems.  Prints one JSON object:
per precision and problem the offered and achieved right-hand sides per
second and the p50/p99 request latency (submit to completion).
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time

import numpy as np
import torch

from . import bddc, inputs

PROBLEMS = {
    "channels": ("two_level_channels_512", lambda: inputs.two_level_channels()),
    "blocks": ("three_level_blocks_1024", lambda: inputs.three_level_blocks()),
    "voronoi": ("three_level_voronoi_2048", lambda: inputs.three_level_voronoi()),
}
CAPACITY_RHS = 96
RTOL = 1e-8


def _capacity(P, n, seed):
    """Closed-loop right-hand sides per second: one warm-up and one timed
    solve of CAPACITY_RHS right-hand sides."""
    B = torch.tensor(inputs.normal_rhs(n, seed, CAPACITY_RHS), device="cuda")
    P.solve(B, rtol=RTOL)
    torch.cuda.synchronize()
    t = time.perf_counter()
    P.solve(B, rtol=RTOL)
    torch.cuda.synchronize()
    return CAPACITY_RHS / (time.perf_counter() - t)


def _budget(wls):
    """HBM budget of the requests in flight: room for the largest request
    (64 right-hand sides, input and solution) of every problem twice over."""
    return int(sum(2 * 2 * 64 * 8 * wl.n_dof for wl in wls))


def arrivals(keys, cap, load, seconds, seed):
    """Per problem a seeded Poisson stream of requests of 1-64 right-hand
    sides at load x cap[k] / len(keys) right-hand sides per second over
    `seconds`: lists of (arrival time, right-hand sides, seed of their
    values).  A problem whose stream draws no request in the window (a slow
    one in a short window) gets one at a drawn time, of a drawn size but no
    more right-hand sides than its stream offers in the window on average,
    so that every problem is measured without adding much work."""
    plans = {}
    for i, k in enumerate(keys):
        rng = np.random.default_rng(seed + 100 + i)
        rate = load * cap[k] / len(keys)
        t, ev = 0.0, []
        while True:
            m = int(rng.integers(1, 65))
            t += rng.exponential(m / rate)
            if t >= seconds:
                break
            ev.append((t, m, int(rng.integers(1 << 31))))
        if not ev:
            # no larger than the stream's expected right-hand sides in the window
            m = min(int(rng.integers(1, 65)), max(1, int(rate * seconds)))
            ev.append((float(rng.uniform(0.0, seconds)), m, int(rng.integers(1 << 31))))
        plans[k] = ev
    return plans


def serve(Ps, wls, load, seconds, seed, budget, cap=None):
    """One mixed stream over the resident problems Ps (same keys as wls),
    offered at load x cap[k] / len(Ps) right-hand sides per second per
    problem (cap: the closed-loop rates, measured here if not given)."""
    keys = list(Ps)
    if cap is None:
        cap = {k: _capacity(Ps[k], wls[k].n_dof, seed + i) for i, k in enumerate(keys)}
    srv = bddc.Server(hbm_budget=budget, max_slots=1)
    plans = arrivals(keys, cap, load, seconds, seed)
    # a short window of large requests can offer far more or less work than
    # `load` of the GPU: the arrival times are scaled so that the sampled
    # requests (GPU time at the closed-loop rates) fill `load` of the window
    work = sum(m / cap[k] for k, ev in plans.items() for _, m, _ in ev)
    scale = work / (load * seconds) if work > 0 else 1.0
    events = sorted(((t * scale, k, m, np.random.default_rng(rs).standard_normal((m, wls[k].n_dof)))
                     for k, ev in plans.items() for t, m, rs in ev), key=lambda e: e[0])
    tickets = []
    lat = {k: [] for k in keys}
    bad = []
    t0 = time.perf_counter()

    def collect():
        i = 0
        while i < len(events):
            while i >= len(tickets):
                time.sleep(1e-4)
            k, tk = tickets[i]
            _, infos, ms = srv.wait(tk)
            miss = [(j["status"], j["iters"], j["relres_true"]) for j in infos
                    if not (j["status"] == 0 and j["relres_true"] <= RTOL)]
            if miss:
                bad.append((k, miss))
            lat[k].append((ms, time.perf_counter()))
            i += 1

    th = threading.Thread(target=collect)
    th.start()
    for t, k, m, b in events:
        while time.perf_counter() - t0 < t:
            time.sleep(min(1e-3, max(0.0, t - (time.perf_counter() - t0))))
        tickets.append((k, srv.submit(Ps[k], b if m > 1 else b[0], rtol=RTOL)))
    th.join()
    srv.close()
    out = {}
    for k in keys:
        ms = sorted(v[0] for v in lat[k])
        n_rhs = sum(m for _, kk, m, _ in events if kk == k)
        if not ms:
            out[PROBLEMS[k][0]] = {"closed_loop_rhs_per_s": cap[k], "requests": 0, "rhs": 0}
            continue
        end = max(v[1] for v in lat[k]) - t0

        def pct(p):
            return ms[min(len(ms) - 1, int(math.ceil(p / 100.0 * len(ms))) - 1)]

        out[PROBLEMS[k][0]] = {"closed_loop_rhs_per_s": cap[k],
                               "offered_rhs_per_s": n_rhs / (seconds * scale),
                               "requests": len(ms), "rhs": n_rhs, "solves_per_s": n_rhs / end,
                               "latency_ms": {"p50": pct(50), "p99": pct(99)}}
    out["all"] = {"solves_per_s": sum(v.get("solves_per_s", 0.0) for v in out.values()),
                  "window_s": seconds * scale, "offered_work_s": work,
                  # right-hand sides that missed the tolerance (none expected)
                  "failed_rhs": sum(len(b) for _, b in bad), "failed_sample": bad[:2]}
    return out, cap


def run(load: float = 0.8, seconds: float = 3.0, seed: int = 5001, precisions=("fp32", "fp64"),
        problems=("channels", "blocks", "voronoi")) -> dict:
    wls = {k: PROBLEMS[k][1]() for k in problems}
    setup_s = {}
    Ps = {}
    for k in problems:
        t = time.perf_counter()
        Ps[k] = bddc.Problem.from_workload(wls[k], precision=precisions[0])
        torch.cuda.synchronize()
        setup_s[PROBLEMS[k][0]] = time.perf_counter() - t
    budget = _budget(wls.values())
    out = {"load": load, "seconds": seconds, "seed": seed, "hbm_budget_bytes": budget,
           "setup_s": setup_s, "stream": "per problem a Poisson stream (seeded), 1-64 N(0,1) right-hand "
                                         "sides per request at load x (closed-loop rate / problems), arrival "
                                         "times scaled so that the sampled requests fill `load` of the window"}
    caps = {}
    try:
        for prec in precisions:
            for P in Ps.values():
                P.set_precision(prec)
            out[prec], caps[prec] = serve(Ps, wls, load, seconds, seed, budget)
        if "fp32" in caps and "fp64" in caps:
            # closed-loop capacity of the mix, and the FP64 stream served in FP32
            # (same arrivals and right-hand sides: the latency comparison)
            out["mixed_over_fp64_capacity"] = sum(caps["fp32"].values()) / sum(caps["fp64"].values())
            for P in Ps.values():
                P.set_precision("fp32")
            out["fp32_on_fp64_stream"], _ = serve(Ps, wls, load, seconds, seed, budget, cap=caps["fp64"])
    finally:
        for P in Ps.values():
            P.close()
    return out


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--seconds", type=float, default=3.0)
    ap.add_argument("--precisions", default="fp32,fp64")
    ap.add_argument("--problems", default="channels,blocks,voronoi")
    a = ap.parse_args()
    print(json.dumps(run(a.load, a.seconds, precisions=tuple(a.precisions.split(",")),
                         problems=tuple(a.problems.split(",")))))


if __name__ == "__main__":
    main()
