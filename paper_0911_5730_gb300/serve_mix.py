"""Serving a mix of problems (config 5): the 512x512 channel problem (two
levels) and the 1024x1024 three-level problem (log-uniform coefficient per
8x8 block), both resident, each fed by its own seeded Poisson stream of
requests of 1-64 N(0,1) right-hand sides, served at once by one server
(continuous batching, three engines per problem).

Usage: ``python -m paper_0911_5730_gb300.serve_mix [--load 0.8] [--seconds 4]``.
The offered rate of each problem is `load` times its share of the GPU: its
own closed-loop rate (one solve of 96 right-hand sides, measured first)
divided by the number of problems.  Prints one JSON object:
per problem the offered and achieved right-hand sides per second and the
p50/p99 request latency (submit to completion).
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


def _capacity(P, n, seed):
    B = torch.tensor(inputs.normal_rhs(n, seed, 96), device="cuda")
    P.solve(B)
    torch.cuda.synchronize()
    t = time.perf_counter()
    P.solve(B)
    torch.cuda.synchronize()
    return 96 / (time.perf_counter() - t)


def run(load: float = 0.8, seconds: float = 4.0, seed: int = 5001) -> dict:
    probs = {"two_level_channels_512": inputs.two_level_channels(),
             "three_level_blocks_1024": inputs.three_level_blocks()}
    Ps = {k: bddc.Problem.from_workload(wl, precision="fp32") for k, wl in probs.items()}
    cap = {k: _capacity(Ps[k], probs[k].n_dof, seed + i) for i, k in enumerate(probs)}
    srv = bddc.Server(hbm_budget=0, max_slots=1)
    plans = {}
    for i, k in enumerate(probs):
        rng = np.random.default_rng(seed + 100 + i)
        rate = load * cap[k] / len(probs)
        t, ev = 0.0, []
        while t < seconds:
            m = int(rng.integers(1, 65))
            ev.append((t, m, rng.standard_normal((m, probs[k].n_dof))))
            t += rng.exponential(m / rate)
        plans[k] = ev
    events = sorted(((t, k, m, b) for k, ev in plans.items() for t, m, b in ev), key=lambda e: e[0])
    tickets = []
    lat = {k: [] for k in probs}
    t0 = time.perf_counter()

    def collect():
        i = 0
        while i < len(events):
            while i >= len(tickets):
                time.sleep(1e-4)
            k, tk = tickets[i]
            _, infos, ms = srv.wait(tk)
            assert all(j["status"] == 0 and j["relres_true"] <= 1e-8 for j in infos)
            lat[k].append((ms, time.perf_counter()))
            i += 1

    th = threading.Thread(target=collect)
    th.start()
    for t, k, m, b in events:
        while time.perf_counter() - t0 < t:
            time.sleep(min(1e-3, max(0.0, t - (time.perf_counter() - t0))))
        tickets.append((k, srv.submit(Ps[k], b if m > 1 else b[0], rtol=1e-8)))
    th.join()
    srv.close()
    out = {"load": load, "seconds": seconds, "seed": seed, "problems": {}}
    for k in probs:
        ms = sorted(v[0] for v in lat[k])
        end = max(v[1] for v in lat[k]) - t0
        n_rhs = sum(m for _, kk, m, _ in events if kk == k)

        def pct(p):
            return ms[min(len(ms) - 1, int(math.ceil(p / 100.0 * len(ms))) - 1)]

        out["problems"][k] = {"closed_loop_rhs_per_s": cap[k], "offered_rhs_per_s": load * cap[k] / len(probs),
                              "requests": len(ms), "rhs": n_rhs, "solves_per_s": n_rhs / end,
                              "latency_ms": {"p50": pct(50), "p99": pct(99)}}
    for P in Ps.values():
        P.close()
    return out


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--seconds", type=float, default=4.0)
    a = ap.parse_args()
    print(json.dumps(run(a.load, a.seconds)))


if __name__ == "__main__":
    main()
