"""Constraint study on the GPU: PCG iterations, Lanczos condition number,
coarse sizes and the indicator omega~ for corner, corner + edge-average and
adaptive constraints at two and three levels.  This is the experiment shape of
the paper's Tables 1-7 (Sec. 6) on the scalar problem of Sec. 5, with
synthetic coefficients:

* ``channels``: 512x512 mesh, 32x32 substructures of 16x16 elements, k = 1e6
  on channels that cut through the substructures (two levels);
* ``blocks``: 512x512 mesh, 64x64 substructures of 8x8 elements, log10 k
  uniform in [0, 6] per substructure, level-2 groups of 8x8 (two and three
  levels).

Usage: ``python -m paper_0911_5730_gb300.study [--precision fp64]``; prints a
markdown table.  Every solve is one right-hand side (the workload's seeded
N(0,1) vector), relative residual 1e-8, FP64 PCG.
"""
from __future__ import annotations

import argparse
import dataclasses
import time

import torch

from . import bddc, inputs

MODES = ("corners", "corners+edges", "adaptive")


def cases(nx: int = 512, tau: float = 10.0):
    ch = inputs.two_level_channels(nx=nx, sub=16, tau=tau)
    bl = inputs.three_level_blocks(nx=nx, sub=8, group=8, tau=tau)
    for mode in MODES:
        yield "channels", 2, dataclasses.replace(ch, constraints=mode)
    for levels in (2, 3):
        for mode in MODES:
            wl = dataclasses.replace(bl, constraints=mode)
            if levels == 2:
                wl = dataclasses.replace(wl, levels=2, sub1_to_sub2=None, n_sub2=0)
            yield "blocks", levels, wl


def run(nx: int = 512, tau: float = 10.0, precision: str = "fp64", maxit: int = 5000) -> list[dict]:
    rows = []
    for coef, levels, wl in cases(nx, tau):
        P = bddc.Problem.from_workload(wl, precision=precision)
        q = P.query(level=None)
        b = torch.tensor(wl.rhs(), device="cuda")
        P.solve(b, rtol=1e-8, maxit=maxit)                     # warm: graphs, workspace
        torch.cuda.synchronize()
        t = time.perf_counter()
        x, info = P.solve(b, rtol=1e-8, maxit=maxit)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        rows.append({"coef": coef, "levels": levels, "constraints": wl.constraints,
                     "n_dof": q["n_dof"], "omega_tilde": q["omega_tilde"],
                     "iters": info[0]["iters"], "kappa": info[0]["kappa_est"],
                     "status": info[0]["status"], "relres": info[0]["relres_true"],
                     "setup_ms": q["setup_ms"], "solve_ms": ms})
        P.close()
    return rows


def table(rows: list[dict]) -> str:
    out = ["| coefficient | L | constraints | DOFs per level | omega~ | iterations | kappa | setup ms | solve ms |",
           "|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        om = "%.3g" % r["omega_tilde"] if r["constraints"] == "adaptive" else "-"
        it = str(r["iters"]) if r["status"] == 0 else "%d (no conv.)" % r["iters"]
        out.append("| %s | %d | %s | %s | %s | %s | %.3g | %.0f | %.1f |" % (
            r["coef"], r["levels"], r["constraints"], " / ".join(str(n) for n in r["n_dof"]), om, it,
            r["kappa"], r["setup_ms"], r["solve_ms"]))
    return "\n".join(out)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--tau", type=float, default=10.0)
    ap.add_argument("--precision", default="fp64", choices=("fp64", "fp32", "bf16"))
    a = ap.parse_args()
    print(table(run(a.nx, a.tau, a.precision)))


if __name__ == "__main__":
    main()
