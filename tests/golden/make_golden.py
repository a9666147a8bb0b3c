"""Write the oracle's results for the full-size workloads to tests/golden/.

Calls only the CPU oracle (oracle/) on the seeded inputs of
paper_0911_5730_gb300.inputs; nothing here touches the CUDA path.  Besides
the JSON summary, the full FP64 solution and apply vectors go to
<workload>_x.npy and <workload>_z.npy for the element-by-element parity of
the full-size GPU tests.

    python tests/golden/make_golden.py two_level_channels_512 three_level_blocks_1024
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import bddc, pcg                      # noqa: E402
from paper_0911_5730_gb300 import inputs          # noqa: E402

WORKLOADS = {
    "two_level_channels_512": lambda: inputs.two_level_channels(nx=512, sub=16, tau=10.0),
    "two_level_unit_32": lambda: inputs.two_level_unit(),
    "three_level_blocks_1024": lambda: inputs.three_level_blocks(),
}
SAMPLE_STRIDE = 997
APPLY_SEED = 19
LAM_EDGES = 2048          # at most about this many edges per level keep their eigenvalues


def _stride(n_edges):
    return max(1, -(-n_edges // LAM_EDGES))


def make(name):
    wl = WORKLOADS[name]()
    t0 = time.time()
    H = bddc.build_workload(wl)
    t_setup = time.time() - t0
    b = wl.rhs()
    r_apply = inputs.normal_rhs(wl.n_dof, APPLY_SEED)
    z_apply = H.apply(r_apply)
    t0 = time.time()
    res = pcg.pcg(H.A, b, H.apply, rtol=1e-8)
    t_solve = time.time() - t0
    idx = np.arange(0, wl.n_dof, SAMPLE_STRIDE)
    out = {
        "workload": name,
        "source": "oracle/ (CPU FP64), seeded inputs of paper_0911_5730_gb300.inputs",
        "n_dof": [b_.lv.n for b_ in H.bl] + [H.bl[-1].nc],
        "n_coarse": H.info["n_coarse"],
        "omega_tilde": H.info["omega_tilde"],
        "n_sel": [[int(r["n_sel"]) for r in reps] for reps in H.info["edge_reports"]],
        "edge_pairs": [[list(map(int, r["pair"])) for r in reps] for reps in H.info["edge_reports"]],
        # top eigenvalues of every LAM_STRIDE-th edge on levels with many edges
        "lam_stride": [_stride(len(reps)) for reps in H.info["edge_reports"]],
        "lam_top": [[[float("%.15g" % v) for v in r["lam"][:4]] for r in reps[::_stride(len(reps))]]
                    for reps in H.info["edge_reports"]],
        "pcg": {"rtol": 1e-8, "iters": res.iters, "kappa": res.kappa, "relres_true": res.relres_true},
        "x_sample_stride": SAMPLE_STRIDE,
        "x_sample": [float(v) for v in res.x[idx]],
        "x_norm": float(np.linalg.norm(res.x)),
        # one FP64 apply z = M^{-1} r of r = normal_rhs(n, APPLY_SEED), sampled
        "apply": {"seed": APPLY_SEED, "z_sample": [float(v) for v in z_apply[idx]],
                  "z_norm": float(np.linalg.norm(z_apply))},
        "oracle_seconds": {"setup": t_setup, "solve": t_solve},
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f)
    np.save(os.path.join(HERE, name + "_x.npy"), res.x)
    np.save(os.path.join(HERE, name + "_z.npy"), z_apply)
    print(name, "iters", res.iters, "nc", H.info["n_coarse"], "setup %.1fs solve %.1fs" % (t_setup, t_solve))


if __name__ == "__main__":
    for name in sys.argv[1:] or list(WORKLOADS):
        make(name)
