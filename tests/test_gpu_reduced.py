"""The interface-reduced solve on the GPU (bddc_pcg_solve_reduced) against
the oracle's (oracle/reduced.py): the same iteration count, the solution
within 1e-10, a true relative residual of 1e-8, and the Lanczos condition
number within 1e-5.  The reduced operator has a cluster of unit eigenvalues
next to its smallest Ritz value, which makes that estimate rounding-sensitive:
the oracle's own kappa moves by 3.6e-6 on the 64^2 Voronoi case when S is
formed as a dense Schur complement instead of substructure by substructure
(equal in exact arithmetic), so 1e-6 would be below the estimate's precision.
With FP32 and BF16 preconditioners (S stays FP64) the solve still reaches 1e-8
in the true residual.  Exact preconditioner: one iteration.  Zero right-hand
side: x = 0 in zero iterations.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import bddc as obddc          # noqa: E402
from oracle.reduced import Reduced        # noqa: E402
from paper_0911_5730_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


WL = {
    "unit_all": inputs.two_level_unit(constraints="all"),
    "channels_64": inputs.two_level_channels(nx=64, sub=16),
    "channels_96_ragged": inputs.two_level_channels(nx=96, sub=16, tau=3.0),
    "three_level_64": inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
    "voronoi_64": inputs.three_level_voronoi(nx=64, cells=4, group=2, levels=2),
    "voronoi_128_large_cells": inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2),
    "voronoi_128_3lev": inputs.three_level_voronoi(nx=128, cells=8, group=2, levels=3),
}


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", [k for k in WL if k != "unit_all"])
def test_reduced_matches_oracle(lib, name):
    wl = WL[name]
    R = Reduced(obddc.build_workload(wl))
    b = wl.rhs()
    xr, ref = R.solve(b, rtol=1e-8)
    P = lib.Problem.from_workload(wl)
    x, info = P.solve_reduced(torch.tensor(b, device="cuda"), rtol=1e-8)
    assert info["status"] == 0
    assert info["iters"] == ref.iters, (name, info["iters"], ref.iters)
    assert _relerr(x.cpu().numpy(), xr) <= 1e-10
    assert info["relres_true"] <= 1e-8
    assert abs(info["kappa_est"] - ref.kappa) <= 1e-5 * ref.kappa
    # the full PCG on the same problem takes the same number of iterations
    xf, inf = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    assert inf[0]["iters"] == info["iters"]
    assert _relerr(x.cpu().numpy(), xf.cpu().numpy()) <= 1e-6
    for prec in ("fp32", "bf16"):
        P.set_precision(prec)
        xm, im = P.solve_reduced(torch.tensor(b, device="cuda"), rtol=1e-8, maxit=500)
        assert im["status"] == 0 and im["relres_true"] <= 1e-8, (name, prec, im)
    P.close()


def test_reduced_exact_preconditioner_and_zero_rhs(lib):
    wl = WL["unit_all"]
    P = lib.Problem.from_workload(wl)
    x, info = P.solve_reduced(torch.tensor(wl.rhs(), device="cuda"), rtol=1e-10)
    assert info["iters"] == 1 and info["status"] == 0
    z, iz = P.solve_reduced(torch.zeros(wl.n_dof, dtype=torch.float64, device="cuda"))
    assert iz["iters"] == 0 and iz["status"] == 0 and float(z.abs().max()) == 0.0
    P.close()
