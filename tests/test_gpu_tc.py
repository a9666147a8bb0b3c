"""Tensor-core interior corrections of batched applies (eqs. 4-5, 10-11).

Where every substructure's interior holds 128-256 DOFs, the setup forms
A_II^{-1} and H = A_II^{-1} A_{I Gamma} per substructure in FP64, and the
batched FP32 and BF16 applies run the pre- and post-corrections as dense
tcgen05 products (three TF32 products for FP32, one BF16 product with the
right-hand sides split in two).  These tests check that the route is taken
and that it keeps the mixed-path bounds of the per-apply output against the
FP64 apply (1e-5 FP32, 1e-2 BF16), against the oracle's apply as well, for
full and ragged batch widths; that it agrees with the triangular-sweep
kernels (BDDC_TC=0) to the same bounds; and that batched PCG with it reaches
the oracle's iteration count and a true relative residual of 1e-8.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import bddc as obddc          # noqa: E402
from oracle import pcg as opcg            # noqa: E402
from paper_0911_5730_gb300 import inputs  # noqa: E402

TOL = {"fp32": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


@pytest.fixture(scope="module")
def case():
    wl = inputs.two_level_channels(nx=64, sub=16, tau=10.0)
    return wl, obddc.build_workload(wl)


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("K", [32, 5])
def test_tc_apply_within_mixed_bounds(lib, case, K, monkeypatch):
    monkeypatch.setenv("BDDC_TC", "all")
    wl, H = case
    P = lib.Problem.from_workload(wl)
    assert P.query()["tc_levels"] & 1, "level 1 should take the tensor-core route"
    R = inputs.normal_rhs(wl.n_dof, 41, K)
    Rt = torch.tensor(R, device="cuda")
    Z64 = P.apply(Rt).cpu().numpy()
    for j in range(K):
        assert _relerr(Z64[j], H.apply(R[j])) <= 1e-10
    for prec, tol in TOL.items():
        P.set_precision(prec)
        Zm = P.apply(Rt).cpu().numpy()
        errs = [_relerr(Zm[j], Z64[j]) for j in range(K)]
        print("%s K=%d: max per-apply error %.3e (bound %.0e)" % (prec, K, max(errs), tol))
        assert max(errs) <= tol, (prec, errs)
        Zm2 = P.apply(Rt).cpu().numpy()          # the same call again: same result
        assert np.array_equal(Zm, Zm2)
    P.close()


def test_tc_agrees_with_sweeps(lib, case):
    wl, _ = case
    R = inputs.normal_rhs(wl.n_dof, 43, 32)
    Rt = torch.tensor(R, device="cuda")
    out = {}
    for route in ("tc", "sweeps"):
        os.environ["BDDC_TC"] = "all" if route == "tc" else "0"
        try:
            P = lib.Problem.from_workload(wl)
            for prec in ("fp32", "bf16"):
                P.set_precision(prec)
                out[route, prec] = P.apply(Rt).cpu().numpy()
            P.close()
        finally:
            os.environ.pop("BDDC_TC", None)
    for prec, tol in TOL.items():
        for j in range(32):
            assert _relerr(out["tc", prec][j], out["sweeps", prec][j]) <= 2 * tol


@pytest.mark.parametrize("route", ["all", "default"])
def test_tc_batched_pcg_matches_oracle(lib, case, route, monkeypatch):
    monkeypatch.setenv("BDDC_TC", route)
    wl, H = case
    P = lib.Problem.from_workload(wl)
    B = inputs.normal_rhs(wl.n_dof, 47, 32)
    ref = [opcg.pcg(H.A, B[j], H.apply, rtol=1e-8) for j in range(0, 32, 8)]
    for prec in ("fp32", "bf16"):
        P.set_precision(prec)
        X, infos = P.solve(torch.tensor(B, device="cuda"), rtol=1e-8)
        X = X.cpu().numpy()
        for j in range(32):
            assert infos[j]["status"] == 0 and infos[j]["batch_width"] == 32
            rt = np.linalg.norm(B[j] - H.A @ X[j]) / np.linalg.norm(B[j])
            assert rt <= 1e-8, (prec, j, rt)
        if prec == "fp32":
            for q, j in enumerate(range(0, 32, 8)):
                assert abs(infos[j]["iters"] - ref[q].iters) <= 1, (j, infos[j]["iters"], ref[q].iters)
    P.close()
