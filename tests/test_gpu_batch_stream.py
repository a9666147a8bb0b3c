"""Batched right-hand sides through the streaming Dirichlet kernel and the
chunked Neumann / averaging kernels (the batch kernels for substructures
whose operators do not fit in shared memory).

Irregular cells of about 1000 DOFs (the cell size of the 4096-cell Voronoi
workload) take these kernels by themselves; BDDC_BATCH_STREAM=1 routes the
smaller workloads there too, so that the block-swizzled factors of uniform
power-of-two blocks and three-level hierarchies are covered as well.  The
checks are those of the staged batch kernels: the oracle's apply column by
column within 1e-10 (FP64), the mixed-path tolerances against the FP64 apply,
and the oracle's PCG iteration counts and solutions.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import bddc as obddc          # noqa: E402
from oracle import pcg as opcg            # noqa: E402
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
    "channels_64": inputs.two_level_channels(nx=64, sub=16),
    "three_level_64": inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
    "voronoi_64": inputs.three_level_voronoi(nx=64, cells=4, group=2, levels=2),
    "voronoi_128_large_cells": inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2),
    "voronoi_128_3lev": inputs.three_level_voronoi(nx=128, cells=8, group=2, levels=3),
}
NATURAL = {"voronoi_128_large_cells"}     # streaming kernels without the switch
_cache = {}


def _oracle(name):
    if name not in _cache:
        _cache[name] = obddc.build_workload(WL[name])
    return _cache[name]


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(params=list(WL))
def case(request, lib, monkeypatch):
    name = request.param
    if name not in NATURAL:
        monkeypatch.setenv("BDDC_BATCH_STREAM", "1")
    else:
        monkeypatch.delenv("BDDC_BATCH_STREAM", raising=False)
    P = lib.Problem.from_workload(WL[name])
    yield name, P
    P.close()


def test_stream_batch_apply_matches_oracle(case):
    name, P = case
    wl = WL[name]
    H = _oracle(name)
    R = inputs.normal_rhs(wl.n_dof, 23, 7)
    Rt = torch.tensor(R, device="cuda")
    Z = P.apply(Rt).cpu().numpy()                       # one call, K = 7
    for j in range(7):
        assert _relerr(Z[j], H.apply(R[j])) <= 1e-10, (name, j)
    for prec, tol in (("fp32", 1e-5), ("bf16", 1e-2)):
        P.set_precision(prec)
        Zm = P.apply(Rt).cpu().numpy()
        for j in range(7):
            assert _relerr(Zm[j], Z[j]) <= tol, (name, prec, j)


def test_stream_batch_pcg_matches_oracle(case):
    name, P = case
    wl = WL[name]
    H = _oracle(name)
    B = inputs.normal_rhs(wl.n_dof, 33, 4)
    B[2] = 0.0                                          # converged at the start
    X, infos = P.solve(torch.tensor(B, device="cuda"), rtol=1e-8)
    X = X.cpu().numpy()
    assert all(i["batch_width"] == 4 for i in infos)    # the lockstep batch ran
    for j in range(4):
        if j == 2:
            assert np.all(X[j] == 0.0) and infos[j]["iters"] == 0
            continue
        ref = opcg.pcg(H.A, B[j], H.apply, rtol=1e-8)
        assert infos[j]["status"] == 0
        assert infos[j]["iters"] == ref.iters, (name, j, infos[j]["iters"], ref.iters)
        assert _relerr(X[j], ref.x) <= 1e-10
        assert abs(infos[j]["kappa_est"] - ref.kappa) <= 1e-6 * ref.kappa


def test_stream_batch_full_width_mixed(case):
    name, P = case
    wl = WL[name]
    B = torch.tensor(inputs.normal_rhs(wl.n_dof, 43, 32), device="cuda")
    X64, inf64 = P.solve(B)
    assert all(i["batch_width"] == 32 and i["status"] == 0 for i in inf64)
    P.set_precision("fp32")
    X32, inf32 = P.solve(B)
    for j in range(32):
        assert inf32[j]["status"] == 0 and inf32[j]["relres_true"] <= 1e-8, (name, j)
        assert _relerr(X32[j].cpu().numpy(), X64[j].cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("mode", ["serial", "parallel"])
def test_size_buckets_serial_and_at_once(lib, monkeypatch, mode):
    """The streaming kernel's size buckets launched one after another or at
    once on forked streams (the autotuner picks; BDDC_BUCKETS forces): 64
    Voronoi cells of about 1000 DOFs fall in several buckets.  FP64 batched
    apply within 1e-10 of the oracle, FP32 within 1e-5 of the FP64 apply, and
    a batched PCG with the oracle's iteration count."""
    monkeypatch.setenv("BDDC_BUCKETS", mode)
    monkeypatch.delenv("BDDC_BATCH_STREAM", raising=False)
    wl = inputs.three_level_voronoi(nx=256, cells=8, group=2, levels=2)
    if "voronoi_256_cells" not in _cache:
        _cache["voronoi_256_cells"] = obddc.build_workload(wl)
    H = _cache["voronoi_256_cells"]
    P = lib.Problem.from_workload(wl)
    try:
        R = inputs.normal_rhs(wl.n_dof, 31, 9)
        Rt = torch.tensor(R, device="cuda")
        Z = P.apply(Rt).cpu().numpy()
        for j in range(9):
            assert _relerr(Z[j], H.apply(R[j])) <= 1e-10, j
        assert bool(P.query(level=None)["tuned_buckets_at_once"] & 1) == (mode == "parallel")
        P.set_precision("fp32")
        Zm = P.apply(Rt).cpu().numpy()
        for j in range(9):
            assert _relerr(Zm[j], Z[j]) <= 1e-5, j
        P.set_precision("fp64")
        b = R[:4]
        X, infos = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
        for j in range(4):
            res = opcg.pcg(H.A, b[j], H.apply, rtol=1e-8)
            assert infos[j]["status"] == 0 and infos[j]["iters"] == res.iters
            assert _relerr(X[j].cpu().numpy(), res.x) <= 1e-10
    finally:
        P.close()
