"""Plane elasticity (the problem of the paper's experiments, Sec. 5) through
the GPU path against the oracle: lambda = 1, mu = 2 (scaled per element by a
seeded coefficient), clamped on x = 0, a jagged level-1 edge and, on three
levels, a jagged level-2 edge.

The bar of the other parity tests: the operator within 1e-13, the apply within
1e-10 per right-hand side (single and batched), the number of selected
constraints per edge identical, and the PCG trajectory: the iterate after a
fixed 8 iterations within 1e-9 of the oracle's (a relative perturbation of
1e-13 in b moves the oracle's own iterate there by at most 4e-12).  Run to the residual 1e-8
in FP64, the adaptive cases (spectrum of M^{-1} A in [1, 2.8]) keep the
oracle's iteration count, solution within 1e-10 and kappa within 1e-6, solved
alone or in a batch of three.  With
corners or corner + edge averages only (spectrum up to 25-50) the iteration
at which the residual crosses 1e-8 is not a property of the method: a
relative perturbation of 1e-12 in b moves the oracle's own residual at the
crossing between 0.7e-8 and 1.1e-8 (25 or 26 iterations; 45 or 47), and its
count differs between the x86 and Arm BLAS builds; there the bar is the
true residual below 1e-8, two iterations either way and kappa within 1e-3.
FP32 and BF16 applies reach the FP64 residual 1e-8.  At the paper's size (768^2, 48 x 48 substructures, 3 x 3 on
level 2) the counts of Tables 1-2 come from the setup itself and the solve is
checked by its true residual and Theorem 2's bound.
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


def _relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _k(nx, seed=71):
    # a seeded coefficient scaling the Lame parameters (contrast 10^2)
    return 10 ** np.random.default_rng(seed).uniform(0, 2, nx * nx)


CASES = {
    "2lev_ce": dict(nx=32, sub=8, levels=2, constraints="corners+edges"),
    "2lev_c": dict(nx=32, sub=8, levels=2, constraints="corners"),
    "2lev_adaptive": dict(nx=32, sub=8, levels=2, constraints="adaptive", tau=3.0),
    "3lev_adaptive": dict(nx=32, sub=8, levels=3, group=2, constraints="adaptive", tau=3.0),
    "3lev_ce": dict(nx=32, sub=4, levels=3, group=4, constraints="corners+edges"),
    "2lev_adaptive_64": dict(nx=64, sub=16, levels=2, constraints="adaptive", tau=10.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_elasticity_matches_oracle(lib, name):
    c = dict(CASES[name])
    wl = inputs.elasticity(k=_k(c["nx"]), **c)
    H = obddc.build_workload(wl)
    P = lib.Problem.from_workload(wl)
    assert P.n == wl.n_dof == H.n
    # the operator
    x = inputs.normal_rhs(wl.n_dof, 3)
    y = torch.empty(wl.n_dof, dtype=torch.float64, device="cuda")
    P.operator(torch.tensor(x, device="cuda"), y)
    assert _relerr(y.cpu().numpy(), H.A @ x) <= 1e-13
    # the apply, single and batched
    R = inputs.normal_rhs(wl.n_dof, 5, 3)
    Z = P.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    z0 = P.apply(torch.tensor(R[0], device="cuda")).cpu().numpy()
    for j in range(3):
        assert _relerr(Z[j], H.apply(R[j])) <= 1e-10
    assert _relerr(z0, H.apply(R[0])) <= 1e-10
    # adaptive selection per edge
    if c["constraints"] == "adaptive":
        q = P.query(level=1)
        assert list(q["n_selected"]) == [e["n_sel"] for e in H.info["edge_reports"][0]]
    # the PCG trajectory: the iterate after a fixed number of iterations
    b = wl.rhs()
    bt = torch.tensor(b, device="cuda")
    x8, i8 = P.solve(bt, rtol=1e-30, maxit=8, check=False)
    r8 = opcg.pcg(H.A, b, H.apply, fixed_iters=8)
    assert i8[0]["iters"] == 8
    assert _relerr(x8.cpu().numpy(), r8.x) <= 1e-9
    # PCG in FP64 to the residual 1e-8
    xs, info = P.solve(bt, rtol=1e-8)
    ref = opcg.pcg(H.A, b, H.apply, rtol=1e-8)
    assert info[0]["status"] == 0
    xg = xs.cpu().numpy()
    assert np.linalg.norm(b - H.A @ xg) <= 1e-8 * np.linalg.norm(b)
    if c["constraints"] == "adaptive":
        assert info[0]["iters"] == ref.iters
        assert _relerr(xg, ref.x) <= 1e-10
        assert abs(info[0]["kappa_est"] - ref.kappa) <= 1e-6 * ref.kappa
    else:
        assert abs(info[0]["iters"] - ref.iters) <= 2
        assert _relerr(xg, ref.x) <= 1e-6
        assert abs(info[0]["kappa_est"] - ref.kappa) <= 1e-3 * ref.kappa
    # batched PCG: each right-hand side as the oracle solves it alone, to the
    # single solve's bar (the same iterations and 1e-10 for the adaptive
    # cases; the corner and edge-average cases as above)
    X, infos = P.solve(torch.tensor(R, device="cuda"), rtol=1e-8)
    for j in range(3):
        rj = opcg.pcg(H.A, R[j], H.apply, rtol=1e-8)
        xj = X[j].cpu().numpy()
        assert infos[j]["status"] == 0 and infos[j]["batch_width"] == 3
        assert np.linalg.norm(R[j] - H.A @ xj) <= 1e-8 * np.linalg.norm(R[j])
        if c["constraints"] == "adaptive":
            assert infos[j]["iters"] == rj.iters, (name, j, infos[j]["iters"], rj.iters)
            assert _relerr(xj, rj.x) <= 1e-10, (name, j)
        else:
            assert abs(infos[j]["iters"] - rj.iters) <= 2
            assert _relerr(xj, rj.x) <= 1e-6
    P.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_elasticity_mixed_precision(lib, precision):
    wl = inputs.elasticity(nx=64, sub=16, levels=2, constraints="adaptive", tau=3.0, k=_k(64))
    P = lib.Problem.from_workload(wl, precision=precision)
    H = obddc.build_workload(wl)
    b = wl.rhs()
    r = inputs.normal_rhs(wl.n_dof, 9)
    z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
    assert _relerr(z, H.apply(r)) <= (1e-5 if precision == "fp32" else 1e-2)
    x, info = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8)
    assert info[0]["status"] == 0 and info[0]["relres_true"] <= 1e-8
    P.close()


def test_elasticity_reduced_matches_oracle(lib):
    from oracle.reduced import Reduced
    wl = inputs.elasticity(nx=32, sub=8, levels=2, constraints="adaptive", tau=3.0, k=_k(32))
    H = obddc.build_workload(wl)
    P = lib.Problem.from_workload(wl)
    b = wl.rhs()
    xr_ref, rr = Reduced(H).solve(b, rtol=1e-8)
    xr, ir = P.solve_reduced(torch.tensor(b, device="cuda"), rtol=1e-8)
    assert ir["status"] == 0 and ir["iters"] == rr.iters
    assert _relerr(xr.cpu().numpy(), xr_ref) <= 1e-10
    P.close()


@pytest.mark.parametrize("levels,constraints,tau", [(2, "corners", np.inf), (3, "corners+edges", np.inf),
                                                    (3, "adaptive", 3.0)])
def test_elasticity_paper_size(lib, levels, constraints, tau):
    wl = inputs.elasticity(nx=768, sub=16, levels=levels, group=16, constraints=constraints, tau=tau)
    P = lib.Problem.from_workload(wl, precision="fp32")
    q = P.query(level=1)
    ncl = q["n_dof"]
    if constraints == "corners":
        assert ncl[1] == 4700                     # 2 (49^2 - 4 - 47): x = 0 clamped
    if constraints == "corners+edges":
        assert ncl[1] == 13724 and ncl[2] == 44   # + 2 (16 - 4 - 2) + 2 * 12 on level 2
    b = torch.tensor(wl.rhs(), device="cuda")
    x, info = P.solve(b, rtol=1e-8)
    assert info[0]["status"] == 0 and info[0]["relres_true"] <= 1e-8
    if constraints == "adaptive":
        om = q["omega_tilde"]
        assert om <= tau ** (levels - 1) * (1 + 1e-12)
        assert info[0]["kappa_est"] <= om * (1 + 1e-3)
    P.close()


GENERIC = {
    "elastic_2lev_64": lambda: inputs.elasticity(nx=64, sub=16, levels=2, constraints="adaptive", tau=10.0,
                                                  k=_k(64)),
    "elastic_3lev_ce": lambda: inputs.elasticity(nx=32, sub=8, levels=3, group=2, constraints="corners+edges",
                                                  k=_k(32)),
    "voronoi_2lev": lambda: inputs.three_level_voronoi(nx=128, cells=4, group=2, levels=2, tau=10.0),
}


@pytest.mark.parametrize("name", list(GENERIC))
def test_generic_dirichlet_kernels(lib, name, monkeypatch):
    """The one-block-per-substructure Dirichlet kernels (the path of level-2
    substructures too large for the streaming kernel's stages, as at the
    paper's size), reached here with BDDC_GENERIC_DIR=1 on every level that
    the warp kernels do not take."""
    monkeypatch.setenv("BDDC_GENERIC_DIR", "1")
    wl = GENERIC[name]()
    H = obddc.build_workload(wl)
    P = lib.Problem.from_workload(wl)
    R = inputs.normal_rhs(wl.n_dof, 17, 2)
    for j in range(2):
        z = P.apply(torch.tensor(R[j], device="cuda")).cpu().numpy()
        assert _relerr(z, H.apply(R[j])) <= 1e-10
    b = wl.rhs()
    x8, _ = P.solve(torch.tensor(b, device="cuda"), rtol=1e-30, maxit=8, check=False)
    assert _relerr(x8.cpu().numpy(), opcg.pcg(H.A, b, H.apply, fixed_iters=8).x) <= 1e-9
    P.set_precision("fp32")
    z32 = P.apply(torch.tensor(R[0], device="cuda")).cpu().numpy()
    assert _relerr(z32, H.apply(R[0])) <= 1e-5
    P.close()
