"""Degenerate and edge cases of the GPU path against the oracle:
one substructure (no interface, no coarse space: the apply is A^{-1}),
substructures of 2x2 elements (one interior DOF each), tau = infinity in the
adaptive mode (no edge constraints: the corners-only preconditioner), an
rhs of zeros, and the bounded device wait giving up with BDDC_E_TIMEOUT."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import bddc as obddc   # noqa: E402
from paper_0911_5730_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    return bddc


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_single_substructure_is_direct_solve(lib):
    nx = 12
    k = inputs.channel_coefficient(nx, 4, 0.1, 1e4)
    P = lib.Problem(nx, k, np.zeros(nx * nx, np.int32), 1, constraints="corners")
    H = obddc.build(nx, k, np.zeros(nx * nx, np.int32), 1, 2, "corners")
    b = inputs.normal_rhs(H.n, 2)
    z = P.apply(torch.tensor(b, device="cuda")).cpu().numpy()
    assert _rel(z, spl.spsolve(H.A.tocsc(), b)) <= 1e-10
    x, info = P.solve(torch.tensor(b, device="cuda"), rtol=1e-10)
    assert info[0]["iters"] == 1
    P.close()


def test_tiny_substructures(lib):
    nx = 8
    e2s, ns = inputs.grid_decomposition(nx, 2)
    k = inputs.block_log_uniform_coefficient(nx, 2, 9, 0.0, 2.0)
    for mode in ("corners", "corners+edges", "all"):
        P = lib.Problem(nx, k, e2s, ns, constraints=mode)
        H = obddc.build(nx, k, e2s, ns, 2, mode)
        r = inputs.normal_rhs(H.n, 3)
        z = P.apply(torch.tensor(r, device="cuda")).cpu().numpy()
        assert _rel(z, H.apply(r)) <= 1e-10
        P.close()


def test_adaptive_with_infinite_tau_is_corners(lib):
    wl = inputs.two_level_channels(nx=64, sub=16, tau=np.inf)
    Pa = lib.Problem.from_workload(wl)
    Pc = lib.Problem(wl.nx, wl.k, wl.elem_to_sub, wl.n_sub1, constraints="corners")
    r = torch.tensor(inputs.normal_rhs(wl.n_dof, 6), device="cuda")
    assert _rel(Pa.apply(r).cpu().numpy(), Pc.apply(r).cpu().numpy()) <= 1e-12
    assert list(Pa.query(level=1)["n_selected"]) == [0] * Pa.query()["n_edges"][0]
    Pa.close(); Pc.close()


def test_zero_rhs(lib):
    wl = inputs.two_level_unit()
    P = lib.Problem.from_workload(wl)
    x, info = P.solve(torch.zeros(wl.n_dof, dtype=torch.float64, device="cuda"))
    assert info[0]["status"] == 0 and info[0]["iters"] == 0
    assert float(x.abs().max()) == 0.0
    P.close()


def test_bounded_wait_timeout(lib):
    code = lib.load().bddc_selftest_wait_timeout(None)
    assert code == -5
    # the device is still usable afterwards, and a wait that gave up elsewhere
    # is not charged to a context: its solves (single and batched) and
    # applies report success, and the applies record no timeout
    # (bddc_info.apply_status)
    wl = inputs.two_level_unit()
    P = lib.Problem.from_workload(wl)
    b = torch.tensor(wl.rhs(), device="cuda")
    for _ in range(2):
        x, info = P.solve(b)
        assert info[0]["status"] == 0
        X, infos = P.solve(torch.stack([b, 2 * b]))
        assert all(i["status"] == 0 for i in infos)
        P.apply(b)
        torch.cuda.synchronize()
        assert P.query()["apply_status"] == 0
        assert lib.load().bddc_selftest_wait_timeout(None) == -5
    P.close()
