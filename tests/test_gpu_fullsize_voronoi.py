"""Config 4 at full size: 2048 x 2048 Q1 mesh, 4096 seeded Voronoi cells
(irregular substructures of about 700-1600 DOFs), 64 level-2 substructures,
three-level adaptive BDDC with tau = 10, log10 k ~ U[0, 6] per 8 x 8-element
block.

The oracle cannot run this size (dense per-substructure algebra on 4096
substructures of ~1000 DOFs), so the checks are properties that hold at any
size and that the GPU path cannot satisfy by accident:
* corners: the number of free nodes in three or more cells, counted here
  from the partition alone;
* PCG: the true relative residual ||b - A x|| / ||b|| <= 1e-8, with A x
  formed here from the oracle's Q1 element stiffness (FP64, numpy);
* Lemma 1 / Theorem 2: the condition-number estimate and the indicator
  omega~ stay below tau^(L-1) = 100;
* the FP32 apply within 1e-5 of the FP64 apply (the mixed-path tolerance).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import fem                    # noqa: E402
from paper_0911_5730_gb300 import inputs  # noqa: E402

TAU = 10.0


@pytest.fixture(scope="module")
def prob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0911_5730_gb300 import bddc
    wl = inputs.three_level_voronoi()
    P = bddc.Problem.from_workload(wl)
    yield wl, P
    P.close()


def _apply_A(nx, k, x):
    """A x for the Q1 operator with zero Dirichlet data, element by element."""
    K = fem.q1_reference_stiffness()
    X = np.zeros((nx + 1, nx + 1))                 # [j, i], boundary rows stay zero
    X[1:nx, 1:nx] = x.reshape(nx - 1, nx - 1)
    kk = k.reshape(nx, nx)                         # [ej, ei]
    # local nodes (0,0), (1,0), (1,1), (0,1) of element (ei, ej)
    corners = [X[:-1, :-1], X[:-1, 1:], X[1:, 1:], X[1:, :-1]]
    Y = np.zeros_like(X)
    for a, (dj, di) in enumerate(((0, 0), (0, 1), (1, 1), (1, 0))):
        contrib = kk * sum(K[a, b] * corners[b] for b in range(4))
        Y[dj:dj + nx, di:di + nx] += contrib
    return Y[1:nx, 1:nx].reshape(-1)


def test_corner_count_from_partition(prob):
    wl, P = prob
    nx = wl.nx
    lab = wl.elem_to_sub.reshape(nx, nx)
    # cells of the four elements around each free node (i, j), 1 <= i, j <= nx-1
    around = np.stack([lab[:-1, :-1], lab[:-1, 1:], lab[1:, :-1], lab[1:, 1:]], -1)[:, :, :]
    s = np.sort(around.reshape(-1, 4), axis=1)
    mult = 1 + (s[:, 1:] != s[:, :-1]).sum(1)
    q = P.query(level=1)
    assert q["n_sub"][0] == wl.n_sub1 == 4096
    assert q["n_corners"][0] == int((mult >= 3).sum())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pcg_full_size_true_residual(prob, prec):
    wl, P = prob
    P.set_precision(prec)
    b = wl.rhs()
    x, info = P.solve(torch.tensor(b, device="cuda"), rtol=1e-8, maxit=400)
    assert info[0]["status"] == 0
    r = b - _apply_A(wl.nx, wl.k, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - info[0]["relres_true"]) <= 1e-10
    assert info[0]["kappa_est"] <= TAU ** 2


def test_indicator_bound_and_mixed_apply(prob):
    wl, P = prob
    q = P.query(level=1)
    assert q["omega_tilde"] <= TAU ** 2 * (1 + 1e-9)
    r = torch.tensor(inputs.normal_rhs(wl.n_dof, 17), device="cuda")
    P.set_precision("fp64")
    z64 = P.apply(r).cpu().numpy()
    P.set_precision("fp32")
    z32 = P.apply(r).cpu().numpy()
    assert np.linalg.norm(z32 - z64) <= 1e-5 * np.linalg.norm(z64)
