"""Pins for the oracle's Algorithm 1 and PCG (Sec. 2, 2.1, 5).

* Exactness: with every interface DOF a coarse DOF, W~ = U and the
  preconditioner is A^{-1} (M A = I; PCG converges in one iteration); the
  same with a single substructure.  This fails on any dropped term, wrong
  sign or transposed operand in eqs. (4)-(11).
* Multilevel consistency: three levels whose level-2 coarse DOFs are all
  level-2 interface DOFs equal two levels (the level-2 solve is exact).
* The preconditioner is symmetric, and the spectrum of M A is real with
  lambda_min >= 1 (the BDDC lower bound).
* The PCG solution matches a sparse direct solve; the Lanczos estimate lies
  inside the true spectrum of M A.
* Coarse basis: the coarse basis functions have unit / zero coarse DOFs and
  Psi_i^T A_i Psi_i equals -Lambda_i of the saddle-point solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

from oracle import bddc, pcg
from paper_0911_5730_gb300 import inputs


def _dense_M(H):
    n = H.n
    return np.column_stack([H.apply(e) for e in np.eye(n)])


def _problem(nx=16, sub=4, seed=5, kind="blocks"):
    e2s, ns = inputs.grid_decomposition(nx, sub)
    if kind == "blocks":
        k = inputs.block_log_uniform_coefficient(nx, sub, seed, 0.0, 3.0)
    elif kind == "channels":
        k = inputs.channel_coefficient(nx, seed, 0.1, 1e4)
    else:
        k = np.ones(nx * nx)
    return nx, k, e2s, ns


@pytest.mark.parametrize("levels", [2, 3])
def test_all_interface_is_exact(levels):
    nx, k, e2s, ns = _problem()
    s2, n2 = inputs.grid_grouping(nx // 4, 2)
    H = bddc.build(nx, k, e2s, ns, levels, "all", sub1_to_sub2=s2, nsub2=n2)
    A = H.A.toarray()
    M = _dense_M(H)
    assert np.linalg.norm(M @ A - np.eye(H.n)) <= 1e-10 * np.linalg.norm(np.eye(H.n))
    b = inputs.normal_rhs(H.n, 11)
    res = pcg.pcg(H.A, b, H.apply)
    assert res.iters == 1


def test_single_substructure_is_exact():
    nx = 8
    k = inputs.channel_coefficient(nx, 1, 0.1, 1e3)
    H = bddc.build(nx, k, np.zeros(nx * nx, np.int32), 1, 2, "corners")
    M = _dense_M(H)
    assert np.allclose(M @ H.A.toarray(), np.eye(H.n), atol=1e-10)


def test_three_level_with_exact_level_two_equals_two_level():
    nx, k, e2s, ns = _problem(nx=24, sub=4)
    s2, n2 = inputs.grid_grouping(nx // 4, 3)
    H2 = bddc.build(nx, k, e2s, ns, 2, "corners+edges")
    H3 = bddc.build(nx, k, e2s, ns, 3, modes=["corners+edges", "all"], sub1_to_sub2=s2, nsub2=n2)
    r = inputs.normal_rhs(H2.n, 4)
    z2, z3 = H2.apply(r), H3.apply(r)
    assert np.linalg.norm(z2 - z3) <= 1e-12 * np.linalg.norm(z2)


@pytest.mark.parametrize("levels,mode", [(2, "corners"), (2, "corners+edges"), (2, "adaptive"),
                                         (3, "corners"), (3, "adaptive")])
def test_symmetric_and_lower_bound(levels, mode):
    nx, k, e2s, ns = _problem(nx=16, sub=4, kind="channels")
    s2, n2 = inputs.grid_grouping(nx // 4, 2)
    H = bddc.build(nx, k, e2s, ns, levels, mode, tau=3.0, sub1_to_sub2=s2, nsub2=n2)
    M = _dense_M(H)
    assert np.linalg.norm(M - M.T) <= 1e-12 * np.linalg.norm(M)
    A = H.A.toarray()
    # M A is similar to A^{1/2} M A^{1/2}: real spectrum, >= 1
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ M @ L)
    assert ev[0] >= 1.0 - 1e-10
    b = inputs.normal_rhs(H.n, 8)
    res = pcg.pcg(H.A, b, H.apply, rtol=1e-8)
    assert res.converged
    assert res.lam_min >= ev[0] * (1 - 1e-8) and res.lam_max <= ev[-1] * (1 + 1e-8)
    assert res.kappa >= 0.5 * ev[-1] / ev[0]


@pytest.mark.parametrize("mode", ["corners", "corners+edges", "adaptive"])
def test_pcg_matches_direct_solve(mode):
    nx, k, e2s, ns = _problem(nx=32, sub=8, kind="channels")
    H = bddc.build(nx, k, e2s, ns, 2, mode, tau=10.0)
    b = inputs.normal_rhs(H.n, 9)
    res = pcg.pcg(H.A, b, H.apply, rtol=1e-13, maxit=500)
    x = spl.spsolve(H.A.tocsc(), b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)


def test_coarse_basis_definition():
    nx, k, e2s, ns = _problem(nx=16, sub=4)
    H = bddc.build(nx, k, e2s, ns, 2, "corners+edges")
    bl = H.bl[0]
    for s in range(ns):
        C, Psi, A = bl.C[s], bl.Psi[s], bl.lv.A_loc[s]
        assert np.allclose(C @ Psi, np.eye(C.shape[0]), atol=1e-10)
        n, m = A.shape[0], C.shape[0]
        K = np.block([[A, C.T], [C, np.zeros((m, m))]])
        sol = np.linalg.solve(K, np.vstack([np.zeros((n, m)), np.eye(m)]))
        assert np.allclose(bl.Ac[s], -sol[n:], atol=1e-9 * np.abs(bl.Ac[s]).max())


def test_lanczos_estimate_exact_on_diagonal():
    # CG on a diagonal matrix with all eigenvalues excited recovers them exactly.
    d = np.array([1.0, 2.0, 5.0, 11.0])
    res = pcg.pcg(np.diag(d), np.ones(4), lambda r: r.copy(), rtol=1e-14, maxit=4)
    assert np.isclose(res.lam_min, 1.0, rtol=1e-10) and np.isclose(res.lam_max, 11.0, rtol=1e-10)


# Irregular substructures (config 4's Voronoi cells, small): the same pins.
def _voronoi(nx=32, cells=4, group=2, seed=4001):
    e2s, ns, s2, n2 = inputs.voronoi_decomposition(nx, cells, seed, group=group)
    k = inputs.block_log_uniform_coefficient(nx, 4, seed + 1, 0.0, 3.0)
    return nx, k, e2s, ns, s2, n2


@pytest.mark.parametrize("levels", [2, 3])
def test_voronoi_all_interface_is_exact(levels):
    nx, k, e2s, ns, s2, n2 = _voronoi()
    H = bddc.build(nx, k, e2s, ns, levels, "all", sub1_to_sub2=s2, nsub2=n2)
    M = _dense_M(H)
    assert np.linalg.norm(M @ H.A.toarray() - np.eye(H.n)) <= 1e-10 * np.sqrt(H.n)


@pytest.mark.parametrize("levels", [2, 3])
def test_voronoi_adaptive_symmetric_bounded_and_direct(levels):
    nx, k, e2s, ns, s2, n2 = _voronoi()
    tau = 10.0
    H = bddc.build(nx, k, e2s, ns, levels, "adaptive", tau=tau, sub1_to_sub2=s2, nsub2=n2)
    M = _dense_M(H)
    assert np.linalg.norm(M - M.T) <= 1e-12 * np.linalg.norm(M)
    A = H.A.toarray()
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ M @ L)
    assert ev[0] >= 1.0 - 1e-10
    # Lemma 1 / Theorem 2: the indicator and the condition number are bounded
    # by tau^(L-1) by construction of the adaptive constraints
    assert H.info["omega_tilde"] <= tau ** (levels - 1) * (1 + 1e-9)
    assert ev[-1] / ev[0] <= tau ** (levels - 1)
    b = inputs.normal_rhs(H.n, 12)
    res = pcg.pcg(H.A, b, H.apply, rtol=1e-13, maxit=500)
    x = spl.spsolve(H.A.tocsc(), b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)
