"""Pins of the oracle's interface-reduced solve (oracle/reduced.py), each
against something other than the reduced code itself:

* S applied substructure by substructure equals the dense Schur complement
  A_GG - A_GI A_II^-1 A_IG of the assembled global matrix;
* the preconditioned reduced operator M_G S has exactly the non-unit
  eigenvalues of Algorithm 1's preconditioned operator M A (dense, both sides
  built column by column), and M_G is symmetric;
* with every interface DOF a coarse constraint the preconditioner is S^-1:
  one iteration;
* the reduced solve reaches a sparse direct solve's solution, and its PCG
  takes as many iterations as the full PCG with Algorithm 1.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import bddc as obddc
from oracle import pcg as opcg
from oracle.reduced import Reduced
from paper_0911_5730_gb300 import inputs

WL = {
    "unit_c+e": inputs.two_level_unit(),
    "unit_all": inputs.two_level_unit(constraints="all"),
    "channels_64": inputs.two_level_channels(nx=64, sub=16),
    "three_level_64": inputs.three_level_blocks(nx=64, sub=8, group=4, tau=10.0),
    "voronoi_64": inputs.three_level_voronoi(nx=64, cells=4, group=2, levels=2),
}
_cache = {}


def _reduced(name):
    if name not in _cache:
        _cache[name] = Reduced(obddc.build_workload(WL[name]))
    return _cache[name]


def _dense(A):
    return A.toarray() if hasattr(A, "toarray") else np.asarray(A)


@pytest.mark.parametrize("name", ["unit_c+e", "channels_64", "voronoi_64"])
def test_schur_apply_equals_dense_schur(name):
    R = _reduced(name)
    A = _dense(R.H.A)
    G, I = R.G, R.I
    S = A[np.ix_(G, G)] - A[np.ix_(G, I)] @ np.linalg.solve(A[np.ix_(I, I)], A[np.ix_(I, G)])
    u = np.random.default_rng(5).standard_normal(len(G))
    assert np.linalg.norm(R.schur_apply(u) - S @ u) <= 1e-13 * np.linalg.norm(S @ u)


def test_spectrum_matches_algorithm_1():
    R = _reduced("unit_c+e")
    H = R.H
    A = _dense(H.A)
    n, ng = A.shape[0], R.n_gamma
    M = np.column_stack([H.apply(e) for e in np.eye(n)])
    MG = np.column_stack([R.precondition(e) for e in np.eye(ng)])
    MS = np.column_stack([R.precondition(R.schur_apply(e)) for e in np.eye(ng)])
    assert np.linalg.norm(MG - MG.T) <= 1e-13 * np.linalg.norm(MG)
    ef = np.sort(np.linalg.eigvals(M @ A).real)
    er = np.sort(np.linalg.eigvals(MS).real)
    nf, nr = ef[np.abs(ef - 1) > 1e-9], er[np.abs(er - 1) > 1e-9]
    assert len(nf) == len(nr) > 10
    assert np.max(np.abs(nf - nr)) <= 1e-10
    assert np.all(er >= 1 - 1e-10)            # BDDC: lambda_min >= 1


def test_all_interface_constraints_one_iteration():
    R = _reduced("unit_all")
    b = WL["unit_all"].rhs()
    x, res = R.solve(b, rtol=1e-10)
    assert res.iters == 1
    A = R.H.A
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["channels_64", "three_level_64", "voronoi_64"])
def test_reduced_solve_direct_and_iterations(name):
    R = _reduced(name)
    wl = WL[name]
    b = wl.rhs()
    A = R.H.A
    xd = spla.spsolve(A.tocsc(), b) if hasattr(A, "tocsc") else np.linalg.solve(A, b)
    x, res = R.solve(b, rtol=1e-13, maxit=500)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    x8, res8 = R.solve(b, rtol=1e-8)
    full = opcg.pcg(A, b, R.H.apply, rtol=1e-8)
    assert res8.converged and res8.iters == full.iters
    assert np.linalg.norm(b - A @ x8) <= 1e-8 * np.linalg.norm(b)
