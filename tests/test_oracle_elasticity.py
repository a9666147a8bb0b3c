"""Pins for the oracle's plane-elasticity problem (the setting of the paper's
experiments, Sec. 5: lambda = 1, mu = 2; Tables 1-2 for the counts).

Checked against what mathematics and the paper fix, not against the oracle:
* element: the energy of every linear displacement field equals the closed
  form lam (div u)^2 + 2 mu |eps(u)|^2 over the unit square (patch test: pins
  the material matrix and the strain operator), the three rigid motions are
  its null space and nothing else is (rank 5: no hourglass modes);
* assembly and numbering: A Z = 0 for the rigid motions on the unclamped
  mesh, and for a homogeneous field u = x (a, c) (zero on the clamped side)
  A u vanishes at every node inside the square (discrete equilibrium of a
  constant stress);
* the paper's constraint counts, from the oracle's own classification of the
  paper's decomposition (48 x 48 substructures, counted on the whole node set
  as the paper's DOF count 1 182 722 = 2 * 769^2 does): 4794 corners and
  13818 with edge averages (Table 1), +24 and +48 on a 3 x 3 level-2 grid
  (Table 2).  The counts do not depend on H/h, so H/h = 2 keeps this cheap;
* with the clamped side removed: the closed form 2 ((N+1)^2 - 4 - (N-1)) for
  the corners of an N x N grid;
* the null space of a floating substructure's Schur complement is spanned by
  the rigid motions (three of them);
* BDDC: every interface DOF constrained gives M^{-1} = A^{-1} (2 and 3
  levels); M^{-1} is symmetric with eigenvalues of M^{-1} A >= 1 (2 and 3
  levels); scaling the material by c scales M^{-1} by exactly 1 / c and
  keeps the selected constraints; two levels
  with an exact level 2 equal the two-level method; PCG reaches the direct
  solution; adaptive selection meets kappa <= tau (Theorem 2) and
  omega~ <= tau^2 on three levels;
* brute force on two substructures: the pair problem is the whole problem,
  so lambda_max(M^{-1} A) is the first local eigenvalue and, after the n
  selected constraints, the (n+1)-st;
* Table 3's observation: the jagged edge carries the large local
  eigenvalues, the regular edges stay in the paper's range; Tables 4-5 on
  level 2: the jagged level-2 edge dominates, and level-2 eigenvalues grow
  as level 1 is constrained more tightly;
* the reading the GPU edge solver implements: the reduced edge form has the
  literal form's eigenvalues, and its null space is exactly the rigid
  motions on the edge when both substructures float (none otherwise); on
  level 2 exactly the coarse values of the rigid motions.
"""
import functools

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import adaptive, bddc, fem, levels, pcg
from paper_0911_5730_gb300 import inputs

LAM, MU = 1.0, 2.0


@functools.lru_cache(maxsize=None)
def _three_level(tau):
    """128^2 mesh, 16 x 16 level-1 substructures, 2 x 2 on level 2 with the
    comb between level-2 substructures 1 and 3; adaptive on both levels."""
    wl = inputs.elasticity(nx=128, sub=8, levels=3, group=8, constraints="adaptive", tau=tau)
    return bddc.build_workload(wl)


def test_element_patch_test_rigid_modes_rank():
    K = fem.elasticity_reference_stiffness(LAM, MU)
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    rng = np.random.default_rng(1)
    for _ in range(5):
        a, b, c, d, e, f = rng.standard_normal(6)
        u = np.zeros(8)
        u[0::2] = a * X[:, 0] + b * X[:, 1] + e
        u[1::2] = c * X[:, 0] + d * X[:, 1] + f
        energy = LAM * (a + d) ** 2 + 2 * MU * (a * a + d * d + 0.5 * (b + c) ** 2)
        assert np.isclose(u @ K @ u, energy, rtol=1e-13)
    Z = fem.rigid_modes(np.repeat(X, 2, axis=0), np.tile([0, 1], 4))
    assert np.abs(K @ Z).max() < 1e-14
    assert np.allclose(K, K.T)
    lam = np.linalg.eigvalsh(K)
    assert np.all(lam[:3] < 1e-13) and lam[3] > 1.0


def test_assembled_rigid_null_and_equilibrium():
    nx = 8
    k = np.ones(nx * nx)
    dofs, mats, n, comp, bnd, xy = fem.elasticity_elements(nx, k, LAM, MU, "none")
    A = fem.assemble(n, dofs, mats)
    assert np.abs(A @ fem.rigid_modes(xy, comp)).max() < 1e-12
    dofs, mats, n, comp, bnd, xy = fem.elasticity_elements(nx, k, LAM, MU, "left")
    A = fem.assemble(n, dofs, mats)
    assert n == inputs.elasticity_n_dof(nx) == 2 * nx * (nx + 1)
    u = np.where(comp == 0, 0.7 * xy[:, 0], -0.3 * xy[:, 0])
    r = A @ u
    inside = ~bnd
    assert np.abs(r[inside]).max() < 1e-12
    assert np.abs(r[bnd]).max() > 1e-3        # tractions act only on the boundary


def test_paper_constraint_counts_tables_1_and_2():
    nx = 96                                    # 48 x 48 substructures, H/h = 2
    e2s, ns = inputs.grid_decomposition(nx, 2)
    s2, n2 = inputs.grid_grouping(48, 16)      # 3 x 3 level-2 substructures
    out = {}
    for mode in ("corners", "corners+edges"):
        lv = levels.level_one_elasticity(nx, np.ones(nx * nx), e2s, ns, LAM, MU, clamp="none")
        bl = bddc.BDDCLevel(lv, bddc.coarse_dofs_for(lv, mode))
        lv2 = bl.next_level(s2, n2)
        out[mode] = (bl.nc, len(bddc.coarse_dofs_for(lv2, mode)))
    assert out["corners"] == (4794, 24)          # Table 1 "c", Table 2 "4794 + 24"
    assert out["corners+edges"] == (13818, 48)   # Table 1 "c+e", Table 2 "13818 + 48"


@pytest.mark.parametrize("N,sub", [(4, 8), (6, 4)])
def test_clamped_counts_closed_form(N, sub):
    nx = N * sub
    e2s, ns = inputs.grid_decomposition(nx, sub)
    lv = levels.level_one_elasticity(nx, np.ones(nx * nx), e2s, ns, LAM, MU, clamp="left")
    corners = 2 * ((N + 1) ** 2 - 4 - (N - 1))
    assert len(lv.corners) == corners
    assert len(bddc.edge_average_dofs(lv)) == 2 * 2 * N * (N - 1)


def test_floating_null_space_is_rigid():
    nx, sub = 16, 4
    e2s, ns = inputs.grid_decomposition(nx, sub)
    lv = levels.level_one_elasticity(nx, np.ones(nx * nx), e2s, ns, LAM, MU)
    s = 5                                     # not touching x = 0: floating
    G = lv.sub_dofs[s][lv.interface_local(s)]
    N0 = adaptive.null_space_sym(lv.schur(s))
    Z = fem.rigid_modes(lv.coords[G], lv.comp[G])
    assert N0.shape[1] == 3
    Q, _ = np.linalg.qr(Z)
    assert np.allclose(Q @ (Q.T @ N0), N0, atol=1e-9)
    assert adaptive.null_space_sym(lv.schur(0)).shape[1] == 0   # clamped on x = 0


def _M(H):
    return np.column_stack([H.apply(e) for e in np.eye(H.n)])


@pytest.mark.parametrize("lev", [2, 3])
def test_all_interface_is_exact(lev):
    wl = inputs.elasticity(nx=16, sub=4, levels=lev, group=2, constraints="all", jagged=False)
    H = bddc.build_workload(wl)
    b = wl.rhs()
    x = spla.spsolve(H.A.tocsc(), b)
    assert np.linalg.norm(H.apply(b) - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("lev,mode", [(2, "corners"), (2, "corners+edges"), (2, "adaptive"),
                                      (3, "corners+edges"), (3, "adaptive")])
def test_symmetric_and_lower_bound(lev, mode):
    wl = inputs.elasticity(nx=16, sub=4, levels=lev, group=2, constraints=mode, tau=3.0, jagged=False)
    H = bddc.build_workload(wl)
    M = _M(H)
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    A = H.A.toarray()
    L = np.linalg.cholesky(A)
    lam = np.linalg.eigvalsh(L.T @ M @ L)
    assert lam[0] >= 1 - 1e-10


def test_three_level_with_exact_level_two_equals_two_level():
    wl = inputs.elasticity(nx=16, sub=4, levels=2, constraints="corners+edges", jagged=False)
    H2 = bddc.build_workload(wl)
    wl3 = inputs.elasticity(nx=16, sub=4, levels=3, group=2, constraints="corners+edges",
                            constraints_level2="all", jagged=False)
    H3 = bddc.build_workload(wl3)
    b = inputs.normal_rhs(wl.n_dof, 5)
    z2, z3 = H2.apply(b), H3.apply(b)
    assert np.linalg.norm(z3 - z2) <= 1e-11 * np.linalg.norm(z2)


@pytest.mark.parametrize("lev,tau", [(2, 10.0), (2, 3.0), (3, 3.0)])
def test_adaptive_bound_and_direct_solution(lev, tau):
    wl = inputs.elasticity(nx=32, sub=8, levels=lev, group=2, constraints="adaptive", tau=tau)
    H = bddc.build_workload(wl)
    b = wl.rhs()
    res = pcg.pcg(H.A, b, H.apply, rtol=1e-10, maxit=300)
    x = spla.spsolve(H.A.tocsc(), b)
    assert res.converged
    assert np.linalg.norm(res.x - x) <= 1e-8 * np.linalg.norm(x)
    om = H.info["omega_tilde"]
    assert om <= tau ** (lev - 1) * (1 + 1e-12)
    assert res.kappa <= tau ** (lev - 1) * (1 + 1e-6)
    # the jagged edge is the one that needs extra constraints
    reps = H.info["edge_reports"][0]
    sel = [r["pair"] for r in reps if r["n_sel"] > 0]
    assert (1, 5) in sel


def test_two_substructure_brute_force():
    nx = 8
    e2s = (np.arange(nx * nx) % nx >= nx // 2).astype(np.int32)    # left | right
    k = 10 ** np.random.default_rng(3).uniform(0, 2, nx * nx)
    H0 = bddc.build(nx, k, e2s, 2, 2, "corners", problem="elasticity")
    lv = H0.bl[0].lv
    (s, t), ed = lv.edges[0]
    pp = adaptive.PairProblem(lv, s, t, ed, lv.schur(s), lv.schur(t), bddc.corner_dofs(lv))
    lam = pp.lam

    def lmax(H):
        A = H.A.toarray()
        L = np.linalg.cholesky(A)
        return np.linalg.eigvalsh(L.T @ _M(H) @ L)[-1]

    assert np.isclose(lmax(H0), lam[0], rtol=1e-8)
    for tau in (0.5 * (lam[1] + lam[2]), 0.5 * (lam[3] + lam[4])):
        H = bddc.build(nx, k, e2s, 2, 2, "adaptive", tau, problem="elasticity")
        n = adaptive.select(lam, tau)
        assert H.bl[0].nc == len(bddc.corner_dofs(lv)) + n
        assert np.isclose(lmax(H), lam[n], rtol=1e-8)


def test_jagged_edge_dominates_local_eigenvalues():
    """Table 3's observation: the jagged edge carries the large eigenvalues
    (the paper's pair (2, 50): 24.3 ... 13.1 over its first eight, the regular
    pairs 3.4-12.6 at most).  On a 4 x 4 grid of H/h = 16 substructures with
    the comb between substructures 1 and 5, the jagged edge's fourth
    eigenvalue exceeds the first eigenvalue of every regular edge, and those
    stay within the paper's range."""
    wl = inputs.elasticity(nx=64, sub=16, levels=2, constraints="adaptive", tau=10.0)
    H = bddc.build_workload(wl)
    reps = H.info["edge_reports"][0]
    jag = [r for r in reps if r["pair"] == (1, 5)][0]
    reg = [r["lam"][0] for r in reps if r["pair"] != (1, 5)]
    assert jag["lam"][3] > max(reg)
    assert 3.0 < min(reg) and max(reg) < 13.0
    assert jag["n_sel"] >= 4 and all(r["n_sel"] <= 1 for r in reps if r["pair"] != (1, 5))


def test_jagged_level_two_edge_tables_4_and_5():
    """Tables 4-5's observations on level 2: the jagged level-2 edge has the
    largest local eigenvalue and needs the most constraints, and the level-2
    eigenvalues grow when level 1 is constrained more tightly (the paper's
    jagged pair: 23.2 at tau = 10, 84.3 at tau = 2).  128^2 mesh, 16 x 16
    level-1 substructures, 2 x 2 on level 2 with the comb between level-2
    substructures 1 and 3."""
    top = {}
    for tau in (10.0, 2.0):
        H = _three_level(tau)
        reps = H.info["edge_reports"][1]
        jag = [r for r in reps if r["pair"] == (1, 3)][0]
        others = [r for r in reps if r["pair"] != (1, 3)]
        assert jag["lam"][0] > max(r["lam"][0] for r in others)
        assert jag["n_sel"] >= max(r["n_sel"] for r in others)
        assert H.info["omega_tilde"] <= tau ** 2 * (1 + 1e-12)
        top[tau] = jag["lam"][0]
    assert top[2.0] > top[10.0]


def _reduced_mt(lv, s, t, ed, Ss, St):
    """The reduced edge matrix: every interface DOF of s and t but the edge
    eliminated by energy minimisation, the shared corners one unknown, then
    eliminated too."""
    Gs = list(lv.sub_dofs[s][lv.interface_local(s)])
    Gt = list(lv.sub_dofs[t][lv.interface_local(t)])
    shared = [g for g in Gs if g in set(Gt) and lv.is_corner[g]]

    def red(S, G):
        keep = [G.index(g) for g in ed] + [G.index(g) for g in shared]
        oth = [a for a in range(len(G)) if a not in keep]
        return S[np.ix_(keep, keep)] - S[np.ix_(keep, oth)] @ np.linalg.solve(S[np.ix_(oth, oth)], S[np.ix_(oth, keep)])

    Rs, Rt = red(Ss, Gs), red(St, Gt)
    ne, nc = len(ed), len(shared)
    M = np.zeros((2 * ne + nc, 2 * ne + nc))
    M[:ne, :ne], M[:ne, 2 * ne:], M[2 * ne:, :ne] = Rs[:ne, :ne], Rs[:ne, ne:], Rs[ne:, :ne]
    M[ne:2 * ne, ne:2 * ne], M[ne:2 * ne, 2 * ne:], M[2 * ne:, ne:2 * ne] = Rt[:ne, :ne], Rt[:ne, ne:], Rt[ne:, :ne]
    M[2 * ne:, 2 * ne:] = Rs[ne:, ne:] + Rt[ne:, ne:]
    if nc == 0:
        return M[:2 * ne, :2 * ne]
    return M[:2 * ne, :2 * ne] - M[:2 * ne, 2 * ne:] @ np.linalg.solve(M[2 * ne:, 2 * ne:], M[2 * ne:, :2 * ne])


@pytest.mark.parametrize("pair", [(5, 6), (5, 9), (0, 1), (1, 5)])
def test_reduced_edge_form_projects_the_rigid_motions(pair):
    """The GPU solves the edge problem in its reduced form (every interface
    DOF but the edge eliminated by energy minimisation, the shared corners as
    one unknown) and projects out the rigid motions restricted to the edge,
    the same on both sides, when both substructures float (Sec. 3: null S is
    in the range of the rigid-body modes).  Here: the reduced form's non-zero
    eigenvalues equal the literal Theorem 1 form's, and the numerical null
    space of the reduced matrix is exactly the span of [z_E; z_E] for the
    three rigid motions z (floating pairs) or empty (a clamped substructure)."""
    from test_oracle_adaptive import reduced_edge_pencil
    wl = inputs.elasticity(nx=64, sub=16, levels=2, constraints="corners")
    lv = levels.level_one_elasticity(64, wl.k, wl.elem_to_sub, wl.n_sub1)
    cd = bddc.corner_dofs(lv)
    (s, t), ed = [(p, d) for p, d in lv.edges if p == pair][0]
    Ss, St = lv.schur(s), lv.schur(t)
    pp = adaptive.PairProblem(lv, s, t, ed, Ss, St, cd)
    lam_r, W, Xd = reduced_edge_pencil(lv, s, t, ed, Ss, St)
    big = pp.lam[pp.lam > 1e-8 * pp.lam[0]]
    assert np.allclose(lam_r[:len(big)], big, rtol=1e-8)
    Mt = _reduced_mt(lv, s, t, ed, Ss, St)
    N = adaptive.null_space_sym(Mt)
    floating = s % 4 != 0 and t % 4 != 0          # column 0 touches the clamped side
    if not floating:
        assert N.shape[1] == 0
        return
    zE = fem.rigid_modes(lv.coords[ed], lv.comp[ed])
    Z = np.vstack([zE, zE])
    assert N.shape[1] == 3
    assert np.max(sla.subspace_angles(N, Z)) < 1e-6


@pytest.mark.parametrize("pair", [(1, 3), (0, 1)])
def test_level_two_edge_null_space_is_the_coarse_rigid_motions(pair):
    """On level 2 the null vectors are the coarse values of the rigid
    motions, sum_k w_k z(dof_k) for every level-1 coarse DOF (Sec. 3: the
    coarse basis functions span the rigid-body modes): the reduced level-2
    edge matrix of a floating pair (the jagged one, level-2 substructures 1
    and 3) has exactly that null space, a pair with a clamped substructure
    none."""
    H = _three_level(10.0)
    lv1, lv2 = H.bl[0].lv, H.bl[1].lv
    Z1 = fem.rigid_modes(lv1.coords, lv1.comp)
    Zc = np.array([cd.weights @ Z1[cd.dofs] for cd in H.bl[0].cdofs])
    (s, t), ed = [(p, d) for p, d in lv2.edges if p == pair][0]
    Mt = _reduced_mt(lv2, s, t, ed, lv2.schur(s), lv2.schur(t))
    N = adaptive.null_space_sym(Mt)
    if 0 in pair or 2 in pair:                    # column 0 of the 2 x 2 grid: clamped
        assert N.shape[1] == 0
        return
    Z = np.vstack([Zc[ed], Zc[ed]])
    assert N.shape[1] == 3
    assert np.max(sla.subspace_angles(N, Z)) < 1e-6


@pytest.mark.parametrize("lev", [2, 3])
def test_material_scaling_scales_the_preconditioner(lev):
    """A = sum_e k_e K_e is linear in the Lame parameters, and every BDDC
    ingredient (interior solves, weights, coarse basis, adaptive selection)
    is invariant under a common factor except the solves, which scale by its
    inverse: with (lambda, mu) -> c (lambda, mu), M^{-1} -> M^{-1} / c and the
    selected constraints stay the same."""
    base = dict(nx=32, sub=8, levels=lev, group=2, constraints="adaptive", tau=3.0)
    H1 = bddc.build_workload(inputs.elasticity(**base))
    H7 = bddc.build_workload(inputs.elasticity(lame=(7.0, 14.0), **base))
    b = inputs.normal_rhs(H1.n, 23)
    z1, z7 = H1.apply(b), H7.apply(b)
    assert np.linalg.norm(7.0 * z7 - z1) <= 1e-11 * np.linalg.norm(z1)
    assert [r["n_sel"] for r in H1.info["edge_reports"][0]] == [r["n_sel"] for r in H7.info["edge_reports"][0]]
