"""Pins for the oracle's adaptive selection (Theorems 1-2, Algorithm 2, eq. 14).

* Brute force on two substructures that both touch the boundary: the pair
  problem is the whole problem, so lambda_max(M A) equals the first local
  eigenvalue, and after adding the n selected constraints it equals
  lambda_{n+1} (Theorem 2, with ||E|| = ||I - E|| for a projection).
* eigh(X, Y) agrees with the explicit Y^{-1/2} X Y^{-1/2} route, and the
  eigenvalues do not depend on the constant a of Theorem 1.
* c^s = -c^t on the shared DOFs before restriction (Sec. 4).
* The reduced edge form (all DOFs but the shared edge eliminated by
  energy minimisation) has the same non-zero eigenvalues and spans the same
  constraints as the literal Theorem 1 form.
* Orthonormalising the kept rows of an edge does not change M^{-1}.
* omega~ <= tau^{L-1} (Theorem 2) and the Lanczos estimate respects it.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import adaptive, bddc, levels, pcg
from paper_0911_5730_gb300 import inputs


def _two_sub(nx=12, seed=0):
    rng = np.random.default_rng(seed)
    k = 10 ** rng.uniform(0, 3, size=nx * nx)
    ej, ei = np.divmod(np.arange(nx * nx), nx)
    return nx, k, (ei >= nx // 2).astype(np.int32)


def _lmax(H):
    A = H.A.toarray()
    M = np.column_stack([H.apply(e) for e in np.eye(H.n)])
    L = np.linalg.cholesky(A)
    return np.linalg.eigvalsh(L.T @ M @ L)[-1]


def test_two_substructure_brute_force():
    nx, k, e2s = _two_sub()
    H0 = bddc.build(nx, k, e2s, 2, 2, "corners")
    lam = None
    lv = H0.bl[0].lv
    (s, t), ed = lv.edges[0]
    pp = adaptive.PairProblem(lv, s, t, ed, lv.schur(s), lv.schur(t), [])
    lam = pp.lam
    assert np.isclose(_lmax(H0), lam[0], rtol=1e-8)
    for tau in (0.5 * (lam[1] + lam[2]), 0.5 * (lam[3] + lam[4])):
        H = bddc.build(nx, k, e2s, 2, 2, "adaptive", tau)
        n = adaptive.select(lam, tau)
        assert H.bl[0].nc == n
        assert np.isclose(_lmax(H), lam[n], rtol=1e-8)


def _pair(nx=16, sub=4, seed=2, which=5):
    e2s, ns = inputs.grid_decomposition(nx, sub)
    k = inputs.channel_coefficient(nx, seed, 0.1, 1e4)
    lv = levels.level_one(nx, k, e2s, ns)
    cd = bddc.corner_dofs(lv)
    (s, t), ed = lv.edges[which]
    return lv, s, t, ed, cd


def test_eigh_independent_route_and_a_independence():
    lv, s, t, ed, cd = _pair()
    Ss, St = lv.schur(s), lv.schur(t)
    pp = adaptive.PairProblem(lv, s, t, ed, Ss, St, cd)
    w, V = np.linalg.eigh(pp.Y)
    Yih = V @ np.diag(w ** -0.5) @ V.T
    lam2 = np.sort(np.linalg.eigvalsh(Yih @ pp.X @ Yih))[::-1]
    assert np.allclose(pp.lam, lam2, atol=1e-9 * pp.lam[0])
    big = pp.lam[pp.lam > 1e-8 * pp.lam[0]]
    for sc in (1e-3, 1e3):
        pq = adaptive.PairProblem(lv, s, t, ed, Ss, St, cd, a_scale=sc)
        assert np.allclose(pq.lam[:len(big)], big, rtol=1e-8)


def test_torn_constraint_blocks_opposite():
    lv, s, t, ed, cd = _pair()
    pp = adaptive.PairProblem(lv, s, t, ed, lv.schur(s), lv.schur(t), cd)
    rows = pp.constraint_rows(3)
    shared = [g for g in pp.Gs if g in set(pp.Gt)]
    ps = [list(pp.Gs).index(g) for g in shared]
    pt = [len(pp.Gs) + list(pp.Gt).index(g) for g in shared]
    assert np.allclose(rows[:, ps], -rows[:, pt], atol=1e-10 * np.abs(rows).max())
    # and the rows vanish off the shared DOFs
    off = np.setdiff1d(np.arange(rows.shape[1]), ps + pt)
    assert np.abs(rows[:, off]).max() <= 1e-10 * np.abs(rows).max()


def reduced_edge_pencil(lv, s, t, ed, Ss, St):
    """Edge-reduced form: keep w_s, w_t on the edge, share the corners,
    minimise the energy over all other interface DOFs."""
    Gs = list(lv.sub_dofs[s][lv.interface_local(s)])
    Gt = list(lv.sub_dofs[t][lv.interface_local(t)])
    shared_c = [g for g in Gs if g in set(Gt) and lv.is_corner[g]]
    def reduce(S, G):
        keep = [G.index(g) for g in ed] + [G.index(g) for g in shared_c]
        oth = [a for a in range(len(G)) if a not in keep]
        Sk = S[np.ix_(keep, keep)]
        if oth:
            Sk = Sk - S[np.ix_(keep, oth)] @ np.linalg.solve(S[np.ix_(oth, oth)], S[np.ix_(oth, keep)])
        return Sk, S[np.ix_(keep[:len(ed)], keep[:len(ed)])]
    Rs, Ss_ee = reduce(Ss, Gs)
    Rt, St_ee = reduce(St, Gt)
    ne, nc = len(ed), len(shared_c)
    M = np.zeros((2 * ne + nc, 2 * ne + nc))
    M[:ne, :ne] = Rs[:ne, :ne]; M[:ne, 2 * ne:] = Rs[:ne, ne:]; M[2 * ne:, :ne] = Rs[ne:, :ne]
    M[ne:2 * ne, ne:2 * ne] = Rt[:ne, :ne]; M[ne:2 * ne, 2 * ne:] = Rt[:ne, ne:]
    M[2 * ne:, ne:2 * ne] = Rt[ne:, :ne]
    M[2 * ne:, 2 * ne:] = Rs[ne:, ne:] + Rt[ne:, ne:]
    if nc:
        Mt = M[:2 * ne, :2 * ne] - M[:2 * ne, 2 * ne:] @ np.linalg.solve(M[2 * ne:, 2 * ne:], M[2 * ne:, :2 * ne])
    else:
        Mt = M[:2 * ne, :2 * ne]
    ds = np.array([lv.A_loc[s][list(lv.sub_dofs[s]).index(g), list(lv.sub_dofs[s]).index(g)] for g in ed])
    dt = np.array([lv.A_loc[t][list(lv.sub_dofs[t]).index(g), list(lv.sub_dofs[t]).index(g)] for g in ed])
    Dls, Dlt = np.diag(ds / (ds + dt)), np.diag(dt / (ds + dt))
    Xd = Dlt @ Ss_ee @ Dlt + Dls @ St_ee @ Dls
    X2 = np.block([[Xd, -Xd], [-Xd, Xd]])
    N = adaptive.null_space_sym(Mt)
    Pb = np.eye(2 * ne) - N @ N.T
    a = np.max(np.diag(Mt))
    Y2 = Pb @ Mt @ Pb + a * (np.eye(2 * ne) - Pb)
    lam, W = sla.eigh(X2, Y2)
    o = np.argsort(lam)[::-1]
    return lam[o], W[:, o], Xd


@pytest.mark.parametrize("which", [0, 5, 11, 17])
def test_reduced_edge_form_matches_literal(which):
    lv, s, t, ed, cd = _pair(which=which)
    Ss, St = lv.schur(s), lv.schur(t)
    pp = adaptive.PairProblem(lv, s, t, ed, Ss, St, cd)
    lam_r, W, Xd = reduced_edge_pencil(lv, s, t, ed, Ss, St)
    big = pp.lam[pp.lam > 1e-8 * pp.lam[0]]
    assert np.allclose(lam_r[:len(big)], big, rtol=1e-9)
    assert np.all(lam_r[len(big):] <= 1e-8 * pp.lam[0])
    k = min(3, len(big))
    lit = pp.constraint_rows(k)[:, pp.edge_pos_s]
    ne = len(ed)
    red = (Xd @ (W[:ne, :k] - W[ne:, :k])).T
    ang = sla.subspace_angles(lit.T, red.T)
    assert np.max(ang) < 1e-7


def test_orthonormalised_rows_do_not_change_preconditioner():
    nx, sub = 16, 4
    e2s, ns = inputs.grid_decomposition(nx, sub)
    k = inputs.channel_coefficient(nx, 2, 0.1, 1e4)
    lv = levels.level_one(nx, k, e2s, ns)
    cd = adaptive.adaptive_dofs(lv, bddc.corner_dofs(lv), 3.0)
    rng = np.random.default_rng(1)
    # rescale and mix the adaptive rows of every edge by a random invertible map
    mixed = [c for c in cd if c.kind == "corner"]
    groups = {}
    for c in cd:
        if c.kind == "adaptive":
            groups.setdefault(c.subs, []).append(c)
    for subs, cs in groups.items():
        R = np.array([c.weights for c in cs])
        T = rng.standard_normal((len(cs), len(cs))) + 3 * np.eye(len(cs))
        for row in T @ R:
            mixed.append(bddc.CoarseDof(cs[0].dofs, row, subs, "adaptive"))
    from oracle.bddc import BDDCLevel, Hierarchy
    H1 = Hierarchy([BDDCLevel(lv, cd)])
    H2 = Hierarchy([BDDCLevel(lv, mixed)])
    r = inputs.normal_rhs(lv.n, 3)
    z1, z2 = H1.apply(r), H2.apply(r)
    assert np.linalg.norm(z1 - z2) <= 1e-12 * np.linalg.norm(z1)


@pytest.mark.parametrize("levels_", [2, 3])
def test_indicator_bound_and_kappa(levels_):
    nx, sub = 32, 4
    e2s, ns = inputs.grid_decomposition(nx, sub)
    s2, n2 = inputs.grid_grouping(nx // sub, 2)
    k = inputs.channel_coefficient(nx, 5, 0.1, 1e5)
    tau = 4.0
    H = bddc.build(nx, k, e2s, ns, levels_, "adaptive", tau, sub1_to_sub2=s2, nsub2=n2)
    assert H.info["omega_tilde"] <= tau ** (levels_ - 1) * (1 + 1e-12)
    res = pcg.pcg(H.A, inputs.normal_rhs(H.n, 1), H.apply)
    assert res.converged
    assert res.kappa <= tau ** (levels_ - 1)
