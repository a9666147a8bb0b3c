"""Adaptive selection of edge coarse DOFs: Theorem 1, Theorem 2, Algorithm 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init``).

For every edge shared by substructures s and t of a level (Sec. 3):

* the pair space holds [w_s; w_t] on the whole interfaces Gamma_s, Gamma_t,
  with S^{st} = blockdiag(S_s, S_t) the Schur complements of A_s, A_t;
* E^{st} averages the DOFs shared by s and t with the pair-local weights
  d_s / (d_s + d_t) (so that E^{st} R^{st} = I, Sec. 5) and is the identity
  elsewhere;
* C^{st} holds the initial constraints shared by s and t (the corners);
* Pi is the orthogonal projection onto null C^{st}(I - E^{st}), Pi-bar removes
  null S^{st} intersected with range Pi, built from a null-space basis Z
  (Sec. 3, after Theorem 1);
* X = Pi (I-E)^T S (I-E) Pi and
  Y = Pi-bar (Pi S Pi + a (I - Pi)) Pi-bar + a (I - Pi-bar)   (eq. 13);
* Theorem 2: the eigenvectors with lambda > tau give the new constraints
  c_k = w_k^T Pi (I-E)^T S (I-E) Pi (eq. 14); the block of s restricted to
  the edge's own DOFs is kept, and the indicator of the edge is the first
  eigenvalue not removed.

Readings: n^{st} = #{lambda_k > tau} (strict, Theorem 2); a = max diag S^{st};
the kept rows of one edge are orthonormalised (a change of basis of the same
constraint space); Z is the numerical null space of each S_i.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .bddc import CoarseDof
from .levels import Level

NULL_TOL = 1e-10
NULL_RANK_TOL = 1e-6
DROP_TOL = 1e-12


def _orth_rows(K: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """Orthonormal basis (as columns) of the row space of K."""
    if K.size == 0:
        return np.zeros((K.shape[1], 0))
    U, sv, Vt = np.linalg.svd(K, full_matrices=False)
    if sv.size == 0 or sv[0] == 0:
        return np.zeros((K.shape[1], 0))
    r = int(np.sum(sv > tol * sv[0]))
    return Vt[:r].T


def null_space_sym(S: np.ndarray) -> np.ndarray:
    """Numerical null space of a symmetric positive semidefinite matrix."""
    lam, V = np.linalg.eigh(S)
    if lam.size == 0:
        return V
    return V[:, lam < NULL_TOL * max(lam[-1], 1e-300)]


class PairProblem:
    """Literal Theorem 1 for the edge shared by substructures s and t."""

    def __init__(self, lv: Level, s: int, t: int, edge_dofs: np.ndarray,
                 S_s: np.ndarray, S_t: np.ndarray, cdofs: list[CoarseDof], a_scale: float = 1.0):
        self.s, self.t = s, t
        Gs = lv.sub_dofs[s][lv.interface_local(s)]
        Gt = lv.sub_dofs[t][lv.interface_local(t)]
        ns_, nt_ = len(Gs), len(Gt)
        n = ns_ + nt_
        self.Gs, self.Gt = Gs, Gt
        pos_s = {g: a for a, g in enumerate(Gs)}
        pos_t = {g: ns_ + a for a, g in enumerate(Gt)}
        S = np.zeros((n, n))
        S[:ns_, :ns_] = S_s
        S[ns_:, ns_:] = S_t
        # Pair-local averaging E^{st} (weights from the diagonals of A_s, A_t).
        diag_s = dict(zip(lv.sub_dofs[s], np.diag(lv.A_loc[s])))
        diag_t = dict(zip(lv.sub_dofs[t], np.diag(lv.A_loc[t])))
        E = np.eye(n)
        shared = [g for g in Gs if g in pos_t]
        for g in shared:
            ps, pt = pos_s[g], pos_t[g]
            ds, dt = diag_s[g], diag_t[g]
            ws, wt = ds / (ds + dt), dt / (ds + dt)
            E[ps, ps], E[ps, pt] = ws, wt
            E[pt, ps], E[pt, pt] = ws, wt
        IE = np.eye(n) - E
        # Initial constraints shared by s and t.
        rows = []
        for cd in cdofs:
            if s in cd.subs and t in cd.subs:
                rs = np.zeros(n); rt = np.zeros(n)
                for g, wgt in zip(cd.dofs, cd.weights):
                    rs[pos_s[g]] += wgt
                    rt[pos_t[g]] += wgt
                rows += [rs, rt]
        C = np.array(rows) if rows else np.zeros((0, n))
        K = C @ IE
        V = _orth_rows(K)
        Pi = np.eye(n) - V @ V.T
        # Null space of S^{st} and the part of it inside range Pi.
        Zs, Zt = null_space_sym(S_s), null_space_sym(S_t)
        Z = np.zeros((n, Zs.shape[1] + Zt.shape[1]))
        Z[:ns_, :Zs.shape[1]] = Zs
        Z[ns_:, Zs.shape[1]:] = Zt
        if Z.shape[1]:
            # Z has orthonormal columns, so a combination that leaves range Pi
            # has (I - Pi) Z c of order one; the computed null vectors are only
            # accurate to eps ||S|| / gap (about 1e-9 at a coefficient contrast
            # of 1e6), hence the loose rank cut.
            M = (np.eye(n) - Pi) @ Z
            _, sv, Vt = np.linalg.svd(M)
            rank = int(np.sum(sv > NULL_RANK_TOL))
            cnull = Vt[rank:].T
            N = _orth_rows((Pi @ Z @ cnull).T) if cnull.shape[1] else np.zeros((n, 0))
        else:
            N = np.zeros((n, 0))
        Pib = np.eye(n) - N @ N.T
        a = a_scale * float(np.max(np.diag(S)))
        Xhat = IE.T @ S @ IE
        X = Pi @ Xhat @ Pi
        Y = Pib @ (Pi @ S @ Pi + a * (np.eye(n) - Pi)) @ Pib + a * (np.eye(n) - Pib)
        X = 0.5 * (X + X.T)
        Y = 0.5 * (Y + Y.T)
        lam, W = sla.eigh(X, Y)
        order = np.argsort(lam)[::-1]
        self.lam = lam[order]
        self.W = W[:, order]
        self.X, self.Y, self.Pi, self.Pib, self.S, self.E, self.N = X, Y, Pi, Pib, S, E, N
        self.Xhat = Xhat
        self.edge_pos_s = np.array([pos_s[g] for g in edge_dofs])
        self.edge_pos_t = np.array([pos_t[g] for g in edge_dofs])
        self.edge_dofs = edge_dofs

    def constraint_rows(self, k: int) -> np.ndarray:
        """c_k = w_k^T Pi (I-E)^T S (I-E) Pi for the first k eigenvectors (eq. 14)."""
        return (self.X @ self.W[:, :k]).T


def select(lam: np.ndarray, tau: float) -> int:
    """n^{st}: how many eigenvalues exceed tau (Theorem 2)."""
    return int(np.sum(lam > tau))


def adaptive_dofs(lv: Level, initial: list[CoarseDof], tau: float,
                  report: dict | None = None, a_scale: float = 1.0) -> list[CoarseDof]:
    """Algorithm 2 on one level: corners plus the selected edge constraints."""
    S = [lv.schur(s) for s in range(lv.nsub)]
    out = list(initial)
    omega_max = 0.0
    reps = []
    for ie, ((s, t), edofs) in enumerate(lv.edges):
        pp = PairProblem(lv, s, t, edofs, S[s], S[t], initial, a_scale)
        nst = select(pp.lam, tau)
        omega = float(pp.lam[nst]) if nst < len(pp.lam) else 0.0
        omega_max = max(omega_max, omega)
        kept = 0
        if nst:
            rows = pp.constraint_rows(nst)[:, pp.edge_pos_s]      # block s, edge DOFs only
            Q, R = np.linalg.qr(rows.T)
            d = np.abs(np.diag(R))
            keep = d > DROP_TOL * d.max() if d.size else np.zeros(0, bool)
            cs = np.unique(lv.comp[edofs])
            comp = int(cs[0]) if len(cs) == 1 else -1        # mixed components: -1
            for j in np.nonzero(keep)[0]:
                out.append(CoarseDof(edofs.copy(), Q[:, j].copy(), (s, t), "adaptive", comp))
                kept += 1
        reps.append({"pair": (s, t), "n_edge": len(edofs), "lam": pp.lam.copy(),
                     "n_sel": nst, "n_kept": kept, "omega": omega,
                     "ambiguous": bool(np.any(np.abs(pp.lam / tau - 1.0) < 1e-9))
                     if np.isfinite(tau) else False})
    if report is not None:
        report["omega_max"] = omega_max
        report["edges"] = reps
    return out
