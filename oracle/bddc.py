"""Coarse degrees of freedom, coarse basis, multilevel hierarchy, Algorithm 1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init``).

Sec. 2: the local coarse DOFs of substructure i are C_i w_i; a global coarse
DOF is a row of Q_P^T, i.e. a functional on the global DOFs (here: a list of
DOFs with weights), and R_c,i picks the global coarse DOFs that touch i.  The
space W~ holds the functions whose coarse DOFs take a common value in every
substructure that shares them (Sec. 2; for functionals along an edge this is
the continuity reading of eq. 3, which is exactly the augmentation of
Theorem 2).

Sec. 2.1: the coarse basis functions are energy minimal with one coarse DOF
equal to one and the others zero; they are the shape functions of the level
l + 1 elements, whose element matrices are Psi_i^T A_i Psi_i.  Level l + 1
substructures agglomerate those elements.  The last level L is solved
directly (Algorithm 1, Algorithm 2).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .levels import Level


@dataclasses.dataclass
class CoarseDof:
    """One global coarse DOF: the functional u -> sum_k weights[k] * u[dofs[k]].

    ``comp`` is the displacement component it measures (-1: mixed) and
    ``bnd`` whether it is a point value on the boundary of the domain; both
    carry over to the DOFs of the next level."""
    dofs: np.ndarray
    weights: np.ndarray
    subs: tuple
    kind: str
    comp: int = 0
    bnd: bool = False


def corner_dofs(lv: Level) -> list[CoarseDof]:
    return [CoarseDof(np.array([g]), np.array([1.0]), lv.subs_of[g], "corner",
                      int(lv.comp[g]), bool(lv.bnd[g]))
            for g in lv.corners]


def edge_average_dofs(lv: Level) -> list[CoarseDof]:
    """One arithmetic average per edge and displacement component over the
    edge's non-corner DOFs (Table 1, c+e: 13818 - 4794 = 2 averages on each
    of the 2 * 48 * 47 edges)."""
    out = []
    for pair, d in lv.edges:
        for c in np.unique(lv.comp[d]):
            sel = d[lv.comp[d] == c]
            out.append(CoarseDof(sel, np.full(len(sel), 1.0 / len(sel)), pair, "edge", int(c)))
    return out


def all_interface_dofs(lv: Level) -> list[CoarseDof]:
    """Every interface DOF is a coarse DOF: then W~ = U and BDDC is exact."""
    return [CoarseDof(np.array([g]), np.array([1.0]), lv.subs_of[g], "all",
                      int(lv.comp[g]), bool(lv.bnd[g]))
            for g in np.nonzero(lv.is_interface)[0]]


class BDDCLevel:
    """Per-substructure operators of one BDDC level (Sec. 2, 2.1)."""

    def __init__(self, lv: Level, cdofs: list[CoarseDof]):
        self.lv = lv
        self.cdofs = cdofs
        self.nc = len(cdofs)
        ns = lv.nsub
        by_sub = [[] for _ in range(ns)]
        for q, cd in enumerate(cdofs):
            for s in cd.subs:
                by_sub[s].append(q)
        self.Rc, self.C, self.Psi, self.Ac, self.saddle, self.AII = [], [], [], [], [], []
        self.I_loc = []
        for s in range(ns):
            dofs = lv.sub_dofs[s]
            loc = {g: a for a, g in enumerate(dofs)}
            qs = np.array(sorted(by_sub[s]), dtype=np.int64)
            C = np.zeros((len(qs), len(dofs)))
            for r, q in enumerate(qs):
                cd = cdofs[q]
                for g, wgt in zip(cd.dofs, cd.weights):
                    C[r, loc[g]] += wgt
            A = lv.A_loc[s]
            n, m = len(dofs), len(qs)
            K = np.zeros((n + m, n + m))
            K[:n, :n] = A
            K[:n, n:] = C.T
            K[n:, :n] = C
            lu = sla.lu_factor(K)
            # Coarse basis: [A C^T; C 0][Psi; Lambda] = [0; I] (energy minimal,
            # unit value of one coarse DOF, zero of the others).
            rhs = np.zeros((n + m, m))
            rhs[n:, :] = np.eye(m)
            Psi = sla.lu_solve(lu, rhs)[:n] if m else np.zeros((n, 0))
            self.Rc.append(qs)
            self.C.append(C)
            self.Psi.append(Psi)
            self.Ac.append(Psi.T @ A @ Psi)
            self.saddle.append(lu)
            I = lv.interior_local(s)
            self.I_loc.append(I)
            self.AII.append(sla.cho_factor(A[np.ix_(I, I)]) if len(I) else None)

    def assembled_coarse(self) -> np.ndarray:
        """A_c = sum_i R_c,i^T (Psi_i^T A_i Psi_i) R_c,i (dense)."""
        Ac = np.zeros((self.nc, self.nc))
        for q, a in zip(self.Rc, self.Ac):
            Ac[np.ix_(q, q)] += a
        return Ac

    def next_level(self, sub_to_next, nsub_next: int) -> Level:
        """Level l+1: level-l substructures become elements (Sec. 2.1)."""
        return Level(self.nc, self.Rc, self.Ac, sub_to_next, nsub_next,
                     [cd.comp for cd in self.cdofs], [cd.bnd for cd in self.cdofs])

    # -- pieces of Algorithm 1 -----------------------------------------------------
    def interior_solve(self, r: np.ndarray) -> np.ndarray:
        """u_I in U_I with a(u_I, z_I) = <r, z_I>: one SPD solve per substructure."""
        u = np.zeros(self.lv.n)
        for s in range(self.lv.nsub):
            I = self.I_loc[s]
            if len(I):
                g = self.lv.sub_dofs[s][I]
                u[g] = sla.cho_solve(self.AII[s], r[g])
        return u

    def substructure_correction(self, s: int, rB: np.ndarray) -> np.ndarray:
        """w_Delta,i: a(w, z) = <r_B, E z> on {C_i w = 0} (eq. 6), one substructure."""
        dofs = self.lv.sub_dofs[s]
        f = self.lv.D[s] * rB[dofs]
        n, m = len(dofs), len(self.Rc[s])
        return sla.lu_solve(self.saddle[s], np.concatenate([f, np.zeros(m)]))[:n]

    def coarse_rhs(self, rB: np.ndarray) -> np.ndarray:
        """r_{l+1} = sum_i R_c,i^T Psi_i^T D_i R_i r_B (eqs. 7-8)."""
        rc = np.zeros(self.nc)
        for s in range(self.lv.nsub):
            f = self.lv.D[s] * rB[self.lv.sub_dofs[s]]
            np.add.at(rc, self.Rc[s], self.Psi[s].T @ f)
        return rc

    def average(self, w: list, uc: np.ndarray) -> np.ndarray:
        """u_B = E (w_Delta + u_{l+1}) = sum_i R_i^T D_i (w_i + Psi_i R_c,i u_c) (eq. 9)."""
        u = np.zeros(self.lv.n)
        for s in range(self.lv.nsub):
            v = w[s] + self.Psi[s] @ uc[self.Rc[s]]
            np.add.at(u, self.lv.sub_dofs[s], self.lv.D[s] * v)
        return u


class Hierarchy:
    """BDDC levels 1..L-1 and the directly factored level L."""

    def __init__(self, bl: list[BDDCLevel], info: dict | None = None):
        self.bl = bl
        self.top = bl[-1].assembled_coarse()
        self.top_chol = sla.cho_factor(self.top) if self.top.size else None
        self.info = info or {}

    @property
    def A(self):
        return self.bl[0].lv.A

    @property
    def n(self) -> int:
        return self.bl[0].lv.n

    def apply(self, r: np.ndarray, level: int = 0) -> np.ndarray:
        """Algorithm 1 on level ``level`` + 1 (0-based here), recursively."""
        L = self.bl[level]
        lv = L.lv
        uI = L.interior_solve(r)                                   # (4)
        rB = r - lv.A @ uI                                         # (5)
        w = [L.substructure_correction(s, rB) for s in range(lv.nsub)]   # (6)
        rc = L.coarse_rhs(rB)                                      # (7), (8)
        if level == len(self.bl) - 1:
            uc = sla.cho_solve(self.top_chol, rc) if rc.size else rc
        else:
            uc = self.apply(rc, level + 1)
        uB = L.average(w, uc)                                      # (9)
        vI = L.interior_solve(lv.A @ uB)                           # (10)
        return uI + uB - vI                                        # (11)


def coarse_dofs_for(lv: Level, mode: str, tau: float = np.inf, report: dict | None = None):
    """Coarse DOFs of one level for the constraint modes of Tables 1-7."""
    if mode == "corners":
        return corner_dofs(lv)
    if mode == "corners+edges":
        return corner_dofs(lv) + edge_average_dofs(lv)
    if mode == "all":
        return all_interface_dofs(lv)
    if mode == "adaptive":
        from .adaptive import adaptive_dofs
        return adaptive_dofs(lv, corner_dofs(lv), tau, report)
    raise ValueError(mode)


def build(nx: int, k, elem_to_sub, nsub1: int, levels: int = 2, mode: str = "corners",
          tau: float = np.inf, sub1_to_sub2=None, nsub2: int = 0,
          modes: list | None = None, problem: str = "diffusion", lame=(1.0, 2.0),
          clamp: str = "left") -> Hierarchy:
    """Set up the hierarchy of Algorithm 2 for the Q1 model problem, or for
    plane elasticity (``problem="elasticity"``, Lame parameters k_e * lame,
    clamped as ``clamp`` says).

    ``modes`` overrides ``mode`` per BDDC level (used by the consistency pins).
    """
    from .levels import level_one, level_one_elasticity
    modes = modes or [mode] * (levels - 1)
    if problem == "elasticity":
        lv = level_one_elasticity(nx, k, elem_to_sub, nsub1, lame[0], lame[1], clamp)
    else:
        lv = level_one(nx, k, elem_to_sub, nsub1)
    bls, info = [], {"omega": [], "edge_reports": []}
    groupings = [(sub1_to_sub2, nsub2)]
    for l in range(levels - 1):
        rep = {}
        cd = coarse_dofs_for(lv, modes[l], tau, rep)
        info["omega"].append(rep.get("omega_max", None))
        info["edge_reports"].append(rep.get("edges", []))
        bl = BDDCLevel(lv, cd)
        bls.append(bl)
        if l < levels - 2:
            to_next, nnext = groupings[l]
            lv = bl.next_level(to_next, nnext)
    info["n_coarse"] = [b.nc for b in bls]
    om = [o for o in info["omega"] if o is not None]
    info["omega_tilde"] = float(np.prod(om)) if om else None
    return Hierarchy(bls, info)


def build_workload(wl, **kw) -> Hierarchy:
    problem = getattr(wl, "problem", "diffusion")
    if problem == "elasticity":
        kw.setdefault("problem", "elasticity")
        kw.setdefault("lame", wl.lame)
        kw.setdefault("clamp", wl.clamp)
    if getattr(wl, "constraints_level2", None) and wl.levels == 3:
        kw.setdefault("modes", [wl.constraints, wl.constraints_level2])
    return build(wl.nx, wl.k, wl.elem_to_sub, wl.n_sub1, wl.levels, wl.constraints,
                 wl.tau, wl.sub1_to_sub2, wl.n_sub2, **kw)
