"""One decomposition level: substructures, interface, corners, edges, weights.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init``).

A level is given the way Sec. 2.1 describes every level: a set of global
degrees of freedom, "elements" that each own a list of those DOFs and a
symmetric positive semidefinite element matrix, and an assignment of elements
to substructures.  On level 1 the elements are the Q1 elements; on level
l + 1 they are the level-l substructures with their coarse matrices, so the
same code serves every level.

Readings of the paper used here:
* A DOF is on the interface when it belongs to two or more substructures;
  otherwise it is interior (the space U_I of Sec. 2).
* A corner is a DOF in three or more substructures (Sec. 2: substructure
  vertices; on level >= 2 the level-1 corners shared by >= 3 level-2
  substructures, Sec. 2.1, Sec. 4 "variable number of nodes per element"),
  or an interface DOF on the boundary of the domain (where an edge meets a
  traction-free side; the counts of Tables 1-2, e.g. 4794 = 2 (49^2 - 4)
  for 48 x 48 substructures, include those vertices).  With zero Dirichlet
  data on the whole boundary, as in the diffusion problem, no such DOF
  exists.
* An edge is a connected chain of non-corner interface DOFs shared by the
  same pair of substructures (Sec. 3: adjacent substructures share an edge).
* The averaging weights are the standard stiffness scaling named in Sec. 1:
  delta_i(j) = (A_i)_jj / sum_k (A_k)_jj over the substructures k holding j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from . import fem


class Level:
    """``dof_comp``: displacement component of each DOF (0 for a scalar
    problem); ``dof_bnd``: the DOF lies on the boundary of the domain."""

    def __init__(self, n: int, elem_dofs, elem_mats, elem_sub, nsub: int,
                 dof_comp=None, dof_bnd=None):
        self.n = int(n)
        self.comp = np.zeros(self.n, np.int64) if dof_comp is None else np.asarray(dof_comp, np.int64)
        self.bnd = np.zeros(self.n, bool) if dof_bnd is None else np.asarray(dof_bnd, bool)
        self.elem_dofs = [np.asarray(d, dtype=np.int64) for d in elem_dofs]
        self.elem_mats = [np.asarray(m, dtype=np.float64) for m in elem_mats]
        self.elem_sub = np.asarray(elem_sub, dtype=np.int64)
        self.nsub = int(nsub)
        self._build_substructures()
        self._classify()
        self._weights()

    # -- substructure matrices A_i (unassembled Neumann matrices) ---------------
    def _build_substructures(self):
        n, ns = self.n, self.nsub
        members = [[] for _ in range(ns)]
        for e, s in enumerate(self.elem_sub):
            members[s].append(e)
        self.sub_elems = members
        self.sub_dofs = []
        self.A_loc = []
        for s in range(ns):
            dofs = np.unique(np.concatenate([self.elem_dofs[e] for e in members[s]]
                                            + [np.zeros(0, np.int64)]))
            loc = {g: a for a, g in enumerate(dofs)}
            A = np.zeros((len(dofs), len(dofs)))
            for e in members[s]:
                idx = [loc[g] for g in self.elem_dofs[e]]
                A[np.ix_(idx, idx)] += self.elem_mats[e]
            self.sub_dofs.append(dofs)
            self.A_loc.append(A)
        subs_of = [[] for _ in range(n)]
        for s in range(ns):
            for g in self.sub_dofs[s]:
                subs_of[g].append(s)
        self.subs_of = [tuple(x) for x in subs_of]
        self.mult = np.array([len(x) for x in subs_of])
        self.A = fem.assemble(n, self.elem_dofs, self.elem_mats)

    # -- interface, corners and edges -------------------------------------------
    def _classify(self):
        self.is_interface = self.mult >= 2
        self.is_corner = (self.mult >= 3) | (self.is_interface & self.bnd)
        # DOF adjacency: two DOFs are neighbours when an element holds both.
        rows, cols = [], []
        for d in self.elem_dofs:
            if len(d):
                rr, cc = np.meshgrid(d, d, indexing="ij")
                rows.append(rr.ravel()); cols.append(cc.ravel())
        adj = sp.csr_matrix((np.ones(sum(len(r) for r in rows)),
                             (np.concatenate(rows), np.concatenate(cols))),
                            shape=(self.n, self.n)) if rows else sp.csr_matrix((self.n, self.n))
        groups = {}
        for g in np.nonzero(self.is_interface & ~self.is_corner)[0]:
            groups.setdefault(self.subs_of[g], []).append(g)
        edges = []
        for pair in sorted(groups):
            dofs = np.array(sorted(groups[pair]))
            sub = adj[dofs][:, dofs]
            ncomp, lab = csg.connected_components(sub, directed=False)
            for c in range(ncomp):
                edges.append((pair, dofs[lab == c]))
        self.edges = edges                      # list of ((s, t), dofs)
        self.corners = np.nonzero(self.is_corner)[0]

    def interior_local(self, s: int) -> np.ndarray:
        return np.nonzero(~self.is_interface[self.sub_dofs[s]])[0]

    def interface_local(self, s: int) -> np.ndarray:
        return np.nonzero(self.is_interface[self.sub_dofs[s]])[0]

    # -- stiffness scaling -------------------------------------------------------
    def _weights(self):
        diag_sum = np.zeros(self.n)
        for s in range(self.nsub):
            np.add.at(diag_sum, self.sub_dofs[s], np.diag(self.A_loc[s]))
        self.D = []
        for s in range(self.nsub):
            d = np.diag(self.A_loc[s]) / diag_sum[self.sub_dofs[s]]
            d[~self.is_interface[self.sub_dofs[s]]] = 1.0
            self.D.append(d)

    def schur(self, s: int) -> np.ndarray:
        """S_s: Schur complement of A_s on all of its interface DOFs."""
        A = self.A_loc[s]
        I, G = self.interior_local(s), self.interface_local(s)
        if len(I) == 0:
            return A[np.ix_(G, G)].copy()
        AII = A[np.ix_(I, I)]
        return A[np.ix_(G, G)] - A[np.ix_(G, I)] @ np.linalg.solve(AII, A[np.ix_(I, G)])


def level_one(nx: int, k, elem_to_sub, nsub: int) -> Level:
    dofs, mats = fem.level1_elements(nx, np.asarray(k, dtype=np.float64))
    return Level((nx - 1) ** 2, dofs, mats, elem_to_sub, nsub)


def level_one_elasticity(nx: int, k, elem_to_sub, nsub: int, lam: float = 1.0, mu: float = 2.0,
                         clamp: str = "left") -> Level:
    dofs, mats, n, comp, bnd, coords = fem.elasticity_elements(
        nx, np.asarray(k, dtype=np.float64), lam, mu, clamp)
    lv = Level(n, dofs, mats, elem_to_sub, nsub, comp, bnd)
    lv.coords = coords
    return lv
