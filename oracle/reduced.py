"""Level 1 reduced to the interface (the closing remark of Sec. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init``).

Instead of the interior pre-correction (eqs. 4-5) and post-correction
(eqs. 10-11) on level 1, the problem is reduced to the interface once:

* Gamma: the level-1 DOFs in two or more substructures; I: the others (each
  in exactly one substructure);
* S = A_GG - A_GI A_II^{-1} A_IG, applied as the sum over substructures of
  R_i^T S_i R_i with the local Schur complements
  S_i = A_i,GG - A_i,GI A_i,II^{-1} A_i,IG of the unassembled A_i;
* g = f_G - A_GI A_II^{-1} f_I;
* the preconditioner is the rest of Algorithm 1 for a residual that lives on
  Gamma: the substructure corrections (6), the coarse correction (7)-(8) on
  the next level (the full Algorithm 1 there, or the direct solve on the top
  level) and the averaging (9), restricted to Gamma;
* after PCG on S u_G = g: u_I = A_II^{-1} (f_I - A_IG u_G).

The stopping test divides by ||f|| (the full right-hand side): once the
interior is reconstructed the full residual is (0, g - S u_G), so this is the
relative residual of the original system, the quantity Sec. 5 stops on.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .bddc import Hierarchy
from .pcg import PCGResult, pcg


class Reduced:
    def __init__(self, H: Hierarchy):
        self.H = H
        self.L = H.bl[0]
        lv = self.L.lv
        self.G = np.nonzero(lv.is_interface)[0]
        self.I = np.nonzero(~lv.is_interface)[0]

    @property
    def n_gamma(self) -> int:
        return len(self.G)

    def schur_apply(self, uG: np.ndarray) -> np.ndarray:
        """S u_G = sum_i R_i^T S_i R_i u_G, substructure by substructure."""
        lv, L = self.L.lv, self.L
        u = np.zeros(lv.n)
        u[self.G] = uG
        out = np.zeros(lv.n)
        for s in range(lv.nsub):
            dofs = lv.sub_dofs[s]
            A = lv.A_loc[s]
            I = L.I_loc[s]
            Gl = np.setdiff1d(np.arange(len(dofs)), I)
            v = A[np.ix_(Gl, Gl)] @ u[dofs[Gl]]
            if len(I):
                v -= A[np.ix_(Gl, I)] @ sla.cho_solve(L.AII[s], A[np.ix_(I, Gl)] @ u[dofs[Gl]])
            np.add.at(out, dofs[Gl], v)
        return out[self.G]

    def precondition(self, rG: np.ndarray) -> np.ndarray:
        """Eqs. (6)-(9) for a residual on Gamma (no interior corrections)."""
        H, L = self.H, self.L
        r = np.zeros(L.lv.n)
        r[self.G] = rG
        w = [L.substructure_correction(s, r) for s in range(L.lv.nsub)]   # (6)
        rc = L.coarse_rhs(r)                                              # (7), (8)
        if len(H.bl) == 1:
            uc = sla.cho_solve(H.top_chol, rc) if rc.size else rc
        else:
            uc = H.apply(rc, 1)
        return L.average(w, uc)[self.G]                                   # (9)

    def rhs(self, f: np.ndarray) -> np.ndarray:
        """g = f_G - A_GI A_II^{-1} f_I."""
        uI = self.L.interior_solve(f)
        return (f - self.L.lv.A @ uI)[self.G]

    def extend(self, f: np.ndarray, uG: np.ndarray) -> np.ndarray:
        """x = (A_II^{-1} (f_I - A_IG u_G), u_G)."""
        u = np.zeros(self.L.lv.n)
        u[self.G] = uG
        return u + self.L.interior_solve(f - self.L.lv.A @ u)

    def solve(self, f: np.ndarray, rtol: float = 1e-8, maxit: int = 1000) -> tuple[np.ndarray, PCGResult]:
        """PCG on S u_G = g to ||g - S u_G|| <= rtol ||f||; returns the full x."""
        f = np.asarray(f, dtype=np.float64)
        g = self.rhs(f)
        gn = np.linalg.norm(g)
        fn = np.linalg.norm(f)
        op = _Op(self.schur_apply, self.n_gamma)
        tol = rtol * fn / gn if gn > 0 else rtol
        res = pcg(op, g, self.precondition, rtol=tol, maxit=maxit)
        return self.extend(f, res.x), res


class _Op:
    """A linear operator for ``pcg`` (which forms A @ x)."""

    def __init__(self, apply, n):
        self.apply, self.shape = apply, (n, n)

    def __matmul__(self, x):
        return self.apply(x)
