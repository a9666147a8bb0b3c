"""Preconditioned conjugate gradients with the Lanczos condition estimate.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init``).

Sec. 5 runs PCG with the adaptive-multilevel BDDC preconditioner to a
relative residual of 1e-8 and reports iterations and a condition-number
estimate (Tables 1-7).  Readings: x0 = 0; Euclidean norms relative to ||b||;
stop on the recursive residual, then confirm with the true residual and keep
iterating if it is not yet below the tolerance; the estimate is
lambda_max / lambda_min of the Lanczos matrix built from the CG coefficients
(diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    relres: float
    relres_true: float
    kappa: float
    lam_min: float
    lam_max: float
    converged: bool
    alphas: list
    betas: list
    true_checks: int = 0   # true residuals computed: more than one if the stop was deferred


def lanczos_extremes(alphas, betas):
    k = len(alphas)
    if k == 0:
        return 1.0, 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def pcg(A, b: np.ndarray, M, rtol: float = 1e-8, maxit: int = 1000,
        fixed_iters: int | None = None) -> PCGResult:
    """Solve A x = b; M(r) applies the preconditioner.  ``fixed_iters`` runs
    exactly that many iterations (used to compare trajectories)."""
    b = np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    if bn == 0.0:
        return PCGResult(x, 0, 0.0, 0.0, 1.0, 1.0, 1.0, True, [], [])
    z = M(r)
    p = z.copy()
    rho = float(r @ z)
    alphas, betas = [], []
    it = 0
    checks = 0
    converged = False
    limit = fixed_iters if fixed_iters is not None else maxit
    while it < limit:
        it += 1
        q = A @ p
        alpha = rho / float(p @ q)
        x += alpha * p
        r -= alpha * q
        alphas.append(alpha)
        if fixed_iters is None and np.linalg.norm(r) <= rtol * bn:
            checks += 1
            if np.linalg.norm(b - A @ x) <= rtol * bn:
                converged = True
                break
        if it == limit:
            break
        z = M(r)
        rho_new = float(r @ z)
        beta = rho_new / rho
        betas.append(beta)
        p = z + beta * p
        rho = rho_new
    lo, hi = lanczos_extremes(alphas, betas)
    rr = float(np.linalg.norm(r) / bn)
    rt = float(np.linalg.norm(b - A @ x) / bn)
    if fixed_iters is not None:
        converged = rt <= rtol
    return PCGResult(x, it, rr, rt, hi / lo, lo, hi, converged, alphas, betas, checks)
