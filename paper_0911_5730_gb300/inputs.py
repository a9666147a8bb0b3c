"""Seeded synthetic workloads for the 2D Q1 diffusion model problem.

This module only draws inputs: coefficient fields, decompositions and
right-hand sides.  It holds none of the BDDC arithmetic, so both the CPU
oracle and the CUDA path may import it.

Conventions (shared by every consumer):

* The domain is the unit square with ``nx * nx`` square Q1 elements, h = 1/nx.
* Element ``(ei, ej)`` covers ``[ei h, (ei+1) h] x [ej h, (ej+1) h]`` and has
  flat index ``e = ej * nx + ei``; per-element arrays are length ``nx*nx``.
* Node ``(i, j)`` sits at ``(i h, j h)``.  Nodes on the boundary carry the
  zero Dirichlet condition; free node ``(i, j)``, ``1 <= i, j <= nx-1``, has
  global index ``g = (j-1)(nx-1) + (i-1)``.
* A decomposition is ``elem_to_sub`` (level-1 substructure of every element)
  and, for three levels, ``sub1_to_sub2`` (level-2 substructure of every
  level-1 substructure).

The named workloads follow the paper's model problem (Sec. 2: P1/Q1 elements,
zero Dirichlet data) and the two-/three-level experiments of Sec. 5, with the
scalar coefficient fields described in each function.
"""
from __future__ import annotations

import dataclasses
import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def grid_decomposition(nx: int, sub_elems: int) -> tuple[np.ndarray, int]:
    """Square ``sub_elems x sub_elems`` element blocks; subs numbered row-major."""
    if nx % sub_elems:
        raise ValueError("nx must be a multiple of the substructure size")
    ns = nx // sub_elems
    ej, ei = np.divmod(np.arange(nx * nx), nx)
    sub = (ej // sub_elems) * ns + (ei // sub_elems)
    return sub.astype(np.int32), ns * ns


def grid_grouping(n_sub_side: int, group: int) -> tuple[np.ndarray, int]:
    """Group a row-major ``n x n`` grid of substructures into ``group x group`` blocks."""
    if n_sub_side % group:
        raise ValueError("substructure grid must be a multiple of the group size")
    ng = n_sub_side // group
    sj, si = np.divmod(np.arange(n_sub_side * n_sub_side), n_sub_side)
    return ((sj // group) * ng + (si // group)).astype(np.int32), ng * ng


def constant_coefficient(nx: int, value: float = 1.0) -> np.ndarray:
    return np.full(nx * nx, value, dtype=np.float64)


def channel_coefficient(nx: int, seed: int, frac: float = 0.10,
                        high: float = 1e6) -> np.ndarray:
    """Full-length, one-element-wide horizontal and vertical channels of ``high``.

    Element rows and columns are drawn uniformly without replacement,
    alternating horizontal / vertical, until at least ``frac`` of the elements
    carry the high coefficient; all other elements have k = 1.
    """
    rng = _rng(seed)
    rows = rng.permutation(nx)
    cols = rng.permutation(nx)
    k = np.ones((nx, nx))           # k[ej, ei]
    ir = ic = 0
    horizontal = True
    while (k == high).mean() < frac:
        if horizontal:
            k[rows[ir], :] = high
            ir += 1
        else:
            k[:, cols[ic]] = high
            ic += 1
        horizontal = not horizontal
    return k.reshape(-1)


def block_log_uniform_coefficient(nx: int, block: int, seed: int,
                                  lo: float = 0.0, hi: float = 6.0) -> np.ndarray:
    """log10 k drawn uniform in [lo, hi], constant on ``block x block`` element blocks."""
    if nx % block:
        raise ValueError("nx must be a multiple of the block size")
    nb = nx // block
    rng = _rng(seed)
    logk = rng.uniform(lo, hi, size=(nb, nb))   # [bj, bi]
    k = 10.0 ** np.repeat(np.repeat(logk, block, axis=0), block, axis=1)
    return k.reshape(-1)


def normal_rhs(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """i.i.d. N(0,1) load vector(s) over the free DOFs in g-order."""
    rng = _rng(seed)
    if nrhs is None:
        return rng.standard_normal(n)
    return rng.standard_normal((nrhs, n))


def unit_load_rhs(nx: int) -> np.ndarray:
    """Load vector of f = 1 for Q1 on a uniform square mesh: h^2 at every free node.

    Each free node touches four elements and the bilinear hat function
    integrates to h^2/4 on each of them.
    """
    h = 1.0 / nx
    return np.full((nx - 1) * (nx - 1), h * h)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    k: np.ndarray
    elem_to_sub: np.ndarray
    n_sub1: int
    levels: int
    tau: float
    constraints: str               # "corners", "corners+edges", "adaptive", "all"
    sub1_to_sub2: np.ndarray | None = None
    n_sub2: int = 0
    rhs_seed: int | None = None

    @property
    def n_dof(self) -> int:
        return (self.nx - 1) ** 2

    def rhs(self, nrhs: int | None = None) -> np.ndarray:
        if self.rhs_seed is None:
            b = unit_load_rhs(self.nx)
            return b if nrhs is None else np.tile(b, (nrhs, 1))
        return normal_rhs(self.n_dof, self.rhs_seed, nrhs)


def two_level_unit(nx: int = 32, sub: int = 8, constraints: str = "corners+edges") -> Workload:
    """32x32 mesh, k = 1, 4x4 substructures (H/h = 8), f = 1."""
    e2s, ns = grid_decomposition(nx, sub)
    return Workload("two_level_unit_%d" % nx, nx, constant_coefficient(nx), e2s, ns,
                    2, np.inf, constraints)


def two_level_channels(nx: int = 512, sub: int = 16, tau: float = 10.0,
                       seed: int = 2001, rhs_seed: int = 2002) -> Workload:
    """512x512 mesh, 32x32 substructures (H/h = 16), k = 1e6 on random channels."""
    e2s, ns = grid_decomposition(nx, sub)
    return Workload("two_level_channels_%d" % nx, nx, channel_coefficient(nx, seed), e2s, ns,
                    2, tau, "adaptive", rhs_seed=rhs_seed)


def three_level_blocks(nx: int = 1024, sub: int = 8, group: int = 8, tau: float = 10.0,
                       seed: int = 3001, rhs_seed: int = 3002) -> Workload:
    """1024x1024 mesh, 128x128 substructures (H/h = 8) grouped 8x8 on level 2."""
    e2s, ns = grid_decomposition(nx, sub)
    s2, n2 = grid_grouping(nx // sub, group)
    return Workload("three_level_blocks_%d" % nx, nx,
                    block_log_uniform_coefficient(nx, 8, seed), e2s, ns,
                    3, tau, "adaptive", s2, n2, rhs_seed=rhs_seed)
