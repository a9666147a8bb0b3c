"""Seeded synthetic workloads for the 2D Q1 diffusion model problem and for
plane linear elasticity (the problem of the paper's experiments, Sec. 5).

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


def voronoi_decomposition(nx: int, cells: int, seed: int, jitter: float = 0.25,
                          group: int = 0) -> tuple[np.ndarray, int, np.ndarray | None, int]:
    """Irregular substructures: a seeded Voronoi partition of the elements.

    ``cells x cells`` seeds sit on a lattice of boxes of ``nx / cells``
    elements, each moved uniformly by up to ``jitter`` box widths in x and y
    (so every seed stays inside its own box).  Every element goes to the seed
    nearest its centroid (ties to the lower seed index; only the 5 x 5 boxes
    around an element can hold its nearest seed).  A cell whose elements fall
    apart (connectivity across element edges) keeps its largest piece; every
    other piece joins the neighbouring cell it shares the most element edges
    with, repeatedly, until every cell is connected.  Empty cells are dropped
    and the rest renumbered in seed order.

    With ``group > 0`` the level-2 substructure of a cell is the ``group x
    group`` block of lattice boxes holding its seed.

    Returns ``(elem_to_sub, n_sub, sub1_to_sub2 or None, n_sub2)``.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    if nx % cells:
        raise ValueError("nx must be a multiple of the number of cells per side")
    w = nx // cells
    rng = _rng(seed)
    off = rng.uniform(-jitter, jitter, size=(cells * cells, 2))
    ia, ib = np.meshgrid(np.arange(cells), np.arange(cells))        # [b, a]
    sx = (ia.reshape(-1) + 0.5 + off[:, 0]) * w                    # seed s = b * cells + a
    sy = (ib.reshape(-1) + 0.5 + off[:, 1]) * w
    ei, ej = np.meshgrid(np.arange(nx), np.arange(nx))              # [ej, ei]
    cx, cy = (ei + 0.5).reshape(-1), (ej + 0.5).reshape(-1)
    ba, bb = (ei // w).reshape(-1), (ej // w).reshape(-1)
    best = np.full(nx * nx, np.inf)
    arg = np.full(nx * nx, -1, dtype=np.int64)
    for db in range(-2, 3):
        for da in range(-2, 3):
            a2, b2 = ba + da, bb + db
            ok = (a2 >= 0) & (a2 < cells) & (b2 >= 0) & (b2 < cells)
            sidx = np.where(ok, b2 * cells + a2, 0)
            d = np.where(ok, (cx - sx[sidx]) ** 2 + (cy - sy[sidx]) ** 2, np.inf)
            take = (d < best) | ((d == best) & (sidx < arg))
            best = np.where(take, d, best)
            arg = np.where(take, sidx, arg)
    lab = arg.reshape(nx, nx)                                       # [ej, ei]

    def pieces(lab):
        idx = np.arange(nx * nx).reshape(nx, nx)
        h = lab[:, 1:] == lab[:, :-1]
        v = lab[1:, :] == lab[:-1, :]
        r = np.concatenate([idx[:, :-1][h], idx[:-1, :][v]])
        c = np.concatenate([idx[:, 1:][h], idx[1:, :][v]])
        g = coo_matrix((np.ones(r.size), (r, c)), shape=(nx * nx, nx * nx))
        return connected_components(g, directed=False)[1].reshape(nx, nx)

    shifts = (((slice(None), slice(1, None)), (slice(None), slice(None, -1))),
              ((slice(None), slice(None, -1)), (slice(None), slice(1, None))),
              ((slice(1, None), slice(None)), (slice(None, -1), slice(None))),
              ((slice(None, -1), slice(None)), (slice(1, None), slice(None))))
    while True:
        comp = pieces(lab)
        flat_l, flat_c = lab.reshape(-1), comp.reshape(-1)
        size = np.bincount(flat_c)
        first = np.full(size.size, -1, dtype=np.int64)
        first[flat_c[::-1]] = np.arange(flat_c.size)[::-1]         # an element of each piece
        cell_of = flat_l[first]
        main = {}                                                  # cell -> its largest piece
        for cpt in np.lexsort((np.arange(size.size), -size)):
            main.setdefault(int(cell_of[cpt]), int(cpt))
        is_main = np.zeros(size.size, dtype=bool)
        is_main[list(main.values())] = True
        frag = [cpt for cpt in range(size.size) if not is_main[cpt]]
        if not frag:
            break
        moved = False
        for cpt in frag:
            mask = comp == cpt
            cnt = {}
            for sl_a, sl_b in shifts:
                # element edges from the piece to the main piece of another cell
                m = mask[sl_a] & is_main[comp[sl_b]] & (lab[sl_b] != cell_of[cpt])
                for nb in lab[sl_b][m]:
                    cnt[int(nb)] = cnt.get(int(nb), 0) + 1
            if cnt:
                lab[mask] = min(cnt, key=lambda c: (-cnt[c], c))
                moved = True
        if not moved:
            raise RuntimeError("Voronoi fragments with no neighbouring main piece")
    used = np.unique(lab)
    renum = np.full(cells * cells, -1, dtype=np.int64)
    renum[used] = np.arange(used.size)
    e2s = renum[lab].reshape(-1).astype(np.int32)
    if group <= 0:
        return e2s, int(used.size), None, 0
    if cells % group:
        raise ValueError("cells must be a multiple of the group size")
    ng = cells // group
    s2 = ((used // cells) // group * ng + (used % cells) // group).astype(np.int32)
    return e2s, int(used.size), s2, ng * ng


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


def elasticity_n_dof(nx: int, clamp: str = "left") -> int:
    """Free DOFs of the plane elasticity problem: two per node, the nodes on
    the clamped side x = 0 removed (``clamp="left"``) or none (``"none"``)."""
    return 2 * (nx + 1) * (nx if clamp == "left" else nx + 1)


def body_force_rhs(nx: int, clamp: str = "left", f=(0.0, -1.0)) -> np.ndarray:
    """Load vector of a constant body force f for bilinear elements: every
    element adds f h^2 / 4 to each of its four nodes (the integral of a hat
    function over one element).  DOF order: 2 * node + component, node
    numbering as in ``elasticity`` workloads."""
    h = 1.0 / nx
    cnt = np.zeros((nx + 1, nx + 1))                   # [j, i]: elements touching node (i, j)
    cnt[:-1, :-1] += 1; cnt[:-1, 1:] += 1; cnt[1:, :-1] += 1; cnt[1:, 1:] += 1
    if clamp == "left":
        cnt = cnt[:, 1:]
    w = (cnt * (h * h / 4.0)).reshape(-1)
    b = np.empty(2 * w.size)
    b[0::2] = f[0] * w
    b[1::2] = f[1] * w
    return b


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
    # "diffusion": scalar -div(k grad u) = f, zero Dirichlet data on the whole
    # boundary.  "elasticity": plane strain with Lame parameters k_e * lame,
    # clamped on x = 0 (``clamp``), traction free elsewhere.
    problem: str = "diffusion"
    lame: tuple = (1.0, 2.0)
    clamp: str = "left"
    constraints_level2: str | None = None

    @property
    def n_dof(self) -> int:
        if self.problem == "elasticity":
            return elasticity_n_dof(self.nx, self.clamp)
        return (self.nx - 1) ** 2

    def rhs(self, nrhs: int | None = None) -> np.ndarray:
        if self.rhs_seed is None:
            b = body_force_rhs(self.nx, self.clamp) if self.problem == "elasticity" else unit_load_rhs(self.nx)
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


def three_level_voronoi(nx: int = 2048, cells: int = 64, group: int = 8, tau: float = 10.0,
                        part_seed: int = 4001, coef_seed: int = 4002, rhs_seed: int = 4003,
                        jitter: float = 0.25, levels: int = 3) -> Workload:
    """2048x2048 mesh cut into 64x64 seeded Voronoi cells (about 700-1600 DOFs
    each at jitter 0.25), grouped by 8x8 lattice blocks of seeds into 64
    level-2 substructures; log10 k uniform in [0, 6] per 8x8-element block
    (not aligned with the cells)."""
    e2s, ns, s2, n2 = voronoi_decomposition(nx, cells, part_seed, jitter,
                                            group if levels == 3 else 0)
    return Workload("three_level_voronoi_%d" % nx if levels == 3 else "two_level_voronoi_%d" % nx,
                    nx, block_log_uniform_coefficient(nx, 8, coef_seed), e2s, ns, levels, tau,
                    "adaptive", s2, n2, rhs_seed=rhs_seed)



def jagged_grid_decomposition(nx: int, sub: int, pair=(1, 0), amp: int = 2, period: int = 2):
    """A grid of ``sub x sub`` element blocks with one jagged edge.

    The horizontal edge above substructure ``pair = (si, sj)`` (between it and
    the one above) becomes a comb: along the edge, leaving ``period`` element
    columns straight at each end, in runs of ``period`` columns, the boundary
    is pushed alternately ``amp`` element rows up (the lower substructure takes
    them) and ``amp`` rows down (the upper one takes them).  Both substructures
    stay connected, the edge keeps its two end points, and no other
    substructure meets it (``amp < sub``).  The paper's figure of its jagged
    edge is not available, so this geometry stands in for it.
    """
    e2s, ns = grid_decomposition(nx, sub)
    m = nx // sub
    si, sj = pair
    lo, hi = sj * m + si, (sj + 1) * m + si
    y0 = (sj + 1) * sub                       # element row where the upper substructure starts
    e = e2s.reshape(nx, nx).copy()            # [ej, ei]
    for c in range(period, sub - period):
        ei = si * sub + c
        if ((c - period) // period) % 2 == 0:
            e[y0:y0 + amp, ei] = lo
        else:
            e[y0 - amp:y0, ei] = hi
    return e.reshape(-1).astype(np.int32), ns


def jagged_grid_grouping(n_sub_side: int, group: int, pair=(1, 0), amp: int = 1, period: int = 2):
    """``grid_grouping`` with the horizontal level-2 edge above level-2
    substructure ``pair`` made a comb of level-1 substructures, as in
    ``jagged_grid_decomposition``."""
    s2, n2 = grid_grouping(n_sub_side, group)
    m = n_sub_side // group
    si, sj = pair
    lo, hi = sj * m + si, (sj + 1) * m + si
    y0 = (sj + 1) * group
    g = s2.reshape(n_sub_side, n_sub_side).copy()
    for c in range(period, group - period):
        x = si * group + c
        if ((c - period) // period) % 2 == 0:
            g[y0:y0 + amp, x] = lo
        else:
            g[y0 - amp:y0, x] = hi
    return g.reshape(-1).astype(np.int32), n2


def elasticity(nx: int = 768, sub: int = 16, levels: int = 2, group: int = 16,
               constraints: str = "adaptive", tau: float = 10.0, jagged: bool = True,
               rhs_seed: int | None = None, k=None, lame=(1.0, 2.0),
               constraints_level2: str | None = None) -> Workload:
    """The setting of the paper's experiments (Sec. 5): plane linear elasticity
    with lambda = 1, mu = 2 on the unit square, 768 x 768 bilinear elements cut
    into 48 x 48 substructures (H/h = 16) and, for three levels, into 3 x 3
    level-2 substructures of 16 x 16 level-1 ones; one level-1 edge (between
    substructures 1 and 1 + 48, the pair the paper numbers (2, 50)) and, for
    three levels, one level-2 edge (level-2 substructures 1 and 4, the paper's
    (2, 5)) jagged.  Clamped on x = 0, body force (0, -1) unless ``rhs_seed``
    asks for N(0, 1) loads; ``k`` scales the Lame parameters per element
    (default 1)."""
    m = nx // sub
    if jagged:
        e2s, ns = jagged_grid_decomposition(nx, sub, (1, 0))
    else:
        e2s, ns = grid_decomposition(nx, sub)
    s2, n2 = None, 0
    if levels == 3:
        if jagged:
            s2, n2 = jagged_grid_grouping(m, group, (1, 0))
        else:
            s2, n2 = grid_grouping(m, group)
    kk = constant_coefficient(nx) if k is None else np.asarray(k, dtype=np.float64)
    name = "elasticity_%d_%dlev" % (nx, levels)
    return Workload(name, nx, kk, e2s, ns, levels, tau, constraints, s2, n2, rhs_seed=rhs_seed,
                    problem="elasticity", lame=tuple(lame), clamp="left",
                    constraints_level2=constraints_level2)
