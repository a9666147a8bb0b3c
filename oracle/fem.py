"""Q1 finite elements for -div(k grad u) = f on the unit square (Sec. 2, eq. 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The space W_i of Sec. 2 is the Q1 functions on substructure i that vanish on
the boundary of the domain; here the elements carry a scalar coefficient k_e
and the bilinear form is a(u, v) = sum_e k_e int_e grad u . grad v.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def q1_reference_stiffness() -> np.ndarray:
    """Element stiffness of grad u . grad v for a square bilinear element.

    Local node order (0,0), (1,0), (1,1), (0,1).  In 2D the matrix does not
    depend on the element size.  Derivation: with phi_a = (1 -+ x)(1 -+ y)
    on [0,1]^2, int grad phi_a . grad phi_b is 2/3 on the diagonal, -1/6 for
    edge neighbours and -1/3 for the opposite node.
    """
    return np.array([[4.0, -1.0, -2.0, -1.0],
                     [-1.0, 4.0, -1.0, -2.0],
                     [-2.0, -1.0, 4.0, -1.0],
                     [-1.0, -2.0, -1.0, 4.0]]) / 6.0


def free_index(nx: int, i: int, j: int) -> int:
    """Global index of node (i, j), or -1 on the Dirichlet boundary."""
    if i <= 0 or j <= 0 or i >= nx or j >= nx:
        return -1
    return (j - 1) * (nx - 1) + (i - 1)


def element_nodes(nx: int, e: int) -> list[int]:
    """Global free indices of the four nodes of element e (-1 = Dirichlet)."""
    ej, ei = divmod(e, nx)
    return [free_index(nx, ei, ej), free_index(nx, ei + 1, ej),
            free_index(nx, ei + 1, ej + 1), free_index(nx, ei, ej + 1)]


def level1_elements(nx: int, k: np.ndarray):
    """Element DOF lists and element matrices with Dirichlet nodes removed.

    Returns (elem_dofs, elem_mats): for each element the free node indices and
    the corresponding principal submatrix of k_e * K_ref.
    """
    kref = q1_reference_stiffness()
    dofs, mats = [], []
    for e in range(nx * nx):
        nodes = np.array(element_nodes(nx, e))
        keep = nodes >= 0
        dofs.append(nodes[keep])
        mats.append(k[e] * kref[np.ix_(keep, keep)])
    return dofs, mats


def assemble(n: int, elem_dofs, elem_mats) -> sp.csr_matrix:
    """A = sum_e R_e^T K_e R_e as a sparse matrix."""
    rows, cols, vals = [], [], []
    for d, m in zip(elem_dofs, elem_mats):
        if len(d) == 0:
            continue
        rr, cc = np.meshgrid(d, d, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(m.ravel())
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def load_vector(nx: int, f=lambda x, y: 1.0) -> np.ndarray:
    """<f, phi_g> by 2x2 Gauss quadrature on every element (exact for f = 1)."""
    h = 1.0 / nx
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    b = np.zeros((nx - 1) ** 2)
    for e in range(nx * nx):
        ej, ei = divmod(e, nx)
        nodes = element_nodes(nx, e)
        for xi in gp:
            for eta in gp:
                phi = [(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta]
                fv = f((ei + xi) * h, (ej + eta) * h)
                for a in range(4):
                    if nodes[a] >= 0:
                        b[nodes[a]] += 0.25 * h * h * fv * phi[a]
    return b


# -- plane linear elasticity (the problem of the experiments of Sec. 5) --------

def elasticity_reference_stiffness(lam: float, mu: float) -> np.ndarray:
    """Element stiffness of a(u, v) = int lam div u div v + 2 mu eps(u):eps(v)
    for a square bilinear element, plane strain.

    DOF order 2a + c: node a in (0,0), (1,0), (1,1), (0,1), component c (x, y).
    In 2D the matrix does not depend on the element size.  Strains in Voigt
    form (eps_xx, eps_yy, 2 eps_xy) = B u with the material matrix
    [[lam + 2mu, lam, 0], [lam, lam + 2mu, 0], [0, 0, mu]]; the 2 x 2 Gauss
    rule is exact (the integrand is at most quadratic in each variable).
    """
    D = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    K = np.zeros((8, 8))
    for x in gp:
        for y in gp:
            dx = np.array([-(1 - y), 1 - y, y, -y])
            dy = np.array([-(1 - x), -x, x, 1 - x])
            B = np.zeros((3, 8))
            B[0, 0::2] = dx
            B[1, 1::2] = dy
            B[2, 0::2] = dy
            B[2, 1::2] = dx
            K += 0.25 * B.T @ D @ B
    return K


def elastic_node_index(nx: int, i: int, j: int, clamp: str = "left") -> int:
    """Node (i, j) -> free node number, or -1 on the clamped side.

    ``clamp="left"``: the nodes with i = 0 (x = 0) are clamped (u = 0), node
    (i, j) with 1 <= i <= nx is j * nx + (i - 1).  ``clamp="none"``: no node
    is removed (the mesh before boundary conditions), node (i, j) is
    j * (nx + 1) + i.  DOF of component c of a node: 2 * node + c.
    """
    if clamp == "left":
        return -1 if i <= 0 else j * nx + (i - 1)
    return j * (nx + 1) + i


def elasticity_elements(nx: int, k: np.ndarray, lam: float, mu: float, clamp: str = "left"):
    """Element DOF lists and matrices k_e * K_ref of the elasticity problem.

    Returns (elem_dofs, elem_mats, n, comp, on_boundary, coords): per DOF its
    component, whether its node lies on the boundary of the square (the
    clamped nodes are gone, so these are the traction-free ones) and its
    node's coordinates.
    """
    kref = elasticity_reference_stiffness(lam, mu)
    h = 1.0 / nx
    nodes_i = range(1, nx + 1) if clamp == "left" else range(0, nx + 1)
    nn = (nx + 1) * len(nodes_i)
    comp = np.tile([0, 1], nn)
    bnd = np.zeros(2 * nn, dtype=bool)
    coords = np.zeros((2 * nn, 2))
    for j in range(nx + 1):
        for i in nodes_i:
            a = elastic_node_index(nx, i, j, clamp)
            on = i == 0 or j == 0 or i == nx or j == nx
            bnd[2 * a:2 * a + 2] = on
            coords[2 * a:2 * a + 2] = (i * h, j * h)
    dofs, mats = [], []
    for e in range(nx * nx):
        ej, ei = divmod(e, nx)
        nd = [elastic_node_index(nx, ei, ej, clamp), elastic_node_index(nx, ei + 1, ej, clamp),
              elastic_node_index(nx, ei + 1, ej + 1, clamp), elastic_node_index(nx, ei, ej + 1, clamp)]
        slots = np.array([2 * a + c if a >= 0 else -1 for a in nd for c in (0, 1)])
        keep = slots >= 0
        dofs.append(slots[keep])
        mats.append(k[e] * kref[np.ix_(keep, keep)])
    return dofs, mats, 2 * nn, comp, bnd, coords


def rigid_modes(coords: np.ndarray, comp: np.ndarray) -> np.ndarray:
    """The three rigid motions (two translations, the rotation (-y, x)) at
    every DOF, as columns."""
    Z = np.zeros((len(comp), 3))
    Z[comp == 0, 0] = 1.0
    Z[comp == 1, 1] = 1.0
    Z[comp == 0, 2] = -coords[comp == 0, 1]
    Z[comp == 1, 2] = coords[comp == 1, 0]
    return Z
