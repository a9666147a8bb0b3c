"""Pins for the oracle's Q1 discretization (Sec. 2, eq. 1).

* The closed-form element matrix equals 2x2 Gauss quadrature of
  grad phi_a . grad phi_b (an independent route), has zero row sums and the
  circulant eigenvalues {0, 2/3, 1, 1}.
* The assembled operator for k = 1 is the classical Q1 nine-point stencil
  (8/3 on the diagonal, -1/3 to each of the eight neighbours).
* The load vector of f = 1 is h^2 per free node.
* The discrete solution of -Laplace u = 1 converges at O(h^2) to the Fourier
  series value u(1/2, 1/2) = 0.07367135...
"""
import numpy as np
import scipy.sparse.linalg as spl

from oracle import fem
from paper_0911_5730_gb300 import inputs


def _gauss_stiffness():
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    K = np.zeros((4, 4))
    for x in gp:
        for y in gp:
            grads = [(-(1 - y), -(1 - x)), ((1 - y), -x), (y, x), (-y, (1 - x))]
            for a in range(4):
                for b in range(4):
                    K[a, b] += 0.25 * (grads[a][0] * grads[b][0] + grads[a][1] * grads[b][1])
    return K


def test_element_matrix_matches_quadrature():
    assert np.allclose(fem.q1_reference_stiffness(), _gauss_stiffness(), atol=1e-15)


def test_element_matrix_rows_and_spectrum():
    K = fem.q1_reference_stiffness()
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-15)
    assert np.allclose(np.sort(np.linalg.eigvalsh(K)), [0.0, 2 / 3, 1.0, 1.0], atol=1e-14)


def test_assembled_nine_point_stencil():
    nx = 6
    dofs, mats = fem.level1_elements(nx, np.ones(nx * nx))
    A = fem.assemble((nx - 1) ** 2, dofs, mats).toarray()
    g = fem.free_index(nx, 3, 3)
    row = A[g]
    assert np.isclose(row[g], 8.0 / 3.0)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            if di or dj:
                assert np.isclose(row[fem.free_index(nx, 3 + di, 3 + dj)], -1.0 / 3.0)
    assert np.count_nonzero(np.abs(row) > 1e-14) == 9
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A)[0] > 0


def test_load_vector_unit_source():
    for nx in (4, 9):
        b = fem.load_vector(nx)
        assert np.allclose(b, 1.0 / nx ** 2, rtol=1e-14)
        assert np.allclose(b, inputs.unit_load_rhs(nx), rtol=1e-14)


def _series_center(terms=60):
    # u = x(1-x)/2 - sum_{m odd} 4/(pi^3 m^3) sin(m pi x) cosh(m pi (y-1/2)) / cosh(m pi/2)
    s = 0.125
    for m in range(1, terms, 2):
        s -= 4.0 / (np.pi ** 3 * m ** 3) * (-1) ** ((m - 1) // 2) / np.cosh(m * np.pi / 2)
    return s


def _double_series_center(terms=400):
    s = 0.0
    for m in range(1, terms, 2):
        for n in range(1, terms, 2):
            sgn = (-1) ** ((m - 1) // 2 + (n - 1) // 2)
            s += sgn * 16.0 / (np.pi ** 4 * m * n * (m * m + n * n))
    return s


def test_convergence_to_series_solution():
    exact = _series_center()
    assert abs(exact - 0.0736713532) < 1e-9
    assert abs(exact - _double_series_center()) < 1e-8
    errs = []
    for nx in (8, 16, 32, 64):
        dofs, mats = fem.level1_elements(nx, np.ones(nx * nx))
        A = fem.assemble((nx - 1) ** 2, dofs, mats)
        u = spl.spsolve(A.tocsc(), fem.load_vector(nx))
        errs.append(abs(u[fem.free_index(nx, nx // 2, nx // 2)] - exact))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < r < 4.5 for r in rates), rates
