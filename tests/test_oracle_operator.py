"""Pins of the oracle's Hamiltonian (Sec. II A) against facts fixed by the mathematics.

* A central difference of order p differentiates polynomials of degree <= p+1
  exactly: on interior points H_T applied to such a polynomial equals
  -1/2 nabla^2 of it, and fails for degree p+2.  This pins the coefficients,
  their sign and scale, and the axis ordering of the Kronecker sum.
* With zero ghosts, the 2nd-order 1D operator is diagonalised by the discrete
  sine transform with eigenvalues (1 - cos(k pi/(N+1)))/h^2.
* A single projector p with sum p^2 h^3 = 1 is an eigenvector of its own
  nonlocal term with eigenvalue E_a.
"""

import numpy as np
import pytest

from workloads import small_problem, grid_coordinates
from oracle.operator import hamiltonian, apply_h, dense_hamiltonian, boundary_rows, transverse_modes, kinetic_1d


def _poly_and_laplacian(deg):
    # a polynomial mixing all three axes with distinct powers, and its Laplacian
    if deg == 3:
        f = lambda x, y, z: x ** 3 + 2 * y ** 2 * z - 0.5 * z ** 3 * 1.0 + x * y * z + 0.3 * y ** 3
        lap = lambda x, y, z: 6 * x + 4 * z - 3.0 * z + 1.8 * y
    elif deg == 5:
        f = lambda x, y, z: x ** 5 - 0.7 * y ** 4 * z + 0.2 * z ** 5 + x ** 2 * y ** 3 + 1.5 * x * z ** 4
        lap = lambda x, y, z: (20 * x ** 3 - 8.4 * y ** 2 * z + 4.0 * z ** 3 + 2 * y ** 3 + 6 * x ** 2 * y
                               + 18.0 * x * z ** 2)
    elif deg == 6:
        f = lambda x, y, z: x ** 6 + 0 * y + 0 * z
        lap = lambda x, y, z: 30 * x ** 4 + 0 * y + 0 * z
    return f, lap


def _interior(grid, R):
    nx, ny, nz = grid
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = (X >= R) & (X < nx - R) & (Y >= R) & (Y < ny - R) & (Z >= R) & (Z < nz - R)
    return m.ravel()


@pytest.mark.parametrize("order,deg", [(2, 3), (4, 5)])
def test_fd_exact_on_polynomials(order, deg):
    p = small_problem(grid=(9, 8, 10), h=0.37, fd_order=order, n_wells=0)
    H, P, wE = hamiltonian(p)
    x, y, z = grid_coordinates(p.grid, p.h)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f, lap = _poly_and_laplacian(deg)
    Hf = apply_h(H, P, wE, f(X, Y, Z).ravel())
    want = -0.5 * lap(X, Y, Z).ravel()
    m = _interior(p.grid, order // 2)
    assert m.sum() > 20
    np.testing.assert_allclose(Hf[m], want[m], rtol=1e-9, atol=1e-8 * np.abs(want).max())


@pytest.mark.parametrize("order", [2, 4])
def test_fd_not_exact_beyond_order(order):
    # degree order+2 polynomial is NOT reproduced: guards against a stencil of the wrong order
    p = small_problem(grid=(11, 6, 7), h=0.3, fd_order=order, n_wells=0)
    H, P, wE = hamiltonian(p)
    x, y, z = grid_coordinates(p.grid, p.h)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    deg = order + 2
    f = X ** deg
    lap = deg * (deg - 1) * X ** (deg - 2)
    m = _interior(p.grid, order // 2)
    err = np.abs(apply_h(H, P, wE, f.ravel())[m] + 0.5 * lap.ravel()[m]).max()
    assert err > 1e-6


def test_dirichlet_spectrum_second_order():
    p = small_problem(grid=(4, 3, 5), h=0.6, fd_order=2, n_wells=0)
    ev = np.linalg.eigvalsh(dense_hamiltonian(p))
    def axis(n):
        k = np.arange(1, n + 1)
        return (1.0 - np.cos(k * np.pi / (n + 1))) / p.h ** 2
    ex, ey, ez = (axis(n) for n in p.grid)
    want = np.sort((ez[:, None, None] + ey[None, :, None] + ex[None, None, :]).ravel())
    np.testing.assert_allclose(ev, want, rtol=0, atol=1e-12 * want.max())


def test_potential_enters_diagonal():
    p = small_problem(grid=(5, 4, 6), fd_order=4, n_wells=3)
    p0 = small_problem(grid=(5, 4, 6), fd_order=4, n_wells=0)
    D = dense_hamiltonian(p) - dense_hamiltonian(p0)
    np.testing.assert_allclose(D, np.diag(p.V.ravel()), atol=1e-14)
    assert np.abs(p.V).max() > 0.1


def test_projector_is_eigvec_of_its_term():
    p = small_problem(grid=(10, 9, 12), h=0.4, fd_order=4, n_wells=0, projectors=1)
    pr = p.proj
    pv = np.zeros(p.N)
    pv[pr.idx] = pr.val
    np.testing.assert_allclose(np.sum(pr.val ** 2) * p.h ** 3, 1.0, rtol=1e-12)
    Hd = dense_hamiltonian(p)
    Hk = dense_hamiltonian(small_problem(grid=(10, 9, 12), h=0.4, fd_order=4, n_wells=0))
    Vnl = Hd - Hk
    np.testing.assert_allclose(Vnl @ pv, pr.E[0] * pv, atol=1e-12)
    assert np.linalg.matrix_rank(Vnl, tol=1e-10) == 1
    np.testing.assert_allclose(Hd, Hd.T, atol=0)


def test_boundary_rows_order():
    b = boundary_rows((3, 2, 5), 2)
    nxy = 6
    want = np.concatenate([np.arange(nxy), nxy + np.arange(nxy), 3 * nxy + np.arange(nxy), 4 * nxy + np.arange(nxy)])
    np.testing.assert_array_equal(b, want)


def test_transverse_modes_dst():
    nx, ny, h = 5, 4, 0.5
    eps, U = transverse_modes(nx, ny, h, 2)
    def axis(n):
        k = np.arange(1, n + 1)
        return (1.0 - np.cos(k * np.pi / (n + 1))) / h ** 2
    want = np.sort((axis(ny)[:, None] + axis(nx)[None, :]).ravel())
    np.testing.assert_allclose(eps, want, atol=1e-12)
    T2 = np.kron(np.eye(ny), kinetic_1d(nx, h, 2).toarray()) + np.kron(kinetic_1d(ny, h, 2).toarray(), np.eye(nx))
    np.testing.assert_allclose(U @ np.diag(eps) @ U.T, T2, atol=1e-12)
