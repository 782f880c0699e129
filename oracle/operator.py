"""The RSFD Hamiltonian of the transition region, H_T (oracle; test infrastructure).

Sec. II A writes the Kohn-Sham Hamiltonian on a real-space grid as a block
tridiagonal matrix in z (Eq. sabun1 and the matrix after it): each plane
block A(z_k) holds the in-plane finite-difference Laplacian plus the
potential, and the coupling between neighbouring planes is proportional to
the identity.  Higher-order finite differences and nonlocal pseudopotentials
are mentioned as extensions (Sec. II A, citing the RSFD book).

Readings used here (the paper prints neither):

* kinetic operator -1/2 nabla^2 in Hartree units with the standard central
  coefficients (1, -2, 1)/h^2 (2nd order) and (-1/12, 4/3, -5/2, 4/3,
  -1/12)/h^2 (4th order) on every axis;
* zero ghosts outside the box on all six faces (Dirichlet walls in x and y;
  along z, H_T is the TT block of Eq. "H matrix", whose couplings to the
  leads are carried by the self-energies);
* nonlocal part  sum_a E_a p_a (p_a^T psi) h^3  (one separable projector
  per atom).

The operator is assembled as a Kronecker sum of 1D truncated Toeplitz
matrices, i.e. by its plain definition.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Central finite-difference coefficients of d^2/dx^2 at offsets 0, 1, 2 (times 1/h^2).
FD_SECOND_DERIVATIVE = {
    2: (-2.0, 1.0),
    4: (-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0),
}


def kinetic_1d(n: int, h: float, fd_order: int) -> sp.csr_matrix:
    """-1/2 d^2/dx^2 on n points with zero ghosts: a truncated symmetric Toeplitz matrix."""
    c = FD_SECOND_DERIVATIVE[fd_order]
    diags, offs = [], []
    for k, ck in enumerate(c):
        val = -0.5 * ck / (h * h)
        if k == 0:
            diags.append(np.full(n, val))
            offs.append(0)
        elif k < n:
            diags += [np.full(n - k, val), np.full(n - k, val)]
            offs += [k, -k]
    return sp.diags(diags, offs, shape=(n, n), format="csr")


def hamiltonian(problem, include_nonlocal: bool = True):
    """Return (H_local, P, wE) with H_T = H_local + P diag(wE) P^T.

    H_local is the sparse kinetic + local-potential part (linear index
    (z*Ny + y)*Nx + x), P is the N x n_atoms sparse projector matrix and
    wE = E_a h^3.  P and wE are None when the problem has no projectors.
    """
    nx, ny, nz = problem.grid
    h = problem.h
    Tx = kinetic_1d(nx, h, problem.fd_order)
    Ty = kinetic_1d(ny, h, problem.fd_order)
    Tz = kinetic_1d(nz, h, problem.fd_order)
    Ix, Iy, Iz = (sp.identity(n, format="csr") for n in (nx, ny, nz))
    H = (sp.kron(Tz, sp.kron(Iy, Ix)) + sp.kron(Iz, sp.kron(Ty, Ix)) + sp.kron(Iz, sp.kron(Iy, Tx)))
    H = (H + sp.diags(np.asarray(problem.V, dtype=np.float64).ravel())).tocsr()
    proj = problem.proj
    if include_nonlocal and proj is not None and proj.n_atoms > 0:
        rows = proj.idx
        cols = np.repeat(np.arange(proj.n_atoms), np.diff(proj.ptr))
        P = sp.csr_matrix((proj.val, (rows, cols)), shape=(problem.N, proj.n_atoms))
        wE = proj.E * problem.h ** 3
        return H, P, wE
    return H, None, None


def apply_h(Hloc, P, wE, psi):
    """H_T psi for a vector or an N x m block."""
    out = Hloc @ psi
    if P is not None:
        out = out + P @ (wE[:, None] * (P.T @ psi) if psi.ndim == 2 else wE * (P.T @ psi))
    return out


def dense_hamiltonian(problem) -> np.ndarray:
    """H_T as a dense FP64 matrix (tiny grids only)."""
    H, P, wE = hamiltonian(problem)
    Hd = H.toarray()
    if P is not None:
        Pd = P.toarray()
        Hd = Hd + (Pd * wE[None, :]) @ Pd.T
    return Hd


def boundary_rows(grid, n_face: int) -> np.ndarray:
    """The boundary row set b: the outer n_face planes on each side, in increasing z, x fastest.

    Sec. II B: the self-energies live on the first and last plane (N=1); with a
    stencil reaching n_face planes the lead couples to n_face planes per side.
    """
    nx, ny, nz = grid
    nxy = nx * ny
    planes = list(range(n_face)) + list(range(nz - n_face, nz))
    return np.concatenate([p * nxy + np.arange(nxy) for p in planes]).astype(np.int64)


def transverse_modes(nx: int, ny: int, h: float, fd_order: int):
    """Eigen-decomposition of the in-plane kinetic operator (index y*Nx + x).

    Returns (eps, U) with eps ascending and U orthogonal (columns = modes).
    """
    ex, Ux = np.linalg.eigh(kinetic_1d(nx, h, fd_order).toarray())
    ey, Uy = np.linalg.eigh(kinetic_1d(ny, h, fd_order).toarray())
    eps = (ey[:, None] + ex[None, :]).ravel()        # mode (j, i) -> j*nx + i
    U = np.kron(Uy, Ux)
    order = np.argsort(eps, kind="stable")
    return eps[order], U[:, order]
