"""Dense resolvents on tiny grids (oracle; test infrastructure).

* Unperturbed Green's function of the transition region, Eq. GF4:
  G0(Z) = (Z - H_T)^{-1}.
* Perturbed Green's function, Eq. GF2 (equivalently the inverse of the
  finite NEGF matrix of Eq. "NEGF Hamiltonian"):
  G(Z) = (Z - H_T - Sigma_L(Z) - Sigma_R(Z))^{-1}, with Sigma_L on the first
  n_face planes and Sigma_R on the last n_face planes (Eq. sec2-01).

The paper calls this direct inversion impractical for real sizes (Sec. III A);
here it is the plain definition the iterative path must reproduce.
"""

from __future__ import annotations

import numpy as np

from .operator import dense_hamiltonian, boundary_rows


def g0_dense(problem, Z, rows=None, cols=None):
    """[(Z - H_T)^{-1}]_{rows, cols} by LU (numpy.linalg.solve)."""
    H = dense_hamiltonian(problem)
    N = H.shape[0]
    cols = np.arange(N) if cols is None else np.asarray(cols)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    E = np.zeros((N, cols.size), np.complex128)
    E[cols, np.arange(cols.size)] = 1.0
    X = np.linalg.solve(Z * np.eye(N) - H, E)
    return X[rows, :]


def g_dense(problem, Z, Sigma_L, Sigma_R, rows=None, cols=None):
    """[(Z - H_T - Sigma_L - Sigma_R)^{-1}]_{rows, cols} by LU (Eq. GF2)."""
    H = dense_hamiltonian(problem)
    N = H.shape[0]
    nf = problem.n_face
    b = boundary_rows(problem.grid, nf)
    ns = b.size // 2
    M = Z * np.eye(N, dtype=np.complex128) - H
    L, R = b[:ns], b[ns:]
    M[np.ix_(L, L)] -= Sigma_L
    M[np.ix_(R, R)] -= Sigma_R
    cols = np.arange(N) if cols is None else np.asarray(cols)
    rows = np.arange(N) if rows is None else np.asarray(rows)
    E = np.zeros((N, cols.size), np.complex128)
    E[cols, np.arange(cols.size)] = 1.0
    X = np.linalg.solve(M, E)
    return X[rows, :]
