"""COCG and shifted COCG with seed switching (oracle; test infrastructure).

Follows the paper's Appendix step by step, in its notation:

* COCG for a complex-symmetric A (A = A^T != A^H), three-term residual form:
  Eqs. Eq, xvec, rvec, pvec, alpha, beta, with the bilinear form
  (x, y) = x^T y (no conjugation).
* Shifted systems (A + sigma_i I) x^(i) = b solved from the seed system
  A x = b through the collinear residuals r_n^(i) = r_n / pi_n^(s,i)
  (Eq. collinear) and the scalar recurrences Eqs. spi, salpha, sbeta, with
  the vector updates of x^(i), p^(i) (Eq. endcollinear and the line above it).
* Iterate until every shift's residual meets the criterion (Sec. III B, last
  paragraph; Appendix, after Eq. endcollinear).
* Seed switching (Appendix, Eq. seedswitch): once the seed has converged, the
  unconverged energy with the largest residual becomes the seed; pi_{n-1},
  pi_n are divided by the new seed's values and alpha^(i), beta^(i), x^(i),
  p^(i) stay as they are.

Readings where the paper is silent or at odds with itself:

1. The Appendix states x_0 = p_0 = 0, which contradicts Eq. pvec with
   beta_{-1} = 0; p_0 = r_0 (= b) is used, i.e. p_{-1} = 0.
2. The convergence test is ||r_n^(i)||_2 / ||b||_2 < tol with the ordinary
   (conjugated) 2-norm and ||r_n^(i)|| = ||r_n|| / |pi_n^(s,i)|.
3. A converged shift is frozen (no further updates).
4. Seed choice: "mid" (index K//2, standing in for the Fermi energy the
   paper starts from), "first" or an explicit index; a new seed is the
   unconverged shift with the largest residual, ties to the lowest index.
5. A quasi-null (r_n, r_n) (|(r,r)| <= 1e-300 or <= 1e-28 ||r||^2 while
   r != 0) is reported as a breakdown; the paper has no look-ahead.
6. After a switch the seed's residual vectors are rescaled by the collinear
   factors r^(s~) = r / pi^(s,s~), the seed's alpha_{n-1} and beta_{n-1} are
   taken from alpha_{n-1}^(s~), beta_{n-1}^(s~), and A becomes Z_s~ - H.
7. Switching to an energy outside the set (the extension the Appendix
   mentions after Eq. seedswitch): such an auxiliary energy is carried as a
   shift of its own through Eqs. spi, salpha, sbeta only (pi_{n-1}, pi_n,
   alpha^(a), beta^(a); no x or p, since nothing of its solution is wanted),
   so Eq. seedswitch applies to it unchanged.  It can be the first seed and it
   is a switch candidate like an unconverged energy of the set (largest
   residual wins; energies of the set come first on ties).  The iteration
   stops when every energy of the set has converged, whatever the auxiliary
   shifts' residuals.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OK, MAXIT, BREAKDOWN = 0, 4, 5


def bilinear(x, y):
    """(x, y) = x^T y, the unconjugated form COCG uses for complex-symmetric A."""
    return np.dot(x, y)


def cocg(apply_A, b, tol, maxit=100000):
    """Conventional COCG for A x = b (Appendix, Eqs. xvec, rvec, pvec, alpha, beta).

    Returns (x, iterations, status, residual history ||r_n||/||b||).
    """
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r_nm2 = b.copy()             # r_{n-2}   (r_{-1} = b)
    r_nm1 = b.copy()             # r_{n-1}   (r_0 = b)
    p_nm1 = b.copy()             # p_{n-1}   (p_0 = r_0, reading 1)
    alpha_nm2 = 1.0 + 0j         # alpha_{-1} = 1
    beta_nm2 = 0.0 + 0j          # beta_{-1} = 0
    rr_nm1 = bilinear(r_nm1, r_nm1)
    hist = [1.0]
    n = 1
    if bnorm == 0.0:
        return x, 0, OK, hist
    while n <= maxit:
        Ar = apply_A(r_nm1)
        # Eq. alpha:  alpha_{n-1} = (r,r) / ((r,Ar) - beta_{n-2}/alpha_{n-2} (r,r))
        alpha_nm1 = rr_nm1 / (bilinear(r_nm1, Ar) - beta_nm2 / alpha_nm2 * rr_nm1)
        # Eq. xvec
        x = x + alpha_nm1 * p_nm1
        # Eq. rvec
        c = beta_nm2 * alpha_nm1 / alpha_nm2
        r_n = (1.0 + c) * r_nm1 - alpha_nm1 * Ar - c * r_nm2
        res = np.linalg.norm(r_n) / bnorm
        hist.append(res)
        if res < tol:
            return x, n, OK, hist
        rr_n = bilinear(r_n, r_n)
        if abs(rr_n) <= 1e-300 or abs(rr_n) <= 1e-28 * np.linalg.norm(r_n) ** 2:
            return x, n, BREAKDOWN, hist
        # Eq. beta, Eq. pvec
        beta_nm1 = rr_n / rr_nm1
        p_n = r_n + beta_nm1 * p_nm1
        r_nm2, r_nm1, p_nm1 = r_nm1, r_n, p_n
        alpha_nm2, beta_nm2, rr_nm1 = alpha_nm1, beta_nm1, rr_n
        n += 1
    return x, maxit, MAXIT, hist


@dataclass
class ShiftedResult:
    x: np.ndarray                 # [K, len(rows)] solutions x^(i) restricted to rows
    iterations: int               # seed iterations (= matrix-vector products)
    switches: int                 # number of seed switches
    status: int                   # OK, MAXIT or BREAKDOWN
    seeds: list = field(default_factory=list)        # seed index after each switch (first = initial)
    converged_at: np.ndarray = None                  # [K] iteration at which each shift converged
    final_res: np.ndarray = None                     # [K] ||r^(i)|| / ||b|| at convergence


def shifted_cocg(apply_H, b, Z, tol, rows=None, seed="mid", maxit=100000, aux=None):
    """Solve (Z_i - H) x^(i) = b for every complex energy Z_i (Appendix, Eqs. collinear ... seedswitch).

    apply_H(v) returns H v for the real-symmetric H_T.  The seed system is
    A x = b with A = Z_s - H; the shifts are sigma_i = Z_i - Z_s so that
    A + sigma_i I = Z_i - H (Sec. III B).  Only the entries of x^(i), p^(i)
    at ``rows`` are kept (the paper keeps only the required elements).

    ``aux`` (optional) lists complex energies outside the set that may serve
    as seeds (reading 7); ``seed=("aux", j)`` starts from aux[j].  Seeds in
    ``seeds`` index the set first, then the auxiliary energies (K + j).
    """
    b = np.asarray(b, dtype=np.complex128)
    Z = np.asarray(Z, dtype=np.complex128)
    K = Z.shape[0]
    aux = np.zeros(0, np.complex128) if aux is None else np.asarray(aux, dtype=np.complex128).ravel()
    rows = np.arange(b.shape[0]) if rows is None else np.asarray(rows)
    bnorm = np.linalg.norm(b)
    if seed == "mid":
        s = K // 2
    elif seed == "first":
        s = 0
    elif isinstance(seed, tuple) and seed[0] == "aux":
        s = K + int(seed[1])
    else:
        s = int(seed)
    Zset = Z
    Z = np.concatenate([Zset, aux])          # every shift the scalar recurrences carry
    KA = Z.shape[0]

    x = np.zeros((K, rows.size), np.complex128)      # x_n^(i) at rows   (x_0 = 0), set energies only
    p = np.zeros((K, rows.size), np.complex128)      # p_{n-1}^(i) at rows  (p_{-1} = 0)
    pi_nm1 = np.ones(KA, np.complex128)              # pi_{n-1}^(s,i)   (pi_{-1} = 1)
    pi_n = np.ones(KA, np.complex128)                # pi_n^(s,i)       (pi_0 = 1)
    alpha_i_nm1 = np.ones(KA, np.complex128)         # alpha_{n-1}^(i)  (alpha_{-1} = 1)
    active = np.ones(KA, bool)
    converged_at = np.full(KA, -1)
    final_res = np.full(KA, np.nan)

    r_nm1 = b.copy()                                 # r_{n-1}  (r_{-1} = b)
    r_n = b.copy()                                   # r_n      (r_0 = b)
    alpha_nm1 = 1.0 + 0j                             # alpha_{-1} = 1
    beta_nm1 = 0.0 + 0j                              # beta_{-1} = 0
    rr_n = bilinear(r_n, r_n)
    sigma = Z - Z[s]
    seeds = [s]
    switches = 0
    n = 0
    if bnorm == 0.0:
        return ShiftedResult(x, 0, 0, OK, seeds, np.zeros(K, int), np.zeros(K))

    def done(status):
        return ShiftedResult(x, n, switches, status, seeds, converged_at[:K], final_res[:K])

    while True:
        # --- convergence test for r_n^(i) = r_n / pi_n^(s,i)  (reading 2, 3)
        rnorm = np.linalg.norm(r_n)
        res = rnorm / (np.abs(pi_n) * bnorm)
        newly = active & (res < tol)
        converged_at[newly] = n
        final_res[newly] = res[newly]
        active &= ~newly
        if not active[:K].any():
            return done(OK)
        if n >= maxit:
            final_res[active] = res[active]
            return done(MAXIT)

        # --- seed switching (Eq. seedswitch; reading 4, 6)
        if not active[s]:
            cand = np.where(active, res, -np.inf)
            s_new = int(np.argmax(cand))
            f_n, f_nm1 = pi_n[s_new], pi_nm1[s_new]
            # collinear residuals of the new seed: r^(s~) = r / pi^(s,s~)
            r_n = r_n / f_n
            r_nm1 = r_nm1 / f_nm1
            rr_n = rr_n / (f_n * f_n)
            # the new seed's own scalars: alpha_{n-1}^(s~), beta_{n-1}^(s~) (Eqs. salpha, sbeta)
            alpha_nm1 = alpha_i_nm1[s_new]
            beta_nm1 = (f_nm1 / f_n) ** 2 * beta_nm1
            # Eq. seedswitch for k = n-1 and n
            pi_n = pi_n / f_n
            pi_nm1 = pi_nm1 / f_nm1
            s = s_new
            sigma = Z - Z[s]
            seeds.append(s)
            switches += 1

        # --- seed system: q = A r_n with A = Z_s - H
        Ar = Z[s] * r_n - apply_H(r_n)
        rAr = bilinear(r_n, Ar)
        if abs(rr_n) <= 1e-300 or abs(rr_n) <= 1e-28 * rnorm ** 2:
            final_res[active] = res[active]
            return done(BREAKDOWN)
        # Eq. alpha (index shifted by one): alpha_n
        alpha_n = rr_n / (rAr - beta_nm1 / alpha_nm1 * rr_n)
        c_n = beta_nm1 * alpha_n / alpha_nm1

        # --- shifted systems (Eqs. sbeta, endcollinear, spi, salpha, and the x^(i) update); the
        # auxiliary shifts carry only their scalars (reading 7)
        a = active
        beta_i = (pi_nm1[a] / pi_n[a]) ** 2 * beta_nm1                       # beta_{n-1}^(i)
        pi_np1 = (1.0 + c_n + alpha_n * sigma[a]) * pi_n[a] - c_n * pi_nm1[a]  # pi_{n+1}
        alpha_i = pi_n[a] / pi_np1 * alpha_n                                 # alpha_n^(i)
        ak = a[:K]
        nk = int(ak.sum())                                                   # set energies come first in a
        p[ak] = r_n[rows][None, :] / pi_n[:K][ak][:, None] + beta_i[:nk, None] * p[ak]   # p_n^(i)
        x[ak] = x[ak] + alpha_i[:nk, None] * p[ak]                           # x_{n+1}^(i)
        alpha_i_nm1[a] = alpha_i
        pi_nm1[a], pi_n[a] = pi_n[a], pi_np1

        # --- seed residual, Eq. rvec (index shifted by one): r_{n+1}
        r_np1 = (1.0 + c_n) * r_n - alpha_n * Ar - c_n * r_nm1
        rr_np1 = bilinear(r_np1, r_np1)
        # Eq. beta: beta_n = (r_{n+1}, r_{n+1}) / (r_n, r_n)
        beta_nm1 = rr_np1 / rr_n
        alpha_nm1 = alpha_n
        r_nm1, r_n, rr_n = r_n, r_np1, rr_np1
        n += 1


def shifted_cocg_columns(problem, cols=None, rows=None, seed="mid", tol=None, maxit=None):
    """Run the shifted COCG of Sec. III B for every right-hand side e_j, j in cols.

    Returns (G0 [K, len(rows), len(cols)], list of ShiftedResult).
    """
    from .operator import hamiltonian, apply_h, boundary_rows

    Hloc, P, wE = hamiltonian(problem)
    cols = problem.cols if cols is None else np.asarray(cols)
    rows = boundary_rows(problem.grid, problem.n_face) if rows is None else np.asarray(rows)
    Z = problem.energies + 1j * problem.eta
    tol = problem.tol if tol is None else tol
    maxit = problem.maxit if maxit is None else maxit
    out = np.zeros((Z.size, rows.size, cols.size), np.complex128)
    results = []
    for jj, j in enumerate(cols):
        b = np.zeros(problem.N, np.complex128)
        b[j] = 1.0
        r = shifted_cocg(lambda v: apply_h(Hloc, P, wE, v), b, Z, tol, rows=rows, seed=seed, maxit=maxit)
        out[:, :, jj] = r.x
        results.append(r)
    return out, results
