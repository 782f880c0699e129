"""Pins of the oracle's COCG / shifted COCG (Appendix) and dense G0 (Eq. GF4).

* G0 at V=0 with the 2nd-order stencil equals the separable DST closed form
  sum_modes phi phi^T / (Z - eps) (independent of the sparse assembly).
* COCG and shifted COCG reproduce a dense LU solve (a library routine) to
  well below the tolerance they were run at, for 2nd/4th order and with
  projectors; seed switching is exercised and does not change the result.
* The true residual b - (Z_i - H) x^(i) matches the collinear estimate
  ||r_n|| / |pi_n^(i)| (Eq. collinear).
* G0 is complex symmetric (G^T = G).
* Planted mistakes make the comparison with the dense solve fail: a conjugated
  bilinear form, a flipped shift sign, and (in a copy of the oracle's source) a
  dropped r_{n-2} term of Eq. rvec, a dropped pi_{n-1} term of Eq. spi and an
  unsquared pi ratio in Eq. sbeta.
"""

import numpy as np
import pytest

from workloads import small_problem
from oracle import cocg as oc
from oracle.operator import hamiltonian, apply_h, dense_hamiltonian, boundary_rows
from oracle.dense import g0_dense


def _dst_g0(p, Z):
    nx, ny, nz = p.grid
    h = p.h
    def basis(n):
        k = np.arange(1, n + 1)
        i = np.arange(1, n + 1)
        phi = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, k) * np.pi / (n + 1))   # [point, mode]
        lam = (1.0 - np.cos(k * np.pi / (n + 1))) / h ** 2
        return phi, lam
    (px, lx), (py, ly), (pz, lz) = basis(nx), basis(ny), basis(nz)
    Phi = np.kron(pz, np.kron(py, px))
    lam = (lz[:, None, None] + ly[None, :, None] + lx[None, None, :]).ravel()
    return (Phi / (Z - lam)[None, :]) @ Phi.T


def test_dense_g0_matches_dst_closed_form():
    p = small_problem(grid=(4, 3, 6), h=0.5, fd_order=2, n_wells=0)
    Z = 0.9 + 0.05j
    np.testing.assert_allclose(g0_dense(p, Z), _dst_g0(p, Z), atol=1e-12)


def test_g0_complex_symmetric():
    p = small_problem(grid=(4, 4, 6), fd_order=4, n_wells=2, projectors=1)
    G = g0_dense(p, 0.5 + 0.01j)
    assert np.abs(G - G.T).max() < 1e-12 * np.abs(G).max()
    assert np.abs(G - G.conj().T).max() > 1e-3 * np.abs(G).max()     # not Hermitian


@pytest.mark.parametrize("order,proj", [(2, 0), (4, 0), (4, 2)])
def test_cocg_single_energy_matches_dense(order, proj):
    p = small_problem(grid=(5, 4, 8), h=0.5, fd_order=order, n_wells=2, projectors=proj)
    H, P, wE = hamiltonian(p)
    Z = 0.7 + 0.02j
    j = 3
    b = np.zeros(p.N, complex)
    b[j] = 1
    x, it, st, hist = oc.cocg(lambda v: Z * v - apply_h(H, P, wE, v), b, 1e-12)
    assert st == oc.OK and hist[-1] < 1e-12
    xd = g0_dense(p, Z, cols=[j])[:, 0]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


@pytest.mark.parametrize("order,proj,seed", [(2, 0, "mid"), (4, 0, "first"), (4, 2, "mid"), (2, 0, 5)])
def test_shifted_matches_dense_and_single(order, proj, seed):
    p = small_problem(grid=(5, 4, 8), h=0.5, fd_order=order, n_wells=2, projectors=proj, n_energies=6,
                      e_range=(-0.5, 2.5), eta=2e-2)
    H, P, wE = hamiltonian(p)
    Z = p.energies + 1j * p.eta
    j = 7
    b = np.zeros(p.N, complex)
    b[j] = 1
    r = oc.shifted_cocg(lambda v: apply_h(H, P, wE, v), b, Z, 1e-12, seed=seed)
    assert r.status == oc.OK
    for k in range(Z.size):
        xd = g0_dense(p, Z[k], cols=[j])[:, 0]
        assert np.linalg.norm(r.x[k] - xd) / np.linalg.norm(xd) < 1e-9, k
        xs, _, st, _ = oc.cocg(lambda v: Z[k] * v - apply_h(H, P, wE, v), b, 1e-12)
        assert np.linalg.norm(r.x[k] - xs) / np.linalg.norm(xs) < 1e-9
        # true residual vs the collinear estimate
        tr = np.linalg.norm(b - (Z[k] * r.x[k] - apply_h(H, P, wE, r.x[k])))
        assert tr < 50 * 1e-12 and r.final_res[k] < 1e-12


def test_seed_switching_exercised_and_invariant():
    # the seed sits far below the spectrum, converges first and must be switched away from
    p = small_problem(grid=(5, 4, 8), h=0.5, fd_order=4, n_wells=2, n_energies=5, eta=1e-2)
    H, P, wE = hamiltonian(p)
    Z = np.array([-6.0, 0.3, 0.8, 1.4, 3.0]) + 1j * p.eta
    b = np.zeros(p.N, complex)
    b[11] = 1
    r0 = oc.shifted_cocg(lambda v: apply_h(H, P, wE, v), b, Z, 1e-12, seed=0)
    assert r0.switches >= 1 and r0.status == oc.OK
    r1 = oc.shifted_cocg(lambda v: apply_h(H, P, wE, v), b, Z, 1e-12, seed=2)
    for k in range(Z.size):
        xd = g0_dense(p, Z[k], cols=[11])[:, 0]
        for r in (r0, r1):
            assert np.linalg.norm(r.x[k] - xd) / np.linalg.norm(xd) < 1e-9


def test_columns_and_rows_restriction():
    p = small_problem(grid=(4, 4, 6), h=0.5, fd_order=2, n_wells=1, n_energies=3, eta=5e-2)
    rows = boundary_rows(p.grid, 1)
    G, res = oc.shifted_cocg_columns(p)
    assert G.shape == (3, rows.size, p.cols.size)
    for k, E in enumerate(p.energies):
        Gd = g0_dense(p, E + 1j * p.eta, rows=rows, cols=p.cols)
        assert np.linalg.norm(G[k] - Gd) / np.linalg.norm(Gd) < 1e-9
        # boundary block of a symmetric matrix with rows == cols is symmetric
        assert np.abs(G[k] - G[k].T).max() < 1e-9 * np.abs(G[k]).max()


def _shifted_err(p, patched, mod=None):
    mod = oc if mod is None else mod
    H, P, wE = hamiltonian(p)
    Z = p.energies + 1j * p.eta
    b = np.zeros(p.N, complex)
    b[5] = 1
    r = mod.shifted_cocg(lambda v: apply_h(H, P, wE, v), b, Z, 1e-10, maxit=2000)
    errs = []
    for k in range(Z.size):
        xd = g0_dense(p, Z[k], cols=[5])[:, 0]
        errs.append(np.linalg.norm(r.x[k] - xd) / np.linalg.norm(xd))
    return max(errs)


@pytest.mark.parametrize("mistake", ["conjugated_form", "flipped_shift"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    p = small_problem(grid=(4, 4, 6), h=0.5, fd_order=2, n_wells=2, n_energies=4, eta=3e-2)
    assert _shifted_err(p, None) < 1e-8
    if mistake == "conjugated_form":
        monkeypatch.setattr(oc, "bilinear", lambda x, y: np.vdot(x, y))
    else:
        orig = oc.shifted_cocg

        def flipped(apply_H, b, Z, tol, **kw):
            # solving (Z_s - H) with shifts of the wrong sign == energies mirrored about the seed
            Zs = Z[Z.size // 2]
            return orig(apply_H, b, 2 * Zs - Z + 2j * Z.imag, tol, **kw)
        monkeypatch.setattr(oc, "shifted_cocg", flipped)
    assert _shifted_err(p, mistake) > 1e-4


def test_chain_shifted_dyson_transmission_matches_dense():
    """G0_bb by shifted COCG -> Dyson -> T equals T from the dense Eq. GF2 (full oracle chain)."""
    from oracle.leads import sigma_bloch
    from oracle.dense import g_dense
    from oracle.dyson import dyson_solve
    from oracle.transmission import transmission
    p = small_problem(grid=(4, 3, 8), h=0.5, fd_order=4, n_wells=2, projectors=1, n_energies=4,
                      e_range=(1.0, 4.0), eta=1e-2)
    b = boundary_rows(p.grid, p.n_face)
    G0, res = oc.shifted_cocg_columns(p, cols=b, rows=b)
    for k, E in enumerate(p.energies):
        Z = E + 1j * p.eta
        SL, SR = sigma_bloch(4, 3, p.h, 4, Z)
        G = dyson_solve(G0[k], SL, SR)
        Gd = g_dense(p, Z, SL, SR, rows=b, cols=b)
        assert np.linalg.norm(G - Gd) / np.linalg.norm(Gd) < 1e-9
        assert abs(transmission(G, SL, SR)[0] - transmission(Gd, SL, SR)[0]) < 1e-9


def _planted_module(old, new):
    """A copy of oracle/cocg.py with one source line changed (the committed oracle is untouched)."""
    import inspect
    import sys
    import types
    src = inspect.getsource(oc)
    assert old in src
    mod = types.ModuleType("oracle_cocg_planted")
    sys.modules[mod.__name__] = mod          # dataclasses resolve their module by name
    try:
        exec(compile(src.replace(old, new), "oracle_cocg_planted", "exec"), mod.__dict__)
    finally:
        del sys.modules[mod.__name__]
    return mod


@pytest.mark.parametrize("old,new", [
    # the r_{n-2} term of the three-term residual recurrence (Eq. rvec)
    ("r_np1 = (1.0 + c_n) * r_n - alpha_n * Ar - c_n * r_nm1", "r_np1 = (1.0 + c_n) * r_n - alpha_n * Ar"),
    # the pi_{n-1} term of the shifted recurrence (Eq. spi)
    ("pi_np1 = (1.0 + c_n + alpha_n * sigma[a]) * pi_n[a] - c_n * pi_nm1[a]",
     "pi_np1 = (1.0 + c_n + alpha_n * sigma[a]) * pi_n[a]"),
    # the square of the pi ratio in the shifted beta (Eq. sbeta)
    ("beta_i = (pi_nm1[a] / pi_n[a]) ** 2 * beta_nm1", "beta_i = (pi_nm1[a] / pi_n[a]) * beta_nm1"),
])
def test_planted_recurrence_mistakes_are_caught(old, new):
    p = small_problem(grid=(4, 4, 6), h=0.5, fd_order=2, n_wells=2, n_energies=4, eta=3e-2)
    assert _shifted_err(p, None) < 1e-8
    assert _shifted_err(p, "planted", _planted_module(old, new)) > 1e-4


def test_breakdown_branch_on_a_quasi_null_right_hand_side():
    """b = e_j + i e_k has b^T b = 1 + i^2 = 0 with b != 0: the unconjugated form of COCG vanishes at
    the start, which the oracle must report as a breakdown (reading 5) instead of dividing by it.  A
    conjugated form (b^H b = 2) would not break down, and a right-hand side that is not quasi-null
    (b = e_j + 0.5 i e_k) must converge to the dense solution as usual."""
    p = small_problem(grid=(5, 4, 6), h=0.5, fd_order=2, n_wells=2, n_energies=4, eta=5e-2, tol=1e-10)
    H, P, wE = hamiltonian(p)
    Z = p.energies + 1j * p.eta
    f = lambda v: apply_h(H, P, wE, v)
    j, k = 3, 17
    b = np.zeros(p.N, complex)
    b[j], b[k] = 1.0, 1j
    assert abs(oc.bilinear(b, b)) == 0.0 and np.linalg.norm(b) > 0
    r = oc.shifted_cocg(f, b, Z, p.tol)
    assert r.status == oc.BREAKDOWN and r.iterations == 0
    assert np.all(r.x == 0)
    x, it, status, _ = oc.cocg(lambda v: Z[1] * v - f(v), b, p.tol)
    assert status == oc.BREAKDOWN and it == 1 and np.all(x == 0)
    # not quasi-null: the usual solution
    b2 = np.zeros(p.N, complex)
    b2[j], b2[k] = 1.0, 0.5j
    r2 = oc.shifted_cocg(f, b2, Z, p.tol)
    assert r2.status == oc.OK
    Hd = dense_hamiltonian(p)
    for i in (0, 3):
        xd = np.linalg.solve(Z[i] * np.eye(p.N) - Hd, b2)
        assert np.linalg.norm(r2.x[i] - xd) <= 1e-8 * np.linalg.norm(xd)


def test_seed_outside_the_energy_set():
    """Seed switching to an energy outside the set (the extension stated after Eq. seedswitch): an
    auxiliary energy carried only through Eqs. spi, salpha, sbeta.  Starting from it, and switching to
    it, must give the same x^(i) as an in-set seed and as the dense solves, to within the tolerance."""
    p = small_problem(grid=(6, 5, 8), h=0.5, fd_order=4, n_wells=2, n_energies=5, e_range=(-3.0, -1.0),
                      eta=5e-2, tol=1e-11)
    H, P, wE = hamiltonian(p)
    Z = p.energies + 1j * p.eta
    f = lambda v: apply_h(H, P, wE, v)
    rows = boundary_rows(p.grid, p.n_face)
    b = np.zeros(p.N, complex)
    b[int(p.cols[1])] = 1.0
    Hd = dense_hamiltonian(p)
    xd = np.stack([np.linalg.solve(z * np.eye(p.N) - Hd, b)[rows] for z in Z])
    ref = oc.shifted_cocg(f, b, Z, p.tol, rows=rows)
    # 1) the first seed is an energy outside the set, far below the spectrum: it converges first and
    #    the seed moves into the set
    z_far = -12.0 + 5e-2j
    r1 = oc.shifted_cocg(f, b, Z, p.tol, rows=rows, seed=("aux", 0), aux=[z_far])
    assert r1.status == oc.OK and r1.seeds[0] == p.K and r1.switches >= 1 and r1.seeds[1] < p.K
    z_in = 1.7 + 3e-2j
    # 2) the set energies lie below the spectrum (fast); the auxiliary one inside it (slow) has the
    #    largest residual when the first seed converges, so the switch goes to it
    r2 = oc.shifted_cocg(f, b, Z, p.tol, rows=rows, seed="first", aux=[z_in])
    assert r2.status == oc.OK and p.K in r2.seeds[1:]
    for r in (r1, r2):
        assert np.linalg.norm(r.x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
        assert np.linalg.norm(r.x - xd) <= 1e-9 * np.linalg.norm(xd)
        assert r.x.shape == ref.x.shape and r.converged_at.shape == (p.K,)
