"""Pins of the oracle's self-energies, Dyson step and transmission.

* Sigma (Eq. self-energy): the Bloch-root closed form agrees with Sancho-Rubio
  decimation (an independent iterative route) and with a brute-force long
  finite lead; it is complex symmetric and Gamma = i(Sigma - Sigma^dag) is
  positive semidefinite.
* For a V=0 wire with the 2nd-order stencil, G_T between any two planes equals
  the infinite wire's closed form  sum_m u_m u_m^T lambda_m^{|k-k'|} /
  (t (lambda_m - 1/lambda_m))  (pins Sigma and the dense Eq. GF2 together).
* Dyson (Eq. sec3-01a) applied to the dense G0_bb reproduces the boundary block
  of the dense (Z - H - Sigma)^{-1}, and so do the block formulas
  Eqs. sec3-02 ... sec3-06.
* Eq. TF: a uniform V=0 wire transmits exactly its number of open channels as
  eta -> 0 (1, 3 or 4 channels at the tested energies), T_LR = T_RL, and
  0 <= T <= N_open with wells.
"""

import numpy as np
import pytest

from workloads import small_problem
from oracle.operator import boundary_rows, transverse_modes
from oracle.leads import sigma_bloch, sigma_sancho_rubio, open_channels, z_hoppings, _layer_blocks
from oracle.dense import g0_dense, g_dense
from oracle.dyson import dyson_solve, dyson_blocks
from oracle.transmission import transmission, transmission_rl, gamma


@pytest.mark.parametrize("order,eta,tol", [(2, 1e-3, 1e-10), (2, 1e-1, 1e-12), (4, 1e-3, 1e-8), (4, 5e-2, 1e-10)])
def test_sigma_bloch_vs_sancho_rubio(order, eta, tol):
    nx, ny, h = 4, 3, 0.5
    for E in (0.3, 1.7, 4.5):
        Z = E + 1j * eta
        SL, SR = sigma_bloch(nx, ny, h, order, Z)
        SL2, SR2 = sigma_sancho_rubio(nx, ny, h, order, Z)
        scale = np.abs(SR2).max()
        assert np.abs(SR - SR2).max() < tol * max(scale, 1.0)
        assert np.abs(SL - SL2).max() < tol * max(scale, 1.0)
        for S in (SL, SR):
            assert np.abs(S - S.T).max() < 1e-12 * max(scale, 1.0)
            assert np.linalg.eigvalsh(gamma(S)).min() > -1e-10


@pytest.mark.parametrize("order", [2, 4])
def test_sigma_vs_long_finite_lead(order):
    # brute force: a finite lead of L layers, eta large enough that |lambda|^(2L) is negligible
    nx, ny, h, eta, L = 2, 2, 0.5, 0.2, 120
    Z = 1.3 + 1j * eta
    H00, H01 = _layer_blocks(nx, ny, h, order)
    n = H00.shape[0]
    M = np.zeros((L * n, L * n), complex)
    for j in range(L):
        M[j * n:(j + 1) * n, j * n:(j + 1) * n] = Z * np.eye(n) - H00
        if j + 1 < L:
            M[j * n:(j + 1) * n, (j + 1) * n:(j + 2) * n] = -H01
            M[(j + 1) * n:(j + 2) * n, j * n:(j + 1) * n] = -H01.T
    g = np.linalg.inv(M)[:n, :n]
    SR_brute = H01 @ g @ H01.T
    _, SR = sigma_bloch(nx, ny, h, order, Z)
    assert np.abs(SR - SR_brute).max() < 1e-10 * np.abs(SR).max()


def test_infinite_wire_closed_form():
    p = small_problem(grid=(3, 4, 6), h=0.5, fd_order=2, n_wells=0, n_face=1)
    Z = 0.9 + 1e-2j
    SL, SR = sigma_bloch(*p.grid[:2], p.h, 2, Z)
    G = g_dense(p, Z, SL, SR)
    eps, U = transverse_modes(p.grid[0], p.grid[1], p.h, 2)
    d0, t1 = z_hoppings(p.h, 2)
    t = -t1
    nxy, nz = p.Nxy, p.grid[2]
    for k in range(nz):
        for kp in (0, nz - 1, k):
            blk = G[k * nxy:(k + 1) * nxy, kp * nxy:(kp + 1) * nxy]
            want = np.zeros((nxy, nxy), complex)
            for m, e in enumerate(eps):
                lam = np.roots([t, (Z - e - d0), t])
                lam = lam[np.argmin(np.abs(lam))]
                want += np.outer(U[:, m], U[:, m]) * lam ** abs(k - kp) / (t * (lam - 1.0 / lam))
            assert np.abs(blk - want).max() < 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("order,proj", [(2, 0), (4, 0), (4, 1)])
def test_dyson_matches_dense_perturbed(order, proj):
    p = small_problem(grid=(4, 3, 8), h=0.5, fd_order=order, n_wells=2, projectors=proj)
    b = boundary_rows(p.grid, p.n_face)
    ns = b.size // 2
    for E in (0.4, 1.9):
        Z = E + 1e-2j
        SL, SR = sigma_bloch(p.grid[0], p.grid[1], p.h, order, Z)
        G0 = g0_dense(p, Z, rows=b, cols=b)
        G = dyson_solve(G0, SL, SR)
        Gd = g_dense(p, Z, SL, SR, rows=b, cols=b)
        assert np.abs(G - Gd).max() < 1e-10 * np.abs(Gd).max()
        G00, GR0, G0R, GRR = dyson_blocks(G0, SL, SR)
        for blk, want in ((G00, Gd[:ns, :ns]), (GR0, Gd[ns:, :ns]), (G0R, Gd[:ns, ns:]), (GRR, Gd[ns:, ns:])):
            assert np.abs(blk - want).max() < 1e-10 * np.abs(Gd).max()


@pytest.mark.parametrize("order,E,n_open", [(2, 3.0, 1), (2, 7.5, 3), (4, 3.0, 1), (4, 8.0, 3), (4, 10.0, 4)])
def test_uniform_wire_integer_transmission(order, E, n_open):
    p = small_problem(grid=(3, 3, 6), h=0.5, fd_order=order, n_wells=0)
    assert open_channels(3, 3, p.h, order, E) == n_open
    b = boundary_rows(p.grid, p.n_face)
    Z = E + 1e-9j
    SL, SR = sigma_bloch(3, 3, p.h, order, Z)
    G = g_dense(p, Z, SL, SR, rows=b, cols=b)
    T, Ti = transmission(G, SL, SR)
    assert abs(T - n_open) < 1e-5 and abs(Ti) < 1e-6


def test_transmission_symmetry_and_bounds():
    p = small_problem(grid=(4, 3, 8), h=0.5, fd_order=4, n_wells=3, projectors=1)
    b = boundary_rows(p.grid, p.n_face)
    for E in np.linspace(0.5, 8.0, 7):
        Z = E + 1e-7j
        SL, SR = sigma_bloch(4, 3, p.h, 4, Z)
        G = g_dense(p, Z, SL, SR, rows=b, cols=b)
        T, _ = transmission(G, SL, SR)
        T2, _ = transmission_rl(G, SL, SR)
        assert abs(T - T2) < 1e-8
        assert -1e-8 <= T <= open_channels(4, 3, p.h, 4, E) + 1e-6


def test_planted_sigma_mistake_is_caught():
    # dropping the second plane's coupling (treating the 4th-order lead as 1-plane) breaks integer T
    p = small_problem(grid=(3, 3, 6), h=0.5, fd_order=4, n_wells=0)
    b = boundary_rows(p.grid, p.n_face)
    Z = 3.0 + 1e-9j
    SL, SR = sigma_bloch(3, 3, p.h, 4, Z)
    ns = SR.shape[0] // 2
    SR_bad = SR.copy()
    SR_bad[:ns, :] = 0
    SR_bad[:, :ns] = 0
    G = g_dense(p, Z, SL, SR_bad, rows=b, cols=b)
    T, _ = transmission(G, SL, SR_bad)
    assert abs(T - 1.0) > 1e-2


@pytest.mark.parametrize("order", [2, 4])
def test_sancho_rubio_constant_lead_potential_is_an_energy_shift(order):
    """A constant lead potential v0 shifts the lead's spectrum: Sigma(Z; V = v0) = Sigma(Z - v0; V = 0),
    and at V = 0 the decimation equals the Bloch-root closed form."""
    nx, ny, h, Z, v0 = 4, 3, 0.5, 1.3 + 2e-2j, 0.37
    R = order // 2
    SL0, SR0 = sigma_sancho_rubio(nx, ny, h, order, Z - v0)
    SLv, SRv = sigma_sancho_rubio(nx, ny, h, order, Z, V_left=np.full((R, ny, nx), v0),
                                  V_right=np.full((R, ny, nx), v0))
    assert np.abs(SLv - SL0).max() <= 1e-11 * np.abs(SL0).max()
    assert np.abs(SRv - SR0).max() <= 1e-11 * np.abs(SR0).max()
    SLb, SRb = sigma_bloch(nx, ny, h, order, Z - v0)
    assert np.abs(SR0 - SRb).max() <= 1e-9 * np.abs(SRb).max()


@pytest.mark.parametrize("order", [2, 4])
def test_sancho_rubio_periodic_lead_fixed_point(order):
    """A lead with a random layer potential: the decimated surface Green's function satisfies its own
    defining relation g = (Z - H00 - H01 g H01^T)^{-1} (right lead) and the left lead's mirror form, and
    Sigma is complex symmetric with a negative semidefinite anti-Hermitian part (retarded)."""
    from oracle.leads import surface_gf_sancho_rubio
    rng = np.random.Generator(np.random.PCG64(5))
    nx, ny, h, Z = 4, 3, 0.5, 0.9 + 1e-2j
    R = order // 2
    VL = rng.uniform(-0.6, 0.2, size=(R, ny, nx))
    VR = rng.uniform(-0.6, 0.2, size=(R, ny, nx))
    H00R, H01 = _layer_blocks(nx, ny, h, order, VR)
    H00L, _ = _layer_blocks(nx, ny, h, order, VL)
    n = H00R.shape[0]
    g = surface_gf_sancho_rubio(H00R, H01, Z)
    res = np.linalg.inv(g) - (Z * np.eye(n) - H00R - H01 @ g @ H01.T)
    assert np.abs(res).max() <= 1e-9 * np.abs(np.linalg.inv(g)).max()
    gL = surface_gf_sancho_rubio(H00L, H01.T, Z)
    resL = np.linalg.inv(gL) - (Z * np.eye(n) - H00L - H01.T @ gL @ H01)
    assert np.abs(resL).max() <= 1e-9 * np.abs(np.linalg.inv(gL)).max()
    SL, SR = sigma_sancho_rubio(nx, ny, h, order, Z, V_left=VL, V_right=VR)
    for S in (SL, SR):
        assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
        assert np.linalg.eigvalsh(0.5j * (S - S.conj().T)).min() >= -1e-12
    # the lead potential changes Sigma (the layer potential enters the decimation)
    SL0, SR0 = sigma_sancho_rubio(nx, ny, h, order, Z)
    assert np.abs(SR - SR0).max() > 1e-2 * np.abs(SR0).max()
    assert np.abs(SL - SL0).max() > 1e-2 * np.abs(SL0).max()
