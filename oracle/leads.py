"""Self-energies of finite-difference leads (oracle; test infrastructure).

Eqs. self-energy and surface green's function define Sigma_L = B^dag g_L B and
Sigma_R = B g_R B^dag from the surface Green's function of a semi-infinite
electrode; Eqs. sec2-01, sec2-02 place Sigma on the outermost plane for the
central (N=1) stencil.  The paper gives no algorithm for the surface Green's
function (it defers to the OBM method).  Two independent routes are written
here for a lead that continues the transition region's grid with V = 0, the
same transverse walls and the same finite-difference order:

* ``sigma_bloch`` -- per transverse mode, the outgoing (|lambda| < 1) Bloch
  roots of the lead's difference equation along z.  With a stencil reaching
  R planes the lead couples to R planes of the transition region, so Sigma is
  an (R*Nxy) x (R*Nxy) block (reading: boundary slab of R planes per side).
* ``sigma_sancho_rubio`` -- the iterative decimation of Lopez Sancho et al.
  on principal layers of R planes, applied to the full transverse blocks.

Orderings: a slab holds its planes in increasing z, each plane x fastest.
Sign and branch: Z = E + i eta with eta > 0 (Eq. GF1), retarded branch.
"""

from __future__ import annotations

import numpy as np

from .operator import FD_SECOND_DERIVATIVE, kinetic_1d, transverse_modes


def z_hoppings(h, fd_order):
    """(d0, t1, ..., tR): the z-part of H's diagonal and the couplings to planes +-k."""
    c = FD_SECOND_DERIVATIVE[fd_order]
    return tuple(-0.5 * ck / (h * h) for ck in c)


def _bloch_roots_decaying(coeffs_desc):
    """Roots with |lambda| < 1 of the polynomial (numpy.roots, highest power first)."""
    r = np.roots(coeffs_desc)
    r = r[np.argsort(np.abs(r))]
    return r


def sigma_modes(eps, h, fd_order, Z):
    """Per-mode self-energy blocks sigma_m (R x R) of the RIGHT lead, slab planes in increasing z."""
    d = z_hoppings(h, fd_order)
    R = len(d) - 1
    out = np.zeros((eps.size, R, R), np.complex128)
    for m, e in enumerate(eps):
        if R == 1:
            t = d[1]                                   # H coupling between neighbouring planes
            # psi_k = lambda^k:  t lambda^2 + (d0 + e - Z) lambda + t = 0
            lam = _bloch_roots_decaying([t, d[0] + e - Z, t])[:1]
            # Sigma psi_T = H_{T,lead} psi_lead = t * lambda * psi_last
            out[m, 0, 0] = t * lam[0]
        else:
            t1, t2 = d[1], d[2]
            # t2 l^4 + t1 l^3 + (d0 + e - Z) l^2 + t1 l + t2 = 0
            lam = _bloch_roots_decaying([t2, t1, d[0] + e - Z, t1, t2])[:2]
            Phi = np.array([[1.0, 1.0], [lam[0], lam[1]]], np.complex128)
            M = Phi @ np.diag(lam ** 2) @ np.linalg.inv(Phi)   # (psi_{m+2}, psi_{m+3}) = M (psi_m, psi_{m+1})
            H01 = np.array([[t2, 0.0], [t1, t2]])               # slab planes (m, m+1) -> lead planes (m+2, m+3)
            out[m] = H01 @ M
    return out


def sigma_bloch(nx, ny, h, fd_order, Z):
    """(Sigma_L, Sigma_R) for a uniform V=0 lead, by Bloch roots per transverse mode."""
    eps, U = transverse_modes(nx, ny, h, fd_order)
    s = sigma_modes(eps, h, fd_order, Z)                    # [Nxy, R, R]
    R = s.shape[1]
    nxy = nx * ny
    SR = np.zeros((R * nxy, R * nxy), np.complex128)
    for a in range(R):
        for c in range(R):
            SR[a * nxy:(a + 1) * nxy, c * nxy:(c + 1) * nxy] = (U * s[:, a, c][None, :]) @ U.T
    # left lead: mirror image (reverse the order of the slab's planes)
    J = np.zeros((R, R))
    J[np.arange(R), R - 1 - np.arange(R)] = 1.0
    P = np.kron(J, np.eye(nxy))
    SL = P @ SR @ P.T
    return SL, SR


def _layer_blocks(nx, ny, h, fd_order, V_layer=None):
    """Principal-layer blocks of the lead (R planes per layer): H00, H01 (layer j -> j+1).

    ``V_layer`` (optional, [R, Ny, Nx]) is the local potential of one principal layer, repeated in
    every layer of the lead (a lead periodic along z with period R planes); it adds to H00's
    diagonal.  None means V = 0.
    """
    d = z_hoppings(h, fd_order)
    R = len(d) - 1
    nxy = nx * ny
    T2 = np.kron(np.eye(ny), kinetic_1d(nx, h, fd_order).toarray()) + \
        np.kron(kinetic_1d(ny, h, fd_order).toarray(), np.eye(nx))
    # full z-coupling between planes a and b: d[|a-b|] for |a-b| <= R
    def zc(k):
        return d[k] if k <= R else 0.0
    H00 = np.zeros((R * nxy, R * nxy))
    H01 = np.zeros((R * nxy, R * nxy))
    V = np.zeros((R, nxy)) if V_layer is None else np.asarray(V_layer, dtype=np.float64).reshape(R, nxy)
    for a in range(R):
        H00[a * nxy:(a + 1) * nxy, a * nxy:(a + 1) * nxy] = T2 + d[0] * np.eye(nxy) + np.diag(V[a])
        for c in range(R):
            if c != a:
                H00[a * nxy:(a + 1) * nxy, c * nxy:(c + 1) * nxy] = zc(abs(a - c)) * np.eye(nxy)
            # plane a of layer j to plane c of layer j+1: distance R + c - a
            H01[a * nxy:(a + 1) * nxy, c * nxy:(c + 1) * nxy] = zc(R + c - a) * np.eye(nxy)
    return H00, H01


def surface_gf_sancho_rubio(H00, H01, Z, tol=1e-15, maxit=10000):
    """Surface Green's function of a semi-infinite chain of layers (Lopez Sancho et al. decimation).

    The chain is H00 on each layer and H01 from layer j to layer j+1; the
    surface is layer 0.  Returns g_s = [(Z - H_eff)^{-1}] of the surface layer.
    """
    n = H00.shape[0]
    I = np.eye(n)
    eps_s = H00.astype(np.complex128).copy()
    eps = H00.astype(np.complex128).copy()
    alpha = H01.astype(np.complex128).copy()
    beta = H01.T.conj().astype(np.complex128).copy()
    for _ in range(maxit):
        g = np.linalg.inv(Z * I - eps)
        agb = alpha @ g @ beta
        bga = beta @ g @ alpha
        eps_s = eps_s + agb
        eps = eps + agb + bga
        alpha = alpha @ g @ alpha
        beta = beta @ g @ beta
        if np.abs(alpha).max() < tol and np.abs(beta).max() < tol:
            break
    return np.linalg.inv(Z * I - eps_s)


def sigma_sancho_rubio(nx, ny, h, fd_order, Z, V_left=None, V_right=None):
    """(Sigma_L, Sigma_R) from decimated surface Green's functions (Eq. self-energy).

    ``V_left`` / ``V_right`` ([R, Ny, Nx] or None) are the potentials of one principal layer of each
    lead, planes in increasing z; each lead repeats its layer (reading: a lead periodic along z whose
    period is the coupling range R, the smallest principal layer of the stencil).
    """
    H00R, H01 = _layer_blocks(nx, ny, h, fd_order, V_right)
    H00L, _ = _layer_blocks(nx, ny, h, fd_order, V_left)
    g = surface_gf_sancho_rubio(H00R, H01, Z)
    # right lead: slab (last R planes) couples to the lead's first layer through H01
    SR = H01 @ g @ H01.T
    # left lead: chain running to -z; its layer couplings are H01^T and the slab couples through H01^T
    gL = surface_gf_sancho_rubio(H00L, H01.T, Z)
    SL = H01.T @ gL @ H01
    return SL, SR


def open_channels(nx, ny, h, fd_order, E):
    """Number of transverse modes whose 1D band along z contains E (V = 0 lead)."""
    eps, _ = transverse_modes(nx, ny, h, fd_order)
    d = z_hoppings(h, fd_order)
    # band of the 1D z-chain: e(k) = d0 + 2 sum_m d_m cos(m k), k in [0, pi] (monotonic for orders 2, 4)
    kk = np.array([0.0, np.pi])
    band = d[0] + sum(2.0 * d[m] * np.cos(m * kk) for m in range(1, len(d)))
    lo, hi = band.min(), band.max()
    return int(np.sum((E - eps > lo) & (E - eps < hi)))
