"""Perturbed boundary Green's function from the unperturbed one (oracle; test infrastructure).

Eq. sec3-01a states G_T(:, l) = G0_T [Sigma_L G_T(z_0, l); 0; ...; I at l; ...;
Sigma_R G_T(z_{m+1}, l)], i.e. G = G0 + G0 Sigma G with Sigma nonzero only on
the boundary planes.  Restricted to the boundary rows b (both slabs) this is

    (I - G0_bb Sigma_bb) G_bb = G0_bb,   Sigma_bb = diag(Sigma_L, Sigma_R),

which ``dyson_solve`` evaluates with one dense LU per energy.  ``dyson_blocks``
evaluates the paper's explicit block formulas Eqs. sec3-02 ... sec3-06 (written
there for one plane per side; the same algebra holds for slabs of R planes).
"""

from __future__ import annotations

import numpy as np


def dyson_solve(G0_bb, Sigma_L, Sigma_R):
    """G_bb = (I - G0_bb Sigma_bb)^{-1} G0_bb for one energy (numpy.linalg.solve)."""
    nb = G0_bb.shape[0]
    ns = nb // 2
    S = np.zeros((nb, nb), np.complex128)
    S[:ns, :ns] = Sigma_L
    S[ns:, ns:] = Sigma_R
    return np.linalg.solve(np.eye(nb) - G0_bb @ S, G0_bb)


def dyson_blocks(G0_bb, Sigma_L, Sigma_R):
    """The four boundary blocks of G_T by Eqs. sec3-02 ... sec3-06.

    Returns (G_00, G_R0, G_0R, G_RR) where 0 is the left slab and R the right slab.
    """
    nb = G0_bb.shape[0]
    ns = nb // 2
    I = np.eye(ns)
    g00, g0R = G0_bb[:ns, :ns], G0_bb[:ns, ns:]
    gR0, gRR = G0_bb[ns:, :ns], G0_bb[ns:, ns:]
    inv = np.linalg.inv
    # modified unperturbed blocks (Eq. sec3-06 and the one before it)
    gt00 = g00 + g0R @ Sigma_R @ inv(I - gRR @ Sigma_R) @ gR0
    gtRR = gRR + gR0 @ Sigma_L @ inv(I - g00 @ Sigma_L) @ g0R
    # Eq. sec3-02 and the three that follow it
    G00 = gt00 @ inv(I - Sigma_L @ gt00)
    GR0 = inv(I - gRR @ Sigma_R) @ gR0 @ inv(I - Sigma_L @ gt00)
    G0R = inv(I - g00 @ Sigma_L) @ g0R @ inv(I - Sigma_R @ gtRR)
    GRR = gtRR @ inv(I - Sigma_R @ gtRR)
    return G00, GR0, G0R, GRR
