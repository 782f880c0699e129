"""Fisher-Lee transmission (oracle; test infrastructure).

Eq. TF: T(E) = Tr[Gamma_L G^a(z_0, z_{m+1}) Gamma_R G^r(z_{m+1}, z_0)] with
Gamma_X = i (Sigma_X - Sigma_X^dag) (the definition after Eq. TF).  The factor
written "Gamma_R(_{m+1}; E)" in the paper is read as Gamma_R(z_{m+1}; E), and
G^a(z_0, z_{m+1}) = [G^r(z_{m+1}, z_0)]^dag.  The retarded Green's function is
evaluated at the same finite eta as the solve; the eta -> 0 limit of the
definition is approached only in tests by taking eta small.
"""

from __future__ import annotations

import numpy as np


def gamma(Sigma):
    """Gamma = i (Sigma - Sigma^dag)."""
    return 1j * (Sigma - Sigma.conj().T)


def transmission(G_bb, Sigma_L, Sigma_R):
    """T = Tr[Gamma_L G_RL^dag Gamma_R G_RL], G_RL = G_bb[right slab, left slab]."""
    ns = G_bb.shape[0] // 2
    G_RL = G_bb[ns:, :ns]
    T = np.trace(gamma(Sigma_L) @ G_RL.conj().T @ gamma(Sigma_R) @ G_RL)
    return T.real, T.imag


def transmission_rl(G_bb, Sigma_L, Sigma_R):
    """The same formula with the leads exchanged: Tr[Gamma_R G_LR^dag Gamma_L G_LR]."""
    ns = G_bb.shape[0] // 2
    G_LR = G_bb[:ns, ns:]
    T = np.trace(gamma(Sigma_R) @ G_LR.conj().T @ gamma(Sigma_L) @ G_LR)
    return T.real, T.imag
