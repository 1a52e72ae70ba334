"""Adaptively compressed exchange (ACE), FP64, CPU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1, Eqs. 11-13, in the paper's order:

1. W_i = Vx[{phi}] phi_i for every orbital of the set (Eq. 11).
2. M_kl = integral phi_k(r) W_l(r) dr.
3. Cholesky of -M:  M = -L L^T, L lower triangular.
4. zeta_k(r) = sum_i W_i(r) (L^{-T})_{ik}  (Eq. 12).
5. V^ACE(r, r') = - sum_k zeta_k(r) zeta_k(r')  (Eq. 13), so that
   V^ACE psi = - sum_k zeta_k <zeta_k, psi>.

Readings where the paper is silent or inconsistent:
* M is symmetrised as (M + M^T)/2 before the factorisation (exactly symmetric in
  exact arithmetic; the paper does not say what to do with rounding asymmetry).
* The operator carries the minus sign of Eq. 13.  Sec. 3.1 also writes the operator
  as zeta zeta^T without the sign; that cannot hold, because -M is the positive
  definite matrix that is factorised, so Eq. 13 is taken as the definition.
* Integrals are the grid sum h^3 sum_r.
"""
import numpy as np

from .coulomb import poisson_fft
from .exchange import exchange_apply


def ace_build(phi, h, poisson=poisson_fft, return_all=False):
    """Build the ACE projectors zeta (same shape as ``phi``) from orbitals ``phi``.

    Returns ``zeta`` or, with ``return_all``, ``(zeta, W, M, L)``.
    Raises ``numpy.linalg.LinAlgError`` when -M is not positive definite.
    """
    phi = np.asarray(phi, dtype=np.float64)
    k = phi.shape[0]
    W = exchange_apply(phi, phi, h, poisson)                      # Eq. 11
    phi2 = phi.reshape(k, -1)
    W2 = W.reshape(k, -1)
    M = h ** 3 * (phi2 @ W2.T)                                    # M_kl = <phi_k, W_l>
    M = 0.5 * (M + M.T)
    L = np.linalg.cholesky(-M)                                    # M = -L L^T
    LinvT = np.linalg.inv(L).T                                    # L^{-T}
    zeta2 = np.einsum("ir,ik->kr", W2, LinvT)                     # Eq. 12
    zeta = zeta2.reshape(phi.shape)
    if return_all:
        return zeta, W, M, L
    return zeta


def ace_apply(zeta, psi, h):
    """V^ACE psi = - sum_k zeta_k <zeta_k, psi>  (Eq. 13)."""
    zeta = np.asarray(zeta, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    k = zeta.shape[0]
    z2 = zeta.reshape(k, -1)
    p2 = psi.reshape(psi.shape[0], -1)
    C = h ** 3 * (z2 @ p2.T)                                      # C_kp = <zeta_k, psi_p>
    out = -(C.T @ z2)
    return out.reshape(psi.shape)
