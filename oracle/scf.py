"""Closed-shell Hartree-Fock ground state by self-consistent iteration, with or without
ACE (FP64, CPU, small grids).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1: inside the SCF cycle the exchange operator of Eq. 2 is built from the current
orbitals; with ACE (Eqs. 11-13) the full exchange is evaluated once per SCF iteration
and the compressed operator is used for the rest of it, and at self-consistency the two
give the same result ("not an approximation").  Sec. 3.2: linear mixing
q_{N+1} = alpha q_{N-1} + (1 - alpha) q_N (Eq. 14) and, Sec. 3.4, the relative density
error eps = (1/N_e) integral |rho_in - rho_out| (Eq. 15) as the convergence measure.

Readings (the paper is silent on these details):
* closed shell, N_e = 2 n_occ electrons, rho = 2 sum_i phi_i^2;
* Hartree potential V_H = V[rho] with the discrete kernel of ``coulomb``;
* exchange: Eq. 2 over the n_occ occupied spatial orbitals (same spin), no factor;
* Fock operator F = -1/2 Lap_FD4 + V_ext + V_H + Vx, Vx built from the orbitals of the
  previous iteration (exact) or its ACE form -zeta zeta^T (ACE);
* mixing of the density: rho_in <- alpha rho_in + (1 - alpha) rho_out (q_{N-1} read as
  the input density of iteration N, q_N as its output);
* mixing of the states (Sec. 3.2 finds it the most robust): the input orbitals of the
  next iteration are alpha phi_in + (1 - alpha) P_out phi_in, orthonormalised by the
  Cholesky factor of their overlap, with P_out the projector on the span of the output
  orbitals (the output orbital space carried over without the arbitrary signs and
  rotations of an eigensolver); the Fock operator of an iteration takes both V_H and Vx
  from its input orbitals;
* energy E = 2 sum_i <phi_i, (T + V_ext) phi_i> + 1/2 <rho, V_H> + sum_i <phi_i, Vx phi_i>;
* each iteration takes the n_occ lowest eigenvectors of the dense Fock matrix (small
  grids only), starting from the non-interacting orbitals of T + V_ext.
"""
import numpy as np

from .ace import ace_build
from .coulomb import C0
from .eigensolver import hamiltonian_dense


def coulomb_matrix(shape, h):
    """G[r, r'] = h^3 g(r - r') on the box: V = G rho is the Poisson solve written out."""
    nz, ny, nx = shape
    idx = np.array([(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)], dtype=np.float64)
    d = np.sqrt(((idx[:, None, :] - idx[None, :, :]) ** 2).sum(axis=2))
    with np.errstate(divide="ignore"):
        g = np.where(d == 0, C0 / h, 1.0 / (h * np.where(d == 0, 1.0, d)))
    return h ** 3 * g


def density(phi):
    """rho = 2 sum_i phi_i^2 (closed shell)."""
    phi = np.asarray(phi, dtype=np.float64)
    return 2.0 * np.sum(phi * phi, axis=0)


def exchange_matrix(phi, G):
    """Vx[r, r'] = - sum_j phi_j(r) G[r, r'] phi_j(r') (Eq. 2 as a matrix on the grid)."""
    P = np.asarray(phi, dtype=np.float64).reshape(phi.shape[0], -1)
    return -sum(P[j][:, None] * G * P[j][None, :] for j in range(P.shape[0]))


def hf_energy(phi, v_ext, h, G):
    """E = 2 sum_i <phi_i, (T + V_ext) phi_i> + 1/2 <rho, V_H> + sum_i <phi_i, Vx phi_i>."""
    phi = np.asarray(phi, dtype=np.float64)
    k = phi.shape[0]
    H0 = hamiltonian_dense(v_ext, h)
    P = phi.reshape(k, -1)
    rho = density(phi).ravel()
    one = 2.0 * h ** 3 * np.einsum("ir,rs,is->", P, H0, P)
    eh = 0.5 * h ** 3 * rho @ (G @ rho)
    ex = h ** 3 * np.einsum("ir,rs,is->", P, exchange_matrix(phi, G), P)
    return one + eh + ex, one, eh, ex


def mix_states(phi_in, phi_out, h, alpha):
    """alpha phi_in + (1 - alpha) P_out phi_in, orthonormalised (Cholesky of the overlap)."""
    k = phi_in.shape[0]
    A = np.asarray(phi_in, dtype=np.float64).reshape(k, -1)
    B = np.asarray(phi_out, dtype=np.float64).reshape(k, -1)
    O = h ** 3 * B @ A.T                         # O[i, j] = <out_i, in_j>
    mixed = alpha * A + (1.0 - alpha) * (O.T @ B)
    L = np.linalg.cholesky(h ** 3 * mixed @ mixed.T)
    return np.linalg.solve(L, mixed).reshape(phi_in.shape)


def scf(v_ext, h, nocc, mode="ace", alpha=0.3, tol=1e-10, max_iter=300, mix="density", mask=None):
    """Self-consistent closed-shell HF on a small grid; mode 'ace' or 'exact', mix
    'density' or 'states'; with `mask` (0/1 per point, e.g. eigensolver.sphere_mask) the
    orbitals live on the kept points only (spherical domain, Sec. 3.4).

    Returns a dict with the orbitals, orbital energies, total energy (and its parts), the
    last relative density error and the iteration count."""
    v_ext = np.asarray(v_ext, dtype=np.float64)
    shape = v_ext.shape
    n = v_ext.size
    G = coulomb_matrix(shape, h)
    H0 = hamiltonian_dense(v_ext, h)
    # the kept points (all of them without a mask): every matrix below lives on them
    keep = np.arange(n) if mask is None else np.flatnonzero(np.asarray(mask).ravel() > 0)
    Gk, H0k = G[np.ix_(keep, keep)], H0[np.ix_(keep, keep)]

    def full(U):
        phi = np.zeros((nocc, n))
        phi[:, keep] = U[:, :nocc].T / h ** 1.5
        return phi.reshape((nocc,) + shape)

    w, U = np.linalg.eigh(0.5 * (H0k + H0k.T))
    phi = full(U)
    rho_in = density(phi).ravel()
    phi_in = phi
    eps, it = np.inf, 0
    for it in range(1, max_iter + 1):
        VH = Gk @ rho_in[keep]
        src = phi_in if mix == "states" else phi      # orbitals the exchange is built from
        if mode == "ace":
            zeta = ace_build(src, h).reshape(nocc, -1)[:, keep]
            VX = -h ** 3 * (zeta.T @ zeta)
        else:
            P = np.asarray(src).reshape(nocc, -1)[:, keep]
            VX = -sum(P[j][:, None] * Gk * P[j][None, :] for j in range(nocc))
        F = H0k + np.diag(VH) + VX
        w, U = np.linalg.eigh(0.5 * (F + F.T))
        phi = full(U)
        rho_out = density(phi).ravel()
        eps = h ** 3 * np.abs(rho_out - rho_in).sum() / (2 * nocc)
        if mix == "states":
            phi_in = mix_states(phi_in, phi, h, alpha)
            rho_in = density(phi_in).ravel()
        else:
            rho_in = alpha * rho_in + (1.0 - alpha) * rho_out
        if eps < tol:
            break
    E, one, eh, ex = hf_energy(phi, v_ext, h, G)
    return {"phi": phi, "eps_orb": w[:nocc], "energy": E, "one_body": one, "hartree": eh, "exchange": ex,
            "reldens": eps, "iters": it, "n": n}
