"""Absorption spectrum from Casida eigenvectors and the full (non-Tamm-Dancoff) TDHF
problem (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2 (after Eq. 7): the many-body transition dipole of excitation k is the
combination d_k = sum_ia <i|r|a> x_{k,ia} of single-particle dipole matrix elements
(Eq. 8); the isotropically averaged oscillator strength is f_k = (2 m_e / 3 hbar^2)
omega_k |d_k|^2 (Eq. 9); the strength function is S(omega) = sum_k f_k
delta(omega - omega_k) (Eq. 10), broadened in practice by a Lorentzian.

The full problem (Eq. 3) couples excitations X and de-excitations Y through A and B
(Eqs. 4-5).  For real orbitals it is equivalent to a symmetric problem of half the
size (Sec. 2): omega^2 are the eigenvalues of (A - B)^{1/2} (A + B) (A - B)^{1/2}.

Readings:
* position r = ((x - nx/2) h, (y - ny/2) h, (z - nz/2) h), the box convention of the
  rest of the oracle; components ordered (x, y, z), x the fastest grid axis;
* <i|r_d|a> = h^3 sum_r phi_i(r) r_d phi_a(r); Eq. 8 as written (no spin factor: the
  closed-shell singlet total over both spins is twice f_k);
* atomic units m_e = hbar = 1, so f_k = (2/3) omega_k |d_k|^2;
* Lorentzian of half-width gamma: L(x) = gamma / (pi (x^2 + gamma^2));
* RHF B, spin-adapted like Eq. 7: B_{ia,jb} = delta_M (ia|bj) - (ib|aj); for real
  orbitals (ia|bj) = K[ia, jb] and (ib|aj) = K[ib, ja] (transition index t = i n_v + a);
* half-size form by Cholesky: A - B = L L^T, M = L^T (A + B) L = Z diag(omega^2) Z^T,
  X + Y = omega^{-1/2} L z (normalised so that X^T X - Y^T Y = 1).
"""
import numpy as np


def positions(shape, h):
    """Grid coordinates (x, y, z) arrays of the given (nz, ny, nx) box."""
    nz, ny, nx = shape
    z = (np.arange(nz) - nz / 2) * h
    y = (np.arange(ny) - ny / 2) * h
    x = (np.arange(nx) - nx / 2) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def dipole_matrix(phi_occ, phi_virt, h):
    """dip[d, i * n_v + a] = <i|r_d|a> (d = x, y, z); shape (3, n_occ * n_virt)."""
    phi_occ = np.asarray(phi_occ, dtype=np.float64)
    phi_virt = np.asarray(phi_virt, dtype=np.float64)
    no, nv = phi_occ.shape[0], phi_virt.shape[0]
    dip = np.empty((3, no * nv))
    for d, R in enumerate(positions(phi_occ.shape[1:], h)):
        for i in range(no):
            for a in range(nv):
                dip[d, i * nv + a] = h ** 3 * np.sum(phi_occ[i] * R * phi_virt[a])
    return dip


def transition_dipoles(X, dip):
    """d_k = sum_t X[k, t] dip[:, t] (Eq. 8); shape (n_roots, 3)."""
    return np.asarray(X, dtype=np.float64) @ np.asarray(dip, dtype=np.float64).T


def oscillator_strengths(omega, X, dip):
    """f_k = (2/3) omega_k |d_k|^2 (Eq. 9, atomic units)."""
    d = transition_dipoles(X, dip)
    return (2.0 / 3.0) * np.asarray(omega, dtype=np.float64) * np.sum(d * d, axis=1)


def strength_function(grid, omega, f, gamma):
    """S(w) = sum_k f_k gamma / (pi ((w - omega_k)^2 + gamma^2)) on the given grid (Eq. 10)."""
    grid = np.asarray(grid, dtype=np.float64)
    S = np.zeros_like(grid)
    for wk, fk in zip(omega, f):
        S += fk * gamma / (np.pi * ((grid - wk) ** 2 + gamma ** 2))
    return S


def exchange_permuted(K, n_occ, n_virt):
    """Kx[ia, jb] = K[ib, ja] = (ib|aj) for real orbitals."""
    K = np.asarray(K, dtype=np.float64)
    Kx = np.empty_like(K)
    for i in range(n_occ):
        for a in range(n_virt):
            for j in range(n_occ):
                for b in range(n_virt):
                    Kx[i * n_virt + a, j * n_virt + b] = K[i * n_virt + b, j * n_virt + a]
    return Kx


def tdhf_matrices(eps_occ, eps_virt, K, Kd=None, delta_M=2.0):
    """A (Eq. 7) and B = delta_M K - Kx of the RHF linear-response problem."""
    eps_occ = np.asarray(eps_occ, dtype=np.float64)
    eps_virt = np.asarray(eps_virt, dtype=np.float64)
    no, nv = eps_occ.size, eps_virt.size
    K = np.asarray(K, dtype=np.float64)
    de = (eps_virt[None, :] - eps_occ[:, None]).ravel()
    A = np.diag(de) + delta_M * K
    if Kd is not None:
        A = A - np.asarray(Kd, dtype=np.float64)
    B = delta_M * K - exchange_permuted(K, no, nv)
    return A, B


def tdhf_solve(A, B, nroots):
    """Lowest ``nroots`` excitation energies and X + Y of the full problem (half-size form).

    A - B must be positive definite (a stable ground state)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    L = np.linalg.cholesky(0.5 * ((A - B) + (A - B).T))
    M = L.T @ (0.5 * ((A + B) + (A + B).T)) @ L
    w2, Z = np.linalg.eigh(0.5 * (M + M.T))
    omega = np.sqrt(w2[:nroots])
    XpY = (L @ Z[:, :nroots]) / np.sqrt(omega)[None, :]
    return omega, XpY.T


def tdhf_solve_nonhermitian(A, B):
    """All positive eigenvalues of the 2n x 2n problem of Eq. 3 (real orbitals),
    [[A, B], [-B, -A]] [X; Y] = omega [X; Y], and X + Y for each (normalised to
    X^T X - Y^T Y = 1), ascending."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n = A.shape[0]
    big = np.block([[A, B], [-B, -A]])
    w, v = np.linalg.eig(big)
    w = w.real
    v = v.real
    keep = np.argsort(w)[n:]                 # the n positive roots
    out_w, out_v = [], []
    for k in keep:
        X, Y = v[:n, k], v[n:, k]
        norm = X @ X - Y @ Y
        s = 1.0 / np.sqrt(norm)
        out_w.append(w[k])
        out_v.append((X + Y) * s)
    return np.array(out_w), np.array(out_v)
