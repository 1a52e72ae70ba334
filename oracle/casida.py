"""Tamm-Dancoff Casida coupling matrices and eigen-solve (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2, Eq. 6 defines the two-electron integral
    (pq|rs) = integral phi_p(r') phi_q(r') phi_r(r) phi_s(r) / |r - r'|
(real orbitals), and Eq. 7 the RHF Tamm-Dancoff matrix
    A_{ia,jb} = delta_ij delta_ab (eps_a - eps_i) + delta_M (ai|jb) - (ab|ji),
delta_M = 2 for singlets, 0 for triplets.  The TDA keeps only A (B = 0) and solves
A X = omega X, a symmetric problem (Sec. 2).  With both integral terms dropped the
excitation energies are the eigenvalue differences (independent-particle
approximation, Sec. 2).

Conventions (readings):
* transition index t = i * n_virt + a (row-major over (occupied, virtual));
* K_{ia,jb} = (ia|jb) = <rho_ia, V[rho_jb]>, rho_ia = phi_i phi_a;
* K_d[ia,jb] = (ab|ji) = <phi_a phi_b, V[phi_j phi_i]>;
* integrals are grid sums with the kernel of ``coulomb`` (V = h^3 sum rho g);
* eigenvalues ascending; energies in Hartree; 1 Ha = 27.211386245988 eV (CODATA 2018).
"""
import numpy as np

from .coulomb import C0, poisson_fft

HARTREE_EV = 27.211386245988


def transition_densities(phi_occ, phi_virt):
    """rho_t = phi_i phi_a for t = i * n_virt + a; shape (n_occ * n_virt, nz, ny, nx)."""
    phi_occ = np.asarray(phi_occ, dtype=np.float64)
    phi_virt = np.asarray(phi_virt, dtype=np.float64)
    no, nv = phi_occ.shape[0], phi_virt.shape[0]
    rho = np.empty((no * nv,) + phi_occ.shape[1:])
    for i in range(no):
        for a in range(nv):
            rho[i * nv + a] = phi_occ[i] * phi_virt[a]
    return rho


def casida_K(phi_occ, phi_virt, h, poisson=poisson_fft):
    """K_{ia,jb} = (ia|jb) = h^3 sum_r rho_ia(r) V[rho_jb](r); symmetric (n_t, n_t)."""
    rho = transition_densities(phi_occ, phi_virt)
    nt = rho.shape[0]
    V = np.stack([poisson(rho[s], h) for s in range(nt)])
    return h ** 3 * (rho.reshape(nt, -1) @ V.reshape(nt, -1).T)


def casida_K_bruteforce(phi_occ, phi_virt, h):
    """(ia|jb) as the explicit double grid sum of Eq. 6 (tiny grids only).

    (ia|jb) = h^6 sum_r sum_r' phi_i(r') phi_a(r') phi_j(r) phi_b(r) g(r - r'),
    g = 1/(h |r - r'|) in grid units, C0/h on the diagonal.
    """
    phi_occ = np.asarray(phi_occ, dtype=np.float64)
    phi_virt = np.asarray(phi_virt, dtype=np.float64)
    nz, ny, nx = phi_occ.shape[1:]
    coords = np.array([(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)],
                      dtype=np.float64)
    G = np.empty((coords.shape[0], coords.shape[0]))
    for u in range(coords.shape[0]):
        d = np.sqrt(((coords - coords[u]) ** 2).sum(axis=1))
        with np.errstate(divide="ignore"):
            G[u] = np.where(d == 0, C0 / h, 1.0 / (h * np.where(d == 0, 1.0, d)))
    no, nv = phi_occ.shape[0], phi_virt.shape[0]
    nt = no * nv
    K = np.empty((nt, nt))
    for i in range(no):
        for a in range(nv):
            left = (phi_occ[i] * phi_virt[a]).ravel()
            for j in range(no):
                for b in range(nv):
                    right = (phi_occ[j] * phi_virt[b]).ravel()
                    K[i * nv + a, j * nv + b] = h ** 6 * (right @ G @ left)
    return K


def casida_Kd(phi_occ, phi_virt, h, poisson=poisson_fft):
    """K_d[ia,jb] = (ab|ji) = h^3 sum_r phi_a phi_b V[phi_j phi_i] (the Coulomb term of Eq. 7)."""
    phi_occ = np.asarray(phi_occ, dtype=np.float64)
    phi_virt = np.asarray(phi_virt, dtype=np.float64)
    no, nv = phi_occ.shape[0], phi_virt.shape[0]
    nt = no * nv
    Kd = np.empty((nt, nt))
    pv = phi_virt.reshape(nv, -1)
    for i in range(no):
        for j in range(no):
            vji = poisson(phi_occ[j] * phi_occ[i], h).ravel()
            block = h ** 3 * ((pv * vji) @ pv.T)          # [a, b]
            Kd[i * nv:(i + 1) * nv, j * nv:(j + 1) * nv] = block
    return Kd


def tda_matrix(eps_occ, eps_virt, K, Kd=None, delta_M=2.0):
    """A = diag(eps_a - eps_i) + delta_M K - K_d  (Eq. 7; K_d omitted when None)."""
    eps_occ = np.asarray(eps_occ, dtype=np.float64)
    eps_virt = np.asarray(eps_virt, dtype=np.float64)
    de = (eps_virt[None, :] - eps_occ[:, None]).ravel()
    A = np.diag(de) + delta_M * np.asarray(K, dtype=np.float64)
    if Kd is not None:
        A = A - np.asarray(Kd, dtype=np.float64)
    return A


def tda_solve(A, nroots):
    """Lowest ``nroots`` eigenpairs of the symmetric TDA matrix, ascending.

    Returns (omega [nroots], X [nroots, n_t]) with X rows the eigenvectors.
    """
    w, v = np.linalg.eigh(0.5 * (A + A.T))
    return w[:nroots], v[:, :nroots].T


# ---------------------------------------------------------------- spin-polarised (UHF) TDA
#
# Sec. 2, Eqs. 4-5 in spin orbitals: A_{ia,jb} = delta_ij delta_ab (eps_a - eps_i)
# + (ia|jb) - (ij|ab), with every integral zero unless the spins pair up inside each
# density.  For real spatial orbitals of spins s (i, a) and t (j, b): (ia|jb) couples
# every pair of spin blocks (the Coulomb-type term), (ij|ab) = (ab|ji) = K_d only within
# one spin (s = t).  Readings: alpha transitions first, t = i * n_virt + a within a spin.


def uhf_K(occ_a, virt_a, occ_b, virt_b, h, poisson=poisson_fft):
    """(ia|jb) over the alpha then beta transitions; symmetric (n_ta + n_tb) square."""
    rho = [transition_densities(occ_a, virt_a)]
    if len(occ_b) and len(virt_b):
        rho.append(transition_densities(occ_b, virt_b))
    rho = np.concatenate(rho)
    nt = rho.shape[0]
    V = np.stack([poisson(rho[s], h) for s in range(nt)])
    return h ** 3 * (rho.reshape(nt, -1) @ V.reshape(nt, -1).T)


def uhf_tda_matrix(eo_a, ev_a, eo_b, ev_b, K, Kd_a=None, Kd_b=None):
    """A = diag(eps_a - eps_i per spin) + K - blockdiag(K_d alpha, K_d beta)."""
    de = [(np.asarray(ev_a, dtype=np.float64)[None, :] - np.asarray(eo_a, dtype=np.float64)[:, None]).ravel()]
    if len(eo_b) and len(ev_b):
        de.append((np.asarray(ev_b, dtype=np.float64)[None, :] - np.asarray(eo_b, dtype=np.float64)[:, None]).ravel())
    de = np.concatenate(de)
    A = np.diag(de) + np.asarray(K, dtype=np.float64)
    na = len(eo_a) * len(ev_a)
    if Kd_a is not None:
        A[:na, :na] -= np.asarray(Kd_a, dtype=np.float64)
    if Kd_b is not None:
        A[na:, na:] -= np.asarray(Kd_b, dtype=np.float64)
    return A
