"""Exact-exchange action and energies (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. 2 (Sec. 2): the exchange operator built from orbitals {phi_j} acts on psi_p as

    (Vx psi_p)(r) = - sum_j phi_j(r) * integral phi_j(r') psi_p(r') / |r - r'| dr'

Orbitals are real.  Sec. 3.1 evaluates the integral as the Poisson potential of the
pair density phi_j psi_p; here that potential is ``coulomb.poisson_fft`` (or any
callable with the same signature).  The equation carries no occupation or spin factor
and none is added.  The discrete inner product is <f, g> = h^3 sum_r f(r) g(r).
"""
import numpy as np

from .coulomb import C0, poisson_fft, potential_at


def inner(f, g, h):
    """<f, g> = h^3 sum_r f(r) g(r), FP64."""
    return h ** 3 * float(np.dot(np.ravel(f).astype(np.float64), np.ravel(g).astype(np.float64)))


def pair_density(a, b):
    """rho(r) = a(r) b(r) for real orbitals (Sec. 3.1, the density solved for in Eq. 2)."""
    return np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)


def exchange_apply(phi, psi, h, poisson=poisson_fft):
    """Vx[phi] psi for every psi (Eq. 2).

    phi : (nocc, nz, ny, nx)   orbitals that define the operator
    psi : (npsi, nz, ny, nx)   functions it acts on
    returns (npsi, nz, ny, nx) FP64
    """
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    out = np.zeros_like(psi)
    for p in range(psi.shape[0]):
        for j in range(phi.shape[0]):
            v = poisson(pair_density(phi[j], psi[p]), h)
            out[p] -= phi[j] * v
    return out


def exchange_apply_bruteforce(phi, psi, h):
    """Eq. 2 as explicit loops over target r, source r' and orbital j (tiny grids only).

    The integral is the same discrete sum as ``poisson_direct``: h^3 sum_{r'} with
    kernel 1/(h|r - r'|) in grid units and C0/h on the diagonal.
    """
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    nz, ny, nx = phi.shape[1:]
    pts = [(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)]
    out = np.zeros_like(psi)
    for p in range(psi.shape[0]):
        for (z, y, x) in pts:
            acc = 0.0
            for j in range(phi.shape[0]):
                integral = 0.0
                for (zz, yy, xx) in pts:
                    d2 = (z - zz) ** 2 + (y - yy) ** 2 + (x - xx) ** 2
                    g = C0 / h if d2 == 0 else 1.0 / (h * d2 ** 0.5)
                    integral += phi[j, zz, yy, xx] * psi[p, zz, yy, xx] * g
                acc -= phi[j, z, y, x] * h ** 3 * integral
            out[p, z, y, x] = acc
    return out


def exchange_energy(phi, h, poisson=poisson_fft):
    """E_x = 1/2 sum_i <phi_i, Vx[phi] phi_i> (reading: the usual HF exchange energy,
    same-spin, no occupation factor, matching Eq. 2 as written)."""
    w = exchange_apply(phi, phi, h, poisson)
    return 0.5 * sum(inner(phi[i], w[i], h) for i in range(phi.shape[0]))


def hartree_energy(rho, h, poisson=poisson_fft):
    """E_H[rho] = 1/2 <rho, V[rho]>."""
    return 0.5 * inner(rho, poisson(rho, h), h)


def exchange_apply_at(phi, psi_p, h, points):
    """(Vx[phi] psi_p)(r) = -sum_j phi_j(r) V[phi_j psi_p](r) (Eq. 2) at selected grid
    points, each potential by the direct sum at those points (``potential_at``)."""
    phi = np.asarray(phi, dtype=np.float64)
    psi_p = np.asarray(psi_p, dtype=np.float64)
    out = np.zeros(len(points))
    for j in range(phi.shape[0]):
        v = potential_at(pair_density(phi[j], psi_p), h, points)
        out -= np.array([phi[j][tuple(int(c) for c in p)] for p in points]) * v
    return out

