"""Discrete isolated-boundary Coulomb kernel and Poisson solve (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is being discretised
-------------------------
Sec. 3.1 of the paper turns the integral of Eq. 2 into a Poisson problem for the
pair density rho = psi_j psi_p, solved at O(N log N) cost instead of the O(N^2)
direct integral.  Sec. 3.4: the grid is uniform with spacing h and the orbitals
vanish outside the domain (zero boundary condition).

The paper does not say which discrete kernel its solver uses.  Our reading:

* potential of a density sampled on the box ``[nz, ny, nx]`` at spacing h::

      V(r) = h^3 * sum_{r'} rho(r') g(r - r')

* kernel samples for an integer offset d (in grid units)::

      g(d) = 1 / (h |d|)            d != 0
      g(0) = C0 / h,   C0 = 3 ln(2 + sqrt 3) - pi/2

  where C0 is the exact integral of 1/|r| over a unit cube centred on the origin,
  i.e. g(0) is the cell average of 1/r.

Padding the box to M = 2n per axis makes every in-box offset satisfy |d_i| <= n - 1
< M/2, so the M-periodic (FFT) convolution equals the aperiodic sum exactly, up to
rounding.  ``poisson_direct`` is that sum written out; ``poisson_fft`` is the same
quantity through a library FFT (a step the definition allows).
"""
import math

import numpy as np

# Integral of 1/|r| over the cube [-1/2, 1/2]^3 (closed form).
C0 = 3.0 * math.log(2.0 + math.sqrt(3.0)) - math.pi / 2.0


def _offsets(m):
    """Periodic integer offsets 0, 1, ..., m/2 - 1, -m/2, ..., -1 for an axis of m points."""
    i = np.arange(m)
    return np.where(i < m // 2, i, i - m).astype(np.float64)


def kernel_samples(shape_padded, h):
    """g(d) on the padded periodic grid ``shape_padded = (Mz, My, Mx)`` (FP64).

    Entry [a, b, c] holds g at the periodic offset (dz, dy, dx) of that index.
    Offsets with |d_i| = M_i/2 never meet an in-box (target, source) pair and their
    values do not change any in-box result; they are filled with the same 1/(h|d|).
    """
    dz, dy, dx = (_offsets(m) for m in shape_padded)
    dist = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        g = 1.0 / (h * dist)
    g[0, 0, 0] = C0 / h
    return g


def padded_shape(shape):
    return tuple(2 * int(s) for s in shape)


def kernel_spectrum(shape_padded, h):
    """Unnormalised forward DFT of the kernel samples, half spectrum along x.

    Real and even: the returned array is the real part of ``rfftn(g)``; shape
    ``(Mz, My, Mx//2 + 1)``.
    """
    return np.fft.rfftn(kernel_samples(shape_padded, h), axes=(0, 1, 2)).real


def poisson_fft(rho, h, ghat=None):
    """Isolated-boundary potential of ``rho`` (shape ``(nz, ny, nx)``, FP64).

    V = h^3 * IDFT( ghat * DFT(rho zero-padded to 2n) ) restricted to the box.
    """
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    mp = padded_shape(shape)
    if ghat is None:
        ghat = kernel_spectrum(mp, h)
    pad = np.zeros(mp)
    pad[: shape[0], : shape[1], : shape[2]] = rho
    spec = np.fft.rfftn(pad, axes=(0, 1, 2)) * ghat
    v = np.fft.irfftn(spec, s=mp, axes=(0, 1, 2))
    return h ** 3 * v[: shape[0], : shape[1], : shape[2]]


def poisson_direct(rho, h, chunk=512):
    """Brute-force O(N^2) sum V(r) = h^3 sum_{r'} rho(r') g(r - r') (FP64).

    The definition the FFT solve must reproduce; used only on small grids.
    """
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([z.ravel(), y.ravel(), x.ravel()], axis=1).astype(np.float64)
    src = rho.ravel()
    out = np.empty(pts.shape[0])
    for s in range(0, pts.shape[0], chunk):
        p = pts[s:s + chunk]
        dist = np.sqrt(((p[:, None, :] - pts[None, :, :]) ** 2).sum(axis=2))
        with np.errstate(divide="ignore"):
            g = 1.0 / (h * dist)
        g[dist == 0] = C0 / h
        out[s:s + chunk] = g @ src
    return h ** 3 * out.reshape(rho.shape)


def potential_at(rho, h, points):
    """V(r) = h^3 sum_{r'} rho(r') g(r - r') at selected grid points only (FP64).

    ``points``: integer (z, y, x) triples inside the box.  The same sum as
    ``poisson_direct`` evaluated one target point at a time, O(N) per point, so that
    large boxes can be checked at a sample of points.
    """
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    out = np.empty(len(points))
    for k, (pz, py, px) in enumerate(points):
        dist = np.sqrt((z - pz) ** 2 + (y - py) ** 2 + (x - px) ** 2)
        with np.errstate(divide="ignore"):
            g = 1.0 / (h * dist)
        g[int(pz), int(py), int(px)] = C0 / h
        out[k] = h ** 3 * float(np.sum(g * rho))
    return out

