"""Plain eigensolver pieces and the 3-D convolution network of the learned
preconditioner (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's eigensolvers are conjugate gradients and preconditioned Lanczos (Sec. 3.1),
on the Hamiltonian of Eq. 1; the preconditioner and the learned part are not in the
paper.  Readings (stated, not taken from the paper):

* Hamiltonian on the box with zero boundary values: H = -1/2 Lap + V, Lap the
  fourth-order central difference  (-f[i-2] + 16 f[i-1] - 30 f[i] + 16 f[i+1] - f[i+2])
  / (12 h^2) along each axis.
* Kinetic-energy preconditioner: x ~ (K + T)^{-1} r, K = -1/2 Lap, T the orbital's
  kinetic energy <psi, K psi>, by `sweeps` damped-Jacobi steps from x0 = r / d with
  weight omega: x <- x + omega (r - (K + T) x) / d, d = 3.75 / h^2 + T.
* One iteration of the block solver (Rayleigh-Ritz on [Psi, W]): S = <B, B>,
  Hs = <B, H B>, S = L L^T, C = L^-1 Hs L^-T, C y = theta y (ascending), new
  Psi = B L^-T y[:, :k].
* Spherical domain (Sec. 3.4: a sphere around the molecule, zero boundary values on its
  surface): the grid points within radius R of the box centre (the grid convention of
  the Coulomb module, point (x, y, z) at ((x - nx/2) h, ...)); H is restricted to them,
  i.e. the operator P H P with P the projector on the kept points, every orbital zero
  elsewhere.
* Convolution layer (stride 1, zero padding 1, 3^3 kernel):
  out[co, z, y, x] = b[co] + sum_{ci, dz, dy, dx} w[co, ci, dz, dy, dx] in[ci, z+dz-1, y+dy-1, x+dx-1].
  Network: conv(2 -> 16) ReLU conv(16 -> 16) ReLU conv(16 -> 1).
"""
import numpy as np


def laplacian_fd4(f, h):
    """Fourth-order finite-difference Laplacian with zero values outside the box."""
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    for ax in range(f.ndim):
        n = f.shape[ax]
        pad = [(0, 0)] * f.ndim
        pad[ax] = (2, 2)
        g = np.pad(f, pad)
        sl = lambda a, b: tuple(slice(a, b) if i == ax else slice(None) for i in range(f.ndim))
        out += (-g[sl(0, n)] + 16 * g[sl(1, n + 1)] - 30 * g[sl(2, n + 2)] + 16 * g[sl(3, n + 3)]
                - g[sl(4, n + 4)]) / (12 * h * h)
    return out


def hamiltonian_apply(psi, v, h):
    """H psi = -1/2 Lap psi + v psi."""
    return -0.5 * laplacian_fd4(psi, h) + np.asarray(v, dtype=np.float64) * psi


def hamiltonian_dense(v, h):
    """Dense matrix of H on a small box (columns = H applied to unit vectors)."""
    n = v.size
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = hamiltonian_apply(e.reshape(v.shape), v, h).ravel()
    return M


def sphere_mask(shape, h, radius):
    """1 at the grid points within `radius` of the box centre, 0 elsewhere (float array)."""
    nz, ny, nx = shape
    z = (np.arange(nz) - nz / 2) * h
    y = (np.arange(ny) - ny / 2) * h
    x = (np.arange(nx) - nx / 2) * h
    r2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
    return (r2 <= radius * radius).astype(np.float64)


def hamiltonian_masked(v, h, mask):
    """H restricted to the kept points (rows and columns of hamiltonian_dense), and the
    flat indices of those points."""
    keep = np.flatnonzero(np.asarray(mask).ravel() > 0)
    H = hamiltonian_dense(v, h)
    return H[np.ix_(keep, keep)], keep


def ke_precondition(r, T, h, sweeps=3, omega=2.0 / 3.0):
    """x ~ (K + T)^{-1} r by damped Jacobi from x0 = r / d (K = -1/2 Lap)."""
    r = np.asarray(r, dtype=np.float64)
    d = 3.75 / (h * h) + T
    x = r / d
    for _ in range(sweeps):
        ax = -0.5 * laplacian_fd4(x, h) + T * x
        x = x + omega * (r - ax) / d
    return x


def rayleigh_ritz(B, HB, k, h):
    """Lowest k Ritz pairs of H on span(B); B, HB: (m, N).  Returns (theta, Q) with
    new Psi = Q^T B, i.e. Q: (m, k)."""
    S = h ** 3 * (B @ B.T)
    Hs = h ** 3 * (B @ HB.T)
    Hs = 0.5 * (Hs + Hs.T)
    L = np.linalg.cholesky(0.5 * (S + S.T))
    Li = np.linalg.inv(L)
    C = Li @ Hs @ Li.T
    theta, Y = np.linalg.eigh(0.5 * (C + C.T))
    Q = Li.T @ Y[:, :k]
    return theta[:k], Q


def conv3d(x, w, b):
    """x: (ci, nz, ny, nx); w: (co, ci, 3, 3, 3); b: (co,).  Zero padding 1, stride 1."""
    x = np.asarray(x, dtype=np.float64)
    ci, nz, ny, nx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((w.shape[0], nz, ny, nx))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]          # (ci, ...)
                out += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx], patch)
    return out + b[:, None, None, None]


def net_forward(x, params):
    """params = [(w1, b1), (w2, b2), (w3, b3)]; returns (out, cache)."""
    (w1, b1), (w2, b2), (w3, b3) = params
    z1 = conv3d(x, w1, b1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv3d(a1, w2, b2)
    a2 = np.maximum(z2, 0.0)
    out = conv3d(a2, w3, b3)
    return out, (x, z1, a1, z2, a2)


def conv3d_backward(x, w, dout):
    """Gradients of sum(dout * conv3d(x, w, b)) w.r.t. x, w, b."""
    ci, nz, ny, nx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                dw[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", dout, patch)
                dxp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx] += np.einsum("oc,ozyx->czyx", w[:, :, dz, dy, dx], dout)
    db = dout.sum(axis=(1, 2, 3))
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, db


def net_loss_and_grads(x, target, params, mask=None):
    """Loss = mean over (masked) voxels of (net(x) - target)^2 and its parameter gradients."""
    out, (x0, z1, a1, z2, a2) = net_forward(x, params)
    diff = out[0] - target
    m = np.ones_like(diff) if mask is None else mask
    nrm = m.sum()
    loss = float((m * diff * diff).sum() / nrm)
    dout = (2.0 * m * diff / nrm)[None]
    (w1, b1), (w2, b2), (w3, b3) = params
    da2, dw3, db3 = conv3d_backward(a2, w3, dout)
    dz2 = da2 * (z2 > 0)
    da1, dw2, db2 = conv3d_backward(a1, w2, dz2)
    dz1 = da1 * (z1 > 0)
    _, dw1, db1 = conv3d_backward(x0, w1, dz1)
    return loss, [(dw1, db1), (dw2, db2), (dw3, db3)]
