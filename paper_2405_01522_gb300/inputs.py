"""Seeded synthetic inputs: Gaussian-sum orbitals on a uniform real-space grid.

This module only *makes inputs*.  It holds none of the exact-exchange arithmetic, so
both the CUDA library and the CPU oracle tests can take their inputs from it.

Random numbers come from one splitmix64 stream per call (64-bit state, the output
finalizer of Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014); a uniform in [0, 1) is the top 53 bits of an output times 2^-53.

Grid: point (z, y, x) sits at r = ((x - nx/2) h, (y - ny/2) h, (z - nz/2) h); arrays
are laid out [orbital][z][y][x] with x fastest.  Orbitals are real s-type Gaussian
sums  phi(r) = sum_g c_g exp(-alpha_g |r - R_g|^2), c ~ U[-1, 1].  Centres are drawn
uniformly in a ball (rejection from the enclosing cube).  Orthonormal sets are made
by Gram-Schmidt with re-orthogonalisation (two projections per vector) in FP64 under
<f, g> = h^3 sum_r f g.
"""
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection-free scaling of a uniform."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def in_ball(self, radius: float):
        while True:
            p = [self.uniform(-radius, radius) for _ in range(3)]
            if p[0] ** 2 + p[1] ** 2 + p[2] ** 2 <= radius ** 2:
                return p


def grid_axes(shape, h):
    """1-D coordinates (z, y, x) of the box ``shape = (nz, ny, nx)``."""
    return tuple((np.arange(n, dtype=np.float64) - n / 2) * h for n in shape)


def gaussian_sum(shape, h, terms):
    """Evaluate sum_g c exp(-alpha |r - R|^2) on the grid (FP64), terms = [(c, alpha, (X, Y, Z))]."""
    az, ay, ax = grid_axes(shape, h)
    out = np.zeros(shape)
    for c, alpha, (X, Y, Z) in terms:
        fx = np.exp(-alpha * (ax - X) ** 2)
        fy = np.exp(-alpha * (ay - Y) ** 2)
        fz = c * np.exp(-alpha * (az - Z) ** 2)
        out += fz[:, None, None] * np.outer(fy, fx)[None, :, :]
    return out


def gram_schmidt(f, h, passes=2):
    """Gram-Schmidt orthonormalisation in FP64 under <f, g> = h^3 sum f g.

    Vector by vector: each new vector is projected against all previous ones
    ``passes`` times (classical Gram-Schmidt with re-orthogonalisation, as stable as
    modified Gram-Schmidt applied twice), then normalised.
    """
    f = np.array(f, dtype=np.float64, copy=True)
    k = f.shape[0]
    v = f.reshape(k, -1)
    for i in range(k):
        for _ in range(passes):
            if i:
                c = h ** 3 * (v[:i] @ v[i])
                v[i] -= c @ v[:i]
        v[i] /= np.sqrt(h ** 3 * np.dot(v[i], v[i]))
    return f


def normalise(f, h):
    f = np.array(f, dtype=np.float64, copy=True)
    for i in range(f.shape[0]):
        f[i] /= np.sqrt(h ** 3 * np.sum(f[i] * f[i]))
    return f


def round_f32(a):
    """FP64 copy of ``a`` whose values are exactly representable in FP32."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def orbitals_independent(rng, shape, h, norb, ngauss, alpha, radius):
    """Each orbital: ``ngauss`` Gaussians with their own centre, exponent, coefficient.

    Draw order per Gaussian: centre (rejection), exponent, coefficient.
    """
    out = np.empty((norb,) + tuple(shape))
    for k in range(norb):
        terms = []
        for _ in range(ngauss):
            X, Y, Z = rng.in_ball(radius)
            a = rng.uniform(*alpha)
            c = rng.uniform(-1.0, 1.0)
            terms.append((c, a, (X, Y, Z)))
        out[k] = gaussian_sum(shape, h, terms)
    return out


def orbitals_shared_centres(rng, shape, h, norb, centres, alpha):
    """Each orbital: one Gaussian on every shared centre, with its own exponent and coefficient."""
    out = np.empty((norb,) + tuple(shape))
    for k in range(norb):
        terms = []
        for (X, Y, Z) in centres:
            a = rng.uniform(*alpha)
            c = rng.uniform(-1.0, 1.0)
            terms.append((c, a, (X, Y, Z)))
        out[k] = gaussian_sum(shape, h, terms)
    return out


@dataclass
class System:
    """One synthetic system: grid, orbitals (FP64 values exactly representable in FP32)."""
    shape: tuple
    h: float
    phi: np.ndarray                      # occupied / operator-defining orbitals
    psi: np.ndarray = None               # trial functions (exchange apply)
    phi_virt: np.ndarray = None          # virtual orbitals (Casida)
    eps_occ: np.ndarray = None
    eps_virt: np.ndarray = None
    meta: dict = field(default_factory=dict)


def exchange_system(n=32, h=0.3, nocc=4, ngauss=3, alpha=(0.5, 2.0), radius=2.0,
                    npsi=0, seed=0, shape=None):
    """Gram-Schmidt-orthonormalised sums of ``ngauss`` s-Gaussians (independent centres).

    Default: 32^3 box, h = 0.3 bohr, 4 orbitals of 3 Gaussians, exponents U[0.5, 2],
    centres within 2 bohr of the box centre, seed 0.  ``npsi`` extra trial functions
    (normalised, not orthogonalised) are drawn after the orbitals from the same stream.
    """
    shape = tuple(shape) if shape is not None else (n, n, n)
    rng = SplitMix64(seed)
    phi = gram_schmidt(orbitals_independent(rng, shape, h, nocc, ngauss, alpha, radius), h)
    psi = None
    if npsi:
        psi = round_f32(normalise(orbitals_independent(rng, shape, h, npsi, ngauss, alpha, radius), h))
    return System(shape=shape, h=h, phi=round_f32(phi), psi=psi,
                  meta=dict(kind="independent", ngauss=ngauss, alpha=alpha, radius=radius, seed=seed))


def batched_system(n=96, h=0.2, nocc=16, ncentres=12, alpha=(0.3, 3.0), radius=3.0,
                   npsi=32, seed=0, shape=None):
    """Occupied set of ``nocc`` orbitals over ``ncentres`` shared random centres.

    Default: 96^3 box at 0.2 bohr, 16 orbitals on 12 centres within 3 bohr of the box
    centre, every (orbital, centre) term with its own exponent U[0.3, 3] and coefficient
    U[-1, 1]; orthonormalised.  Then ``npsi`` trial functions on the same centres with
    fresh exponents and coefficients (normalised, not orthogonalised).
    """
    shape = tuple(shape) if shape is not None else (n, n, n)
    rng = SplitMix64(seed)
    centres = [rng.in_ball(radius) for _ in range(ncentres)]
    phi = gram_schmidt(orbitals_shared_centres(rng, shape, h, nocc, centres, alpha), h)
    psi = None
    if npsi:
        psi = round_f32(normalise(orbitals_shared_centres(rng, shape, h, npsi, centres, alpha), h))
    return System(shape=shape, h=h, phi=round_f32(phi), psi=psi,
                  meta=dict(kind="shared", ncentres=ncentres, alpha=alpha, radius=radius, seed=seed))


def casida_system(n=80, h=0.25, nocc=8, nvirt=64, ngauss=3, alpha=(0.3, 3.0), radius=3.0,
                  eps_occ=(-0.8, -0.3), eps_virt=(-0.1, 0.5), seed=0, shape=None):
    """Occupied + virtual orthonormal set for the Tamm-Dancoff matrix.

    Default: 80^3 box at 0.25 bohr, 8 + 64 orbitals, each a sum of 3 Gaussians with
    own centre (within 3 bohr), exponent U[0.3, 3] and coefficient; the 72 are
    orthonormalised together (occupied first).  Eigenvalues eps_occ ~ U[-0.8, -0.3],
    eps_virt ~ U[-0.1, 0.5] Ha, each set sorted ascending, drawn after the orbitals.
    """
    shape = tuple(shape) if shape is not None else (n, n, n)
    rng = SplitMix64(seed)
    allorb = gram_schmidt(orbitals_independent(rng, shape, h, nocc + nvirt, ngauss, alpha, radius), h)
    eo = np.sort([rng.uniform(*eps_occ) for _ in range(nocc)])
    ev = np.sort([rng.uniform(*eps_virt) for _ in range(nvirt)])
    allorb = round_f32(allorb)
    return System(shape=shape, h=h, phi=allorb[:nocc], phi_virt=allorb[nocc:],
                  eps_occ=np.asarray(eo), eps_virt=np.asarray(ev),
                  meta=dict(kind="casida", ngauss=ngauss, alpha=alpha, radius=radius, seed=seed))


def uneven_batch(nmol=64, edges=(48, 64, 80, 96, 112), h=0.2, nocc_range=(2, 24),
                 ncentres=12, alpha=(0.3, 3.0), radius=3.0, seed=0):
    """Descriptors of ``nmol`` independent molecules: edge from ``edges``, N_occ ~ U{2..24}.

    Returns a list of (edge, nocc, seed_k); the orbitals of molecule k come from
    ``batched_system(edge, h, nocc, ncentres, alpha, radius, npsi=0, seed=seed_k)``.
    """
    rng = SplitMix64(seed)
    out = []
    for k in range(nmol):
        e = edges[rng.integer(0, len(edges) - 1)]
        no = rng.integer(*nocc_range)
        out.append((e, no, (seed * 1000003 + k + 1) & _MASK))
    return out


def model_potential(n=96, h=0.2, natoms=4, Z=4.0, rc=0.6, radius=2.5, seed=0):
    """Smooth attractive potential of ``natoms`` pseudo-nuclei (input for the eigensolver):
    V(r) = - sum_A Z erf(|r - R_A| / rc) / |r - R_A|, centres uniform in a ball of
    ``radius`` bohr (seeded splitmix64), value -2 Z / (sqrt(pi) rc) at a centre."""
    from scipy.special import erf
    rng = SplitMix64(seed)
    az, ay, ax = grid_axes((n, n, n), h)
    V = np.zeros((n, n, n))
    for _ in range(natoms):
        X, Y, Zc = rng.in_ball(radius)
        d = np.sqrt((az[:, None, None] - Zc) ** 2 + (ay[None, :, None] - Y) ** 2 + (ax[None, None, :] - X) ** 2)
        with np.errstate(invalid="ignore", divide="ignore"):
            v = np.where(d > 1e-12, erf(d / rc) / np.where(d > 1e-12, d, 1.0), 2.0 / (np.sqrt(np.pi) * rc))
        V -= Z * v
    return V.astype(np.float32).astype(np.float64)


def starting_orbitals(n=96, h=0.2, nband=16, radius=2.5, seed=0):
    """Linearly independent Gaussian-sum starting guesses (3 Gaussians each, exponents
    U[0.3, 1.5]), normalised, not orthogonalised."""
    rng = SplitMix64(seed)
    f = orbitals_independent(rng, (n, n, n), h, nband, 3, (0.3, 1.5), radius)
    return round_f32(normalise(f, h))
