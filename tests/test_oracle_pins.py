"""Pins of the FP64 CPU oracle against closed forms, brute force and invariants.

Nothing here calls the CUDA library.  Each test is chosen so that a plausible slip in
the oracle (a dropped h^3, a wrong sign, a transposed operand, a wrong transition
index) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

import oracle
from paper_2405_01522_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "constants.json")))


def rng_fields(shape, k, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((k,) + tuple(shape))


# ---------------------------------------------------------------- kernel and Poisson


def test_c0_equals_cube_integral():
    v, _ = integrate.tplquad(lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z),
                             0, 0.5, 0, 0.5, 0, 0.5, epsabs=1e-12, epsrel=1e-12)
    assert abs(8 * v - oracle.C0) < 1e-9
    assert abs(oracle.C0 - GOLDEN["C0_cube_integral"]["value"]) < 1e-15


@pytest.mark.parametrize("shape", [(16, 16, 16), (6, 10, 8), (5, 7, 3)])
def test_poisson_fft_equals_direct_sum(shape):
    """2x padding makes the periodic FFT convolution the exact aperiodic sum (Sec. 3.1)."""
    rho = rng_fields(shape, 1, 1)[0]
    h = 0.37
    vf = oracle.poisson_fft(rho, h)
    vd = oracle.poisson_direct(rho, h)
    assert np.max(np.abs(vf - vd)) <= 1e-12 * np.max(np.abs(vd))


def test_kernel_spectrum_real_even_positive():
    g = oracle.kernel_samples((24, 20, 16), 0.3)
    full = np.fft.fftn(g)
    assert np.max(np.abs(full.imag)) < 1e-10 * np.max(np.abs(full.real))
    assert full.real.min() > 0.0
    half = oracle.kernel_spectrum((24, 20, 16), 0.3)
    assert np.allclose(half, full.real[:, :, :9])


def gaussian_case(h, L=12.0):
    n = int(round(L / h))
    n += n % 2
    z, y, x = inputs.grid_axes((n, n, n), h)
    r2 = z[:, None, None] ** 2 + y[None, :, None] ** 2 + x[None, None, :] ** 2
    rho = np.exp(-r2) / math.pi ** 1.5
    return n, rho, np.sqrt(r2)


def test_gaussian_density_erf_potential_converges():
    """Normalised Gaussian: V -> erf(r)/r, E_H -> 1/sqrt(2 pi), error O(h^2)."""
    errs = []
    hs = (0.4, 0.3, 0.2)
    for h in hs:
        n, rho, r = gaussian_case(h)
        v = oracle.poisson_fft(rho, h)
        exact = np.where(r > 0, erf(r) / np.where(r > 0, r, 1.0), 2 / math.sqrt(math.pi))
        assert np.max(np.abs(v - exact)) < 0.1 * h ** 2
        eh = 0.5 * h ** 3 * np.sum(rho * v)
        err = abs(eh - GOLDEN["gaussian_hartree_alpha1"]["value"])
        assert err < 0.015 * h ** 2
        errs.append(err)
    for (h1, e1), (h2, e2) in zip(zip(hs, errs), zip(hs[1:], errs[1:])):
        order = math.log(e1 / e2) / math.log(h1 / h2)
        assert 1.7 < order < 2.4, order
    # the centre value approaches 2/sqrt(pi)
    n, rho, r = gaussian_case(0.2)
    v = oracle.poisson_fft(rho, 0.2)
    assert abs(v[n // 2, n // 2, n // 2] - GOLDEN["gaussian_potential_origin_alpha1"]["value"]) < 5e-3


# ---------------------------------------------------------------- exchange (Eq. 2)


def test_point_sampled_potential_and_exchange_match_the_full_sums():
    """The point-by-point forms used on large boxes equal the full direct sum (Poisson)
    and the brute-force exchange loops at the same points, on ragged small boxes."""
    shape, h = (5, 7, 6), 0.4
    rho = rng_fields(shape, 1, 31)[0]
    pts = [(0, 0, 0), (4, 6, 5), (2, 3, 1), (1, 5, 4)]
    full = oracle.poisson_direct(rho, h)
    assert np.allclose(oracle.potential_at(rho, h, pts), [full[p] for p in pts], rtol=0, atol=1e-12)
    phi = rng_fields((4, 4, 3), 2, 32)
    psi = rng_fields((4, 4, 3), 1, 33)
    ref = oracle.exchange_apply_bruteforce(phi, psi, 0.5)[0]
    pts = [(0, 0, 0), (3, 3, 2), (1, 2, 0)]
    assert np.allclose(oracle.exchange_apply_at(phi, psi[0], 0.5, pts), [ref[p] for p in pts], rtol=0, atol=1e-12)


def test_exchange_matches_bruteforce_loops():
    phi = rng_fields((3, 4, 3), 2, 2)
    psi = rng_fields((3, 4, 3), 3, 3)
    h = 0.5
    a = oracle.exchange_apply(phi, psi, h)
    b = oracle.exchange_apply_bruteforce(phi, psi, h)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_one_orbital_exchange_is_minus_hartree():
    s = inputs.exchange_system(n=16, h=0.4, nocc=1)
    ex = oracle.exchange_energy(s.phi, s.h)
    eh = oracle.hartree_energy(s.phi[0] ** 2, s.h)
    assert ex < 0 and eh > 0
    assert abs(ex + eh) <= 1e-12 * eh


def test_exchange_symmetric_and_negative_definite():
    s = inputs.exchange_system(n=16, h=0.4, nocc=3, npsi=4)
    f = np.concatenate([s.phi, s.psi])
    vf = oracle.exchange_apply(s.phi, f, s.h)
    X = s.h ** 3 * f.reshape(len(f), -1) @ vf.reshape(len(f), -1).T
    assert np.max(np.abs(X - X.T)) <= 1e-12 * np.max(np.abs(X))
    assert np.linalg.eigvalsh(0.5 * (X + X.T)).max() < 0


def test_exchange_linear_in_psi_and_quadratic_in_phi():
    s = inputs.exchange_system(n=12, h=0.5, nocc=2, npsi=2)
    a = oracle.exchange_apply(s.phi, s.psi, s.h)
    comb = oracle.exchange_apply(s.phi, (2.0 * s.psi[0] - 3.0 * s.psi[1])[None], s.h)[0]
    assert np.allclose(comb, 2.0 * a[0] - 3.0 * a[1], rtol=0, atol=1e-12 * np.abs(a).max())
    scaled = oracle.exchange_apply(2.0 * s.phi, s.psi, s.h)
    assert np.allclose(scaled, 4.0 * a, rtol=0, atol=1e-12 * np.abs(a).max())


# ---------------------------------------------------------------- ACE (Eqs. 11-13)


def test_ace_reproduces_exchange_on_its_orbitals():
    s = inputs.exchange_system(n=16, h=0.4, nocc=4, npsi=3)
    zeta, W, M, L = oracle.ace_build(s.phi, s.h, return_all=True)
    assert np.allclose(L @ L.T, -M, atol=1e-13 * np.abs(M).max())
    vace = oracle.ace_apply(zeta, s.phi, s.h)
    assert np.max(np.abs(vace - W)) <= 1e-11 * np.max(np.abs(W))
    # rank k: zeta spans span(W)
    k = s.phi.shape[0]
    assert np.linalg.matrix_rank(zeta.reshape(k, -1), tol=1e-8 * np.abs(zeta).max()) == k


def test_ace_bounds_exchange_from_above():
    """With Vx negative definite, V^ACE - Vx is positive semi-definite."""
    s = inputs.exchange_system(n=16, h=0.4, nocc=3, npsi=5)
    zeta = oracle.ace_build(s.phi, s.h)
    vx = oracle.exchange_apply(s.phi, s.psi, s.h)
    va = oracle.ace_apply(zeta, s.psi, s.h)
    for p in range(s.psi.shape[0]):
        ex = oracle.inner(s.psi[p], vx[p], s.h)
        ea = oracle.inner(s.psi[p], va[p], s.h)
        assert ea >= ex - 1e-12 * abs(ex)
        assert ea < 0


# ---------------------------------------------------------------- Casida (Eq. 7)


def test_casida_K_matches_bruteforce_double_sum():
    rng = np.random.default_rng(5)
    po = rng.standard_normal((2, 3, 4, 3))
    pv = rng.standard_normal((3, 3, 4, 3))
    h = 0.45
    a = oracle.casida_K(po, pv, h)
    b = oracle.casida_K_bruteforce(po, pv, h)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_casida_K_symmetric_psd_and_Kd_symmetric():
    s = inputs.casida_system(n=12, h=0.5, nocc=2, nvirt=3)
    K = oracle.casida_K(s.phi, s.phi_virt, s.h)
    Kd = oracle.casida_Kd(s.phi, s.phi_virt, s.h)
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > -1e-12 * np.abs(K).max()
    assert np.max(np.abs(Kd - Kd.T)) <= 1e-13 * np.abs(Kd).max()
    # transition index t = i * nv + a: (ia|ia) is the self energy of rho_ia
    nv = s.phi_virt.shape[0]
    for i in range(2):
        for a in range(nv):
            e = 2 * oracle.hartree_energy(s.phi[i] * s.phi_virt[a], s.h)
            assert abs(K[i * nv + a, i * nv + a] - e) <= 1e-12 * abs(e)
    # K_d[ia, jb] = (ab|ji): the diagonal is <phi_a^2, V[phi_i^2]>
    for i in range(2):
        for a in range(nv):
            v = oracle.poisson_fft(s.phi[i] ** 2, s.h)
            e = oracle.inner(s.phi_virt[a] ** 2, v, s.h)
            assert abs(Kd[i * nv + a, i * nv + a] - e) <= 1e-12 * abs(e)


def test_casida_independent_particle_limit():
    s = inputs.casida_system(n=8, h=0.6, nocc=3, nvirt=4)
    nt = 12
    A = oracle.tda_matrix(s.eps_occ, s.eps_virt, np.zeros((nt, nt)), None, delta_M=2.0)
    w, _ = oracle.tda_solve(A, nt)
    ipa = np.sort((s.eps_virt[None, :] - s.eps_occ[:, None]).ravel())
    assert np.allclose(w, ipa, atol=1e-14)


def test_casida_one_transition_closed_form():
    s = inputs.casida_system(n=10, h=0.5, nocc=1, nvirt=1)
    K = oracle.casida_K(s.phi, s.phi_virt, s.h)
    Kd = oracle.casida_Kd(s.phi, s.phi_virt, s.h)
    for dm in (2.0, 0.0, 1.0):
        A = oracle.tda_matrix(s.eps_occ, s.eps_virt, K, Kd, delta_M=dm)
        w, x = oracle.tda_solve(A, 1)
        exact = s.eps_virt[0] - s.eps_occ[0] + dm * K[0, 0] - Kd[0, 0]
        assert abs(w[0] - exact) < 1e-14
        assert abs(abs(x[0, 0]) - 1) < 1e-14


def test_tda_solve_eigenpairs():
    s = inputs.casida_system(n=10, h=0.5, nocc=2, nvirt=3)
    K = oracle.casida_K(s.phi, s.phi_virt, s.h)
    A = oracle.tda_matrix(s.eps_occ, s.eps_virt, K, None, delta_M=1.0)
    w, X = oracle.tda_solve(A, 4)
    assert np.all(np.diff(w) >= 0)
    for k in range(4):
        assert np.linalg.norm(A @ X[k] - w[k] * X[k]) < 1e-12
    assert np.allclose(X @ X.T, np.eye(4), atol=1e-12)


# ---------------------------------------------------------------- shared input generator


def test_splitmix64_published_outputs():
    r = inputs.SplitMix64(0)
    got = [hex(r.next_u64()), hex(r.next_u64())]
    assert got == GOLDEN["splitmix64_seed0_first_outputs"]["value"]


def test_orbitals_orthonormal():
    s = inputs.exchange_system(n=16, h=0.4, nocc=4)
    f = s.phi.reshape(4, -1)
    S = s.h ** 3 * f @ f.T
    assert np.allclose(S, np.eye(4), atol=1e-6)


# ---------------------------------------------------------------- eigensolver and network pieces

from oracle import eigensolver as oe  # noqa: E402


def test_fd4_laplacian_exact_on_quartics_in_the_interior():
    n, h = 14, 0.3
    z, y, x = np.meshgrid(*(np.arange(n) * h for _ in range(3)), indexing="ij")
    f = x ** 4 - 2 * y ** 3 * z + 3 * z ** 2
    lap = oe.laplacian_fd4(f, h)
    exact = 12 * x ** 2 - 12 * y * z + 6
    sl = (slice(2, -2),) * 3
    assert np.max(np.abs(lap[sl] - exact[sl])) < 1e-8 * np.max(np.abs(exact))


def test_free_hamiltonian_is_a_kronecker_sum():
    n, h = 6, 0.4
    H = oe.hamiltonian_dense(np.zeros((n, n, n)), h)
    assert np.allclose(H, H.T)
    e1 = np.zeros(n)
    T1 = np.zeros((n, n))
    for j in range(n):
        e1[:] = 0
        e1[j] = 1
        g = np.pad(e1, 2)
        T1[:, j] = -0.5 * (-g[0:n] + 16 * g[1:n + 1] - 30 * g[2:n + 2] + 16 * g[3:n + 3] - g[4:n + 4]) / (12 * h * h)
    l1 = np.linalg.eigvalsh(T1)
    kron = np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(H), kron, atol=1e-10)


def test_ke_preconditioner_converges_to_the_shifted_inverse():
    n, h, T = 6, 0.4, 0.7
    r = np.random.default_rng(3).standard_normal((n, n, n))
    A = oe.hamiltonian_dense(np.zeros((n, n, n)), h) + T * np.eye(n ** 3)
    exact = np.linalg.solve(A, r.ravel()).reshape(r.shape)
    e3 = np.abs(oe.ke_precondition(r, T, h, sweeps=3) - exact).max()
    e300 = np.abs(oe.ke_precondition(r, T, h, sweeps=300) - exact).max()
    assert e300 < 1e-8 * np.abs(exact).max() and e300 < e3


def test_rayleigh_ritz_recovers_exact_eigenpairs():
    n, h = 6, 0.5
    v = -1.0 / (1.0 + np.sum((np.indices((n, n, n)) - 2.5) ** 2, axis=0))
    H = oe.hamiltonian_dense(v, h)
    w, U = np.linalg.eigh(H)
    rng = np.random.default_rng(0)
    B = np.concatenate([U[:, :3].T, rng.standard_normal((3, n ** 3))])    # exact lowest 3 + noise
    HB = np.stack([oe.hamiltonian_apply(b.reshape(n, n, n), v, h).ravel() for b in B])
    th, Q = oe.rayleigh_ritz(B, HB, 3, h)
    assert np.allclose(th, w[:3], atol=1e-10)


def test_conv3d_single_channel_is_a_correlation():
    from scipy import ndimage
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 7, 6, 5))
    w = rng.standard_normal((1, 1, 3, 3, 3))
    out = oe.conv3d(x, w, np.array([0.25]))
    ref = ndimage.correlate(x[0], w[0, 0], mode="constant", cval=0.0) + 0.25
    assert np.allclose(out[0], ref, atol=1e-12)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = [(0.3 * rng.standard_normal((16, 2, 3, 3, 3)), 0.1 * rng.standard_normal(16)),
              (0.1 * rng.standard_normal((16, 16, 3, 3, 3)), 0.1 * rng.standard_normal(16)),
              (0.1 * rng.standard_normal((1, 16, 3, 3, 3)), 0.1 * rng.standard_normal(1))]
    x = rng.standard_normal((2, 6, 5, 5))
    t = rng.standard_normal((6, 5, 5))
    loss, grads = oe.net_loss_and_grads(x, t, params)
    for li, (name, idx) in enumerate([("w", (3, 1, 0, 2, 1)), ("b", (5,)), ("w", (7, 11, 1, 1, 0)),
                                      ("b", (2,)), ("w", (0, 9, 2, 0, 1)), ("b", (0,))]):
        layer = li // 2
        which = 0 if name == "w" else 1
        eps = 1e-6
        p_plus = [list(p) for p in params]
        arr = p_plus[layer][which].copy()
        arr[idx] += eps
        p_plus[layer][which] = arr
        lp, _ = oe.net_loss_and_grads(x, t, [tuple(p) for p in p_plus])
        arr2 = arr.copy()
        arr2[idx] -= 2 * eps
        p_plus[layer][which] = arr2
        lm, _ = oe.net_loss_and_grads(x, t, [tuple(p) for p in p_plus])
        fd = (lp - lm) / (2 * eps)
        an = grads[layer][which][idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, layer, fd, an)


# ---------------------------------------------------------------- spectra and full TDHF

import oracle.spectra as osp  # noqa: E402


def test_oscillator_sum_rule_in_the_complete_basis():
    """Thomas-Reiche-Kuhn identity on a tiny grid: with every eigenvector of a dense
    Hamiltonian as the virtual space and independent-particle excitations (K = 0, X = 1),
    sum_k f_k = (2/3) * 1/2 * sum_i sum_d <i|[r_d, [H, r_d]]|i> exactly (Eqs. 8-9)."""
    import oracle.eigensolver as oe
    n, h, no = 6, 0.4, 3
    rng = np.random.default_rng(3)
    v = -1.0 + 0.3 * rng.standard_normal((n, n, n))
    H = oe.hamiltonian_dense(v, h)
    w, U = np.linalg.eigh(0.5 * (H + H.T))
    phi = (U.T / h ** 1.5).reshape(n ** 3, n, n, n)          # h^3 sum phi^2 = 1
    occ, virt = phi[:no], phi[no:]
    dip = osp.dipole_matrix(occ, virt, h)
    de = (w[no:][None, :] - w[:no][:, None]).ravel()
    f = osp.oscillator_strengths(de, np.eye(de.size), dip)
    rhs = 0.0
    for R in osp.positions((n, n, n), h):
        Rm = np.diag(R.ravel())
        C = Rm @ (H @ Rm - Rm @ H) - (H @ Rm - Rm @ H) @ Rm    # [r, [H, r]]
        rhs += sum(U[:, i] @ C @ U[:, i] for i in range(no))
    assert abs(f.sum() - (2.0 / 3.0) * 0.5 * rhs) < 1e-10 * abs(rhs)
    # the position matrix elements themselves: x_ia against the dense operator
    X = np.diag(osp.positions((n, n, n), h)[0].ravel())
    assert abs(dip[0, 1 * (n ** 3 - no) + 4] - U[:, 1] @ X @ U[:, no + 4]) < 1e-12


def test_dipoles_follow_the_axis_order_and_transition_index():
    """<i|r|a> with an even occupied Gaussian and odd virtuals around the grid's centre of
    symmetry c = -h/2: (Z - c) g has a dipole with g only along z, (X - c) g only along x
    (x is the fastest grid axis), and t = i n_v + a."""
    n, h = 16, 0.3
    X, Y, Z = osp.positions((n, n, n), h)
    c = -h / 2
    g0 = np.exp(-((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2))
    dip = osp.dipole_matrix(g0[None], np.stack([(Z - c) * g0, (X - c) * g0]), h)
    ref = h ** 3 * np.sum((X - c) ** 2 * g0 * g0)
    assert abs(dip[0, 0]) < 1e-13 and abs(dip[1, 0]) < 1e-13 and abs(dip[2, 0] - ref) < 1e-13
    assert abs(dip[1, 1]) < 1e-13 and abs(dip[2, 1]) < 1e-13 and abs(dip[0, 1] - ref) < 1e-13
    assert ref > 1e-2


def test_strength_function_lorentzian_closed_forms():
    omega, f, gamma = np.array([0.3, 0.7]), np.array([0.2, 0.5]), 0.01
    # at an isolated peak S = f / (pi gamma) + the other line's tail
    s = osp.strength_function([0.3], omega, f, gamma)[0]
    tail = 0.5 * gamma / (np.pi * (0.4 ** 2 + gamma ** 2))
    assert abs(s - (0.2 / (np.pi * gamma) + tail)) < 1e-12
    # integral over [-W, W] around each line: sum f_k (2/pi) atan(W/gamma)
    W = 0.15
    grid = np.linspace(0.3 - W, 0.3 + W, 200001)
    one = osp.strength_function(grid, omega[:1], f[:1], gamma)
    assert abs(integrate.trapezoid(one, grid) - 0.2 * (2 / np.pi) * np.arctan(W / gamma)) < 1e-8


def _tdhf_case(no=2, nv=3, seed=5):
    """A small K from the FFT oracle on orthonormal orbitals, and eigenvalue gaps."""
    shape, h = (8, 8, 8), 0.4
    rng = inputs.SplitMix64(seed)
    phi = inputs.orbitals_independent(rng, shape, h, no + nv, 2, (0.4, 1.2), 1.0)
    phi = inputs.gram_schmidt(phi, h)
    K = oracle.casida_K(phi[:no], phi[no:], h)
    Kd = oracle.casida_Kd(phi[:no], phi[no:], h)
    eo = np.array([-2.0, -1.6])[:no]
    ev = np.array([0.5, 0.75, 1.0])[:nv]
    return eo, ev, K, Kd, phi


def test_full_tdhf_half_size_form_equals_the_non_hermitian_problem():
    """Eq. 3 solved directly (2n x 2n, numpy eig) and through the half-size symmetric
    form agree: excitation energies and X + Y (up to sign)."""
    eo, ev, K, Kd, _ = _tdhf_case()
    for dm in (2.0, 0.0):
        A, B = osp.tdhf_matrices(eo, ev, K, Kd, dm)
        w, XpY = osp.tdhf_solve(A, B, 6)
        w2, XpY2 = osp.tdhf_solve_nonhermitian(A, B)
        assert np.allclose(w, w2, rtol=0, atol=1e-12)
        for k in range(6):
            s = np.sign(XpY[k] @ XpY2[k])
            assert np.allclose(XpY[k], s * XpY2[k], atol=1e-10)


def test_full_tdhf_reduces_to_tda_and_closed_forms():
    eo, ev, K, Kd, _ = _tdhf_case()
    A, B = osp.tdhf_matrices(eo, ev, K, Kd, 2.0)
    # B = 0: the Tamm-Dancoff eigenvalues
    w0, _ = osp.tdhf_solve(A, np.zeros_like(B), 6)
    assert np.allclose(w0, np.linalg.eigvalsh(A), atol=1e-12)
    # full TDHF lies below the TDA for the lowest root (A - B, A + B positive definite)
    w, _ = osp.tdhf_solve(A, B, 1)
    assert w[0] <= np.linalg.eigvalsh(A)[0] + 1e-14
    # B uses the exchange-permuted K: B[ia, jb] = 2 K[ia, jb] - K[ib, ja]
    nv = ev.size
    assert abs(B[0 * nv + 1, 1 * nv + 2] - (2 * K[0 * nv + 1, 1 * nv + 2] - K[0 * nv + 2, 1 * nv + 1])) < 1e-15
    # one transition: omega = sqrt((a - b)(a + b)), b = delta_M K - K (i = j, a = b)
    A1, B1 = osp.tdhf_matrices(eo[:1], ev[:1], K[:1, :1], Kd[:1, :1], 2.0)
    a, b = A1[0, 0], B1[0, 0]
    assert abs(b - K[0, 0]) < 1e-15
    assert abs(osp.tdhf_solve(A1, B1, 1)[0][0] - math.sqrt((a - b) * (a + b))) < 1e-14


def _spin_orbital_tdhf_roots(eo, ev, phi_occ, phi_virt, h):
    """Positive roots of Eq. 3 built in spin orbitals from Eqs. 4-5, closed shell.

    Every two-electron integral (pq|rs) = <phi_p phi_q, V[phi_r phi_s]> is its own direct
    Coulomb sum (no FFT, no K matrix reused); a spin-orbital integral vanishes unless p, q
    share a spin and r, s share a spin.  Transitions: alpha (i, a) first, then beta.
    A_{ia,jb} = delta (eps_a - eps_i) + (ai|jb) - (ab|ji),  B_{ia,jb} = (ai|bj) - (aj|bi).
    """
    no, nv = len(eo), len(ev)
    orb = list(phi_occ) + list(phi_virt)           # spatial orbitals: occupied, then virtual
    n = no + nv
    pot = {}

    def V(r, s_):
        key = (min(r, s_), max(r, s_))
        if key not in pot:
            pot[key] = oracle.poisson_direct(orb[r] * orb[s_], h)
        return pot[key]

    def eri(p, q, r, s_):
        return h ** 3 * float(np.sum(orb[p] * orb[q] * V(r, s_)))

    trans = [(sp, i, no + a) for sp in (0, 1) for i in range(no) for a in range(nv)]
    m = len(trans)
    A, B = np.zeros((m, m)), np.zeros((m, m))
    for u, (s1, i, a) in enumerate(trans):
        for w, (s2, j, b) in enumerate(trans):
            same = s1 == s2
            A[u, w] = (eri(a, i, j, b)                                   # (ai|jb): any spins
                       - (eri(a, b, j, i) if same else 0.0))             # (ab|ji): one spin
            if u == w:
                A[u, w] += ev[a - no] - eo[i]
            B[u, w] = eri(a, i, b, j) - (eri(a, j, b, i) if same else 0.0)
    big = np.block([[A, B], [-B, -A]])
    w = np.sort(np.linalg.eigvals(big).real)
    return w[m:]


def test_rhf_b_matrix_from_the_spin_orbital_equations():
    """Eqs. 4-5 in spin orbitals for a closed shell (alpha = beta) split into the singlet
    and triplet RHF problems, so the full-TDHF roots of the spin-orbital matrices (every
    integral a direct sum) are the union of the oracle's half-size roots at delta_M = 2 and
    delta_M = 0.  A B with the exchange-type index of the wrong kind must fail."""
    shape, h = (6, 6, 6), 0.45
    rng = inputs.SplitMix64(9)
    phi = inputs.gram_schmidt(inputs.orbitals_independent(rng, shape, h, 5, 2, (0.4, 1.2), 0.9), h)
    po, pv = phi[:2], phi[2:]
    eo, ev = np.array([-1.1, -0.8]), np.array([0.3, 0.45, 0.7])
    ref = _spin_orbital_tdhf_roots(eo, ev, po, pv, h)
    K = oracle.casida_K(po, pv, h)
    Kd = oracle.casida_Kd(po, pv, h)

    def union(Bfun):
        roots = []
        for dm in (2.0, 0.0):
            A, _ = osp.tdhf_matrices(eo, ev, K, Kd, dm)
            roots.append(osp.tdhf_solve(A, Bfun(dm), A.shape[0])[0])
        return np.sort(np.concatenate(roots))

    got = union(lambda dm: osp.tdhf_matrices(eo, ev, K, Kd, dm)[1])
    assert np.allclose(got, ref, rtol=0, atol=1e-10), np.abs(got - ref).max()
    # planted mistakes: exchange-type term taken unpermuted, or as the Coulomb term K_d
    scale = np.abs(ref).max()
    with np.errstate(invalid="ignore"):        # a wrong B can make omega^2 < 0 (NaN roots)
        for wrong in (lambda dm: dm * K - K, lambda dm: dm * K - Kd, lambda dm: dm * K - K.T[::-1, ::-1]):
            assert not np.allclose(union(wrong), ref, rtol=0, atol=1e-6 * scale)


# ---------------------------------------------------------------- SCF (closed-shell HF)

import oracle.scf as oscf  # noqa: E402


def _scf_potential():
    return inputs.model_potential(n=8, h=0.5, natoms=2, Z=2.0, rc=0.8, radius=0.8, seed=3)


def test_coulomb_matrix_is_the_poisson_solve():
    """G rho equals the FFT Poisson solve of the same density (and its direct sum)."""
    rho = rng_fields((5, 6, 4), 1, 7)[0]
    G = oscf.coulomb_matrix(rho.shape, 0.4)
    assert np.allclose((G @ rho.ravel()).reshape(rho.shape), oracle.poisson_fft(rho, 0.4), rtol=0, atol=1e-11)


def test_scf_with_ace_converges_to_the_exact_exchange_result():
    """Sec. 3.1: at self-consistency ACE is not an approximation, so the ACE cycle and the
    exact-exchange cycle reach the same energy and orbital energies."""
    v = _scf_potential()
    a = oscf.scf(v, 0.5, 2, mode="ace", tol=1e-11)
    b = oscf.scf(v, 0.5, 2, mode="exact", tol=1e-11)
    assert a["reldens"] < 1e-11 and b["reldens"] < 1e-11
    assert abs(a["energy"] - b["energy"]) < 1e-9 * abs(b["energy"])
    assert np.allclose(a["eps_orb"], b["eps_orb"], rtol=0, atol=1e-8)
    assert b["exchange"] < 0 < b["hartree"]


def test_scf_one_orbital_exchange_is_minus_half_hartree():
    """Two electrons in one orbital: E_x = -(phi phi|phi phi) and E_H = 2 (phi phi|phi phi),
    whatever the orbital (the closed-shell density and exchange factors)."""
    r = oscf.scf(_scf_potential(), 0.5, 1, mode="exact", tol=1e-10)
    assert abs(r["exchange"] + 0.5 * r["hartree"]) < 1e-12 * r["hartree"]
    phi = rng_fields((8, 8, 8), 1, 4)
    phi /= np.sqrt(0.5 ** 3 * np.sum(phi ** 2))
    _, _, eh, ex = oscf.hf_energy(phi, _scf_potential(), 0.5, oscf.coulomb_matrix((8, 8, 8), 0.5))
    assert abs(ex + 0.5 * eh) < 1e-12 * eh


def test_scf_fixed_point_solves_the_hf_equations_and_minimises_the_energy():
    """The converged orbitals satisfy F[phi] phi_i = eps_i phi_i with the exact exchange,
    and the HF energy rises quadratically when an orbital is rotated out of the
    occupied space (first variation zero, second positive)."""
    v, h = _scf_potential(), 0.5
    r = oscf.scf(v, h, 2, mode="exact", tol=1e-12)
    phi = r["phi"]
    G = oscf.coulomb_matrix(v.shape, h)
    F = oracle.eigensolver.hamiltonian_dense(v, h) + np.diag(G @ oscf.density(phi).ravel()) + \
        oscf.exchange_matrix(phi, G)
    P = phi.reshape(2, -1)
    for i in range(2):
        res = F @ P[i] - r["eps_orb"][i] * P[i]
        assert np.linalg.norm(res) < 1e-7 * np.linalg.norm(F @ P[i])
    d = rng_fields((8, 8, 8), 1, 5)[0].ravel()
    d -= P.T @ (h ** 3 * (P @ d))                   # orthogonal to the occupied space
    dE = []
    for delta in (1e-3, 5e-4):
        q = P.copy()
        q[0] = q[0] + delta * d
        q[0] /= np.sqrt(h ** 3 * q[0] @ q[0])
        dE.append(oscf.hf_energy(q.reshape(phi.shape), v, h, G)[0] - r["energy"])
    assert dE[0] > 0 and dE[1] > 0
    assert abs(dE[0] / dE[1] - 4.0) < 0.05


def test_scf_state_mixing_reaches_the_same_ground_state():
    """Sec. 3.2: mixing states instead of the density changes the path, not the fixed
    point -- same energy and orbital energies as density mixing."""
    v = _scf_potential()
    a = oscf.scf(v, 0.5, 2, mode="ace", tol=1e-11, mix="states")
    b = oscf.scf(v, 0.5, 2, mode="ace", tol=1e-11, mix="density")
    assert a["reldens"] < 1e-11
    assert abs(a["energy"] - b["energy"]) < 1e-9 * abs(b["energy"])
    assert np.allclose(a["eps_orb"], b["eps_orb"], rtol=0, atol=1e-8)


def test_state_mixing_keeps_an_orthonormal_set_and_is_rotation_blind():
    """The mixed states are orthonormal; mixing with a rotated and sign-flipped copy of the
    same output space gives the same result (only the span of the output enters)."""
    h = 0.5
    rng = np.random.default_rng(9)
    A = np.linalg.qr(rng.standard_normal((64, 3)))[0].T / h ** 1.5
    B = np.linalg.qr(rng.standard_normal((64, 3)))[0].T / h ** 1.5
    Q = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    m1 = oscf.mix_states(A, B, h, 0.4)
    m2 = oscf.mix_states(A, Q @ B, h, 0.4)
    assert np.allclose(h ** 3 * m1 @ m1.T, np.eye(3), atol=1e-12)
    assert np.allclose(m1, m2, atol=1e-12)
    assert np.allclose(oscf.mix_states(A, A, h, 0.4), A, atol=1e-12)   # fixed point


# ---------------------------------------------------------------- spin-polarised TDA (Eqs. 4-5)


def test_uhf_cross_spin_coupling_is_the_double_sum():
    """The alpha-beta block of the UHF coupling is Eq. 6 written out between an alpha
    and a beta transition density (direct double sum, no FFT)."""
    rng = np.random.default_rng(21)
    oa, va = rng.standard_normal((2, 3, 3, 4)), rng.standard_normal((2, 3, 3, 4))
    ob, vb = rng.standard_normal((1, 3, 3, 4)), rng.standard_normal((3, 3, 3, 4))
    h = 0.5
    K = oracle.uhf_K(oa, va, ob, vb, h)
    ra = oracle.transition_densities(oa, va)
    rb = oracle.transition_densities(ob, vb)
    cross = np.array([[h ** 3 * np.sum(ra[t] * oracle.poisson_direct(rb[s], h)) for s in range(3)]
                      for t in range(4)])
    assert K.shape == (7, 7)
    assert np.max(np.abs(K[:4, 4:] - cross)) <= 1e-12 * np.abs(cross).max()
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.abs(K).max()


def test_uhf_closed_shell_splits_into_singlets_and_triplets():
    """Equal alpha and beta orbitals: the spin-orbital matrix [[D + K - Kd, K], [K,
    D + K - Kd]] block-diagonalises into D + 2K - Kd (singlets, delta_M = 2 of Eq. 7) and
    D - Kd (triplets, delta_M = 0), so its spectrum is the union of the two."""
    s = inputs.casida_system(n=12, h=0.5, nocc=2, nvirt=3)
    po, pv = s.phi, s.phi_virt
    eo, ev = np.array([-0.7, -0.45]), np.array([0.05, 0.2, 0.4])
    K = oracle.uhf_K(po, pv, po, pv, s.h)
    Kd = oracle.casida_Kd(po, pv, s.h)
    w_uhf = np.linalg.eigvalsh(oracle.uhf_tda_matrix(eo, ev, eo, ev, K, Kd, Kd))
    K1 = oracle.casida_K(po, pv, s.h)
    sing = np.linalg.eigvalsh(oracle.tda_matrix(eo, ev, K1, Kd, delta_M=2.0))
    trip = np.linalg.eigvalsh(oracle.tda_matrix(eo, ev, K1, Kd, delta_M=0.0))
    assert np.allclose(w_uhf, np.sort(np.concatenate([sing, trip])), rtol=0, atol=1e-12)


def test_uhf_without_beta_transitions_is_the_spin_orbital_block():
    """No beta transitions: A is the alpha block alone, diag + (ia|jb) - (ij|ab)."""
    s = inputs.casida_system(n=12, h=0.5, nocc=1, nvirt=4)
    eo, ev = np.array([-0.5]), np.array([0.1, 0.2, 0.3, 0.6])
    K = oracle.uhf_K(s.phi, s.phi_virt, s.phi[:0], s.phi_virt[:0], s.h)
    Kd = oracle.casida_Kd(s.phi, s.phi_virt, s.h)
    A = oracle.uhf_tda_matrix(eo, ev, [], [], K, Kd)
    assert np.allclose(A, oracle.tda_matrix(eo, ev, oracle.casida_K(s.phi, s.phi_virt, s.h), Kd, delta_M=1.0),
                       rtol=0, atol=1e-13)


# ---------------------------------------------------------------- spherical domain (Sec. 3.4)


@pytest.mark.parametrize("n,h", [(12, 0.6), (16, 0.5)])
def test_sphere_levels_of_a_free_particle(n, h):
    """V = 0 inside a sphere with zero boundary values: the levels are x^2 / (2 R^2), x the
    zeros of the spherical Bessel functions (j0: pi; j1: 4.4934..., the root of tan x = x).
    On the grid the boundary sits between the last kept point (radius <= R) and the first
    dropped one (<= R + h), so E0 lies between the two radii's values; the ratio E1 / E0
    does not depend on the radius, and the p level stays threefold."""
    R = (n / 2 - 1) * h
    H, keep = oe.hamiltonian_masked(np.zeros((n, n, n)), h, oe.sphere_mask((n, n, n), h, R))
    w = np.linalg.eigvalsh(0.5 * (H + H.T))[:4]
    x11 = 4.493409457909064
    assert abs(math.tan(x11) - x11) < 1e-9
    assert math.pi ** 2 / (2 * (R + h) ** 2) < w[0] < math.pi ** 2 / (2 * R ** 2)
    assert abs(w[1] / w[0] - (x11 / math.pi) ** 2) < 0.01 * (x11 / math.pi) ** 2
    assert np.ptp(w[1:4]) < 1e-10 * w[1]


def test_sphere_restriction_raises_every_level():
    """Restricting H to a subset of the points can only raise each eigenvalue
    (Courant-Fischer), and a sphere holding the whole box restricts nothing."""
    v = inputs.model_potential(n=10, h=0.5, natoms=2, Z=2.0, rc=0.8, radius=0.8, seed=3)
    full = np.linalg.eigvalsh(oe.hamiltonian_dense(v, 0.5))[:6]
    Hm, _ = oe.hamiltonian_masked(v, 0.5, oe.sphere_mask(v.shape, 0.5, 2.0))
    part = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[:6]
    assert np.all(part >= full - 1e-12)
    Hw, keep = oe.hamiltonian_masked(v, 0.5, oe.sphere_mask(v.shape, 0.5, 100.0))
    assert keep.size == v.size and np.allclose(np.linalg.eigvalsh(0.5 * (Hw + Hw.T))[:6], full, atol=1e-12)


def test_masked_scf_stays_in_the_sphere_and_ace_is_exact_there():
    v = _scf_potential()
    m = oe.sphere_mask(v.shape, 0.5, 1.6)
    a = oscf.scf(v, 0.5, 2, mode="ace", tol=1e-11, mask=m)
    b = oscf.scf(v, 0.5, 2, mode="exact", tol=1e-11, mask=m)
    assert np.max(np.abs(a["phi"][:, m == 0])) < 1e-12
    assert abs(a["energy"] - b["energy"]) < 1e-9 * abs(b["energy"])
    free = oscf.scf(v, 0.5, 2, mode="exact", tol=1e-11)
    assert b["energy"] > free["energy"]           # a smaller domain, a higher variational energy
