"""GPU tests of the single-density Poisson solve, the exchange term of the block
eigensolver and the closed-shell HF SCF loop (Sec. 3.1-3.2) against the FP64 oracle."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import oracle.scf as oscf
from oracle.eigensolver import hamiltonian_dense
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import TOL, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scf_16cubed.json")


@pytest.mark.parametrize("shape,h,prec", [((16, 16, 16), 0.4, "fp32"), ((24, 24, 40), 0.3, "fp32"),
                                          ((16, 16, 24), 0.4, "fp64")])
def test_poisson_parity(shape, h, prec):
    need_gpu()
    rho = np.random.default_rng(11).standard_normal(shape).astype(np.float32).astype(np.float64)
    ref = oracle.poisson_fft(rho, h)
    ctx = rsx.Context(shape, h, prec)
    V = ctx.poisson(to_dev(rho, prec))
    ctx.sync()
    assert rel_max_err(V.double().cpu().numpy(), ref) < TOL[prec]


def _case():
    with open(GOLDEN) as f:
        g = json.load(f)
    c = g["case"]
    v = inputs.model_potential(n=c["n"], h=c["h"], natoms=c["natoms"], Z=c["Z"], rc=c["rc"], radius=c["radius"],
                               seed=c["seed"])
    psi0 = inputs.starting_orbitals(n=c["n"], h=c["h"], nband=c["nocc"], radius=c["radius"], seed=5)
    return g, c, v, psi0


def _run_scf(ace, iters=80, inner=2, tol=2e-6, mix="density"):
    g, c, v, psi0 = _case()
    ctx = rsx.Context((c["n"],) * 3, c["h"], "fp32")
    vd = to_dev(v, "fp32")
    scf = rsx.SCF(ctx, vd, c["nocc"], ace=ace, alpha=c["alpha"], mix=mix)
    scf.init(to_dev(psi0, "fp32"))
    hist = []
    for _ in range(iters):
        r = scf.step(inner=inner)
        hist.append(r)
        if len(hist) > 1 and 0 < r["reldens"] < tol:
            break
    return g, c, v, scf, ctx, hist


def test_eigensolver_exchange_ace_equals_exact_on_the_orbital_span():
    """Eq. 13: the ACE operator built from phi acts like Vx[phi] on span(phi), so Rayleigh-
    Ritz on the orbitals gives the same values either way -- and those of the oracle's
    dense (T + V + Vx[phi]) projected on the orbitals."""
    need_gpu()
    g, c, v, psi0 = _case()
    n, h, k = c["n"], c["h"], c["nocc"]
    H0 = hamiltonian_dense(v, h)
    w, U = np.linalg.eigh(0.5 * (H0 + H0.T))
    phi = (U[:, :k].T / h ** 1.5).reshape((k, n, n, n)).astype(np.float32).astype(np.float64)
    ctx = rsx.Context((n,) * 3, h, "fp32")
    vd, phid = to_dev(v, "fp32"), to_dev(phi, "fp32")
    xi = ctx.ace_build(phid)
    ctx.sync()
    eig = rsx.Eigensolver(vd, h, k)
    eig.init(phid)
    eig.set_exchange(xi, mode=1)
    t_ace = np.array(eig.refresh())
    eig.set_exchange(phid, mode=2, ctx=ctx)
    t_exact = np.array(eig.refresh())
    eig.set_exchange(None, mode=0)
    t_none = np.array(eig.refresh())
    G = oscf.coulomb_matrix((n,) * 3, h)
    P = phi.reshape(k, -1)
    F = H0 + oscf.exchange_matrix(phi, G)
    S = h ** 3 * P @ P.T
    A = h ** 3 * P @ (0.5 * (F + F.T)) @ P.T
    L = np.linalg.cholesky(S)
    ref = np.linalg.eigvalsh(np.linalg.solve(L, np.linalg.solve(L, A).T).T)
    assert np.max(np.abs(t_ace - ref)) < 2e-5 * np.max(np.abs(ref))
    assert np.max(np.abs(t_exact - ref)) < 2e-5 * np.max(np.abs(ref))
    assert np.all(t_ace < t_none)                 # exchange lowers the orbital energies
    eig.close()


def test_scf_energy_terms_vs_oracle():
    """The energy the SCF step reports for the orbitals entering it equals the oracle's HF
    energy of those orbitals, term by term."""
    need_gpu()
    g, c, v, scf, ctx, hist = _run_scf(True, iters=6)
    phi = scf.orbitals().double().cpu().numpy()
    r = scf.step(inner=2)
    E, one, eh, ex = oscf.hf_energy(phi, v, c["h"], oscf.coulomb_matrix(v.shape, c["h"]))
    assert abs(r["energy"] - E) < 1e-5 * abs(E)
    assert abs(r["one_body"] - one) < 1e-5 * abs(one)
    assert abs(r["hartree"] - eh) < 1e-5 * abs(eh)
    assert abs(r["exchange"] - ex) < 1e-5 * abs(ex)


@pytest.mark.parametrize("ace,mix", [(True, "density"), (False, "density"), (True, "states")])
def test_scf_converges_to_the_oracle_ground_state(ace, mix):
    """Both cycles reach the oracle's self-consistent HF energy and orbital energies
    (Sec. 3.1: with ACE the fixed point is unchanged; Sec. 3.2: nor does it depend on
    mixing the density or the states), with the density error of Eq. 15 falling to the
    FP32 level."""
    need_gpu()
    g, c, v, scf, ctx, hist = _run_scf(ace, mix=mix)
    ref = g["ace" if ace else "exact"]
    last = hist[-1]
    assert 0 < last["reldens"] < 2e-6, [h["reldens"] for h in hist]
    assert abs(last["energy"] - ref["energy"]) < 2e-5 * abs(ref["energy"])
    assert abs(last["exchange"] - ref["exchange"]) < 1e-4 * abs(ref["exchange"])
    assert abs(last["theta_sum"] - sum(ref["eps_orb"])) < 1e-4 * abs(sum(ref["eps_orb"]))
    # orbitals solve the HF equations of the oracle's Fock operator
    phi = scf.orbitals().double().cpu().numpy()
    G = oscf.coulomb_matrix(v.shape, c["h"])
    F = hamiltonian_dense(v, c["h"]) + np.diag(G @ oscf.density(phi).ravel()) + oscf.exchange_matrix(phi, G)
    P = phi.reshape(c["nocc"], -1)
    Fp = P @ F.T                                   # rows F p_i
    C = np.linalg.solve(P @ P.T, P @ Fp.T)         # projection of F p_i on span(P)
    R = Fp - C.T @ P
    assert np.linalg.norm(R) < 2e-3 * np.linalg.norm(Fp)
    scf.close()


def test_scf_invalid_arguments():
    need_gpu()
    ctx = rsx.Context((16, 16, 16), 0.5, "fp32")
    v = torch.zeros((16, 16, 16), device="cuda")
    with pytest.raises(rsx.RsxError):
        rsx.SCF(ctx, v, 0)
    with pytest.raises(rsx.RsxError):
        rsx.SCF(ctx, v, 2, alpha=1.0)
    ctx64 = rsx.Context((16, 16, 16), 0.5, "fp64")
    with pytest.raises(rsx.RsxError):
        rsx.SCF(ctx64, v, 2)
    with pytest.raises(ValueError):
        rsx.SCF(ctx, v, 2, mix="potential").init(torch.zeros((2, 16, 16, 16), device="cuda"))
