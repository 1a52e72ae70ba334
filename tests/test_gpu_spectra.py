"""GPU parity for the absorption spectrum (Eqs. 8-10) and the full TDHF problem
(Eqs. 3-5, half-size form) through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import oracle.spectra as osp
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

# dipoles: a weighted grid sum; FP32 inputs and positions rounded to single precision
TOL_DIP = {"fp32": 1e-6, "fp64": 1e-12}


def system(shape, h, no, nv, seed=0):
    return inputs.casida_system(h=h, nocc=no, nvirt=nv, shape=shape, radius=1.5, alpha=(0.5, 2.0), seed=seed)


@pytest.mark.parametrize("shape,h,no,nv,prec", [((16, 16, 16), 0.5, 2, 3, "fp32"), ((24, 24, 40), 0.4, 3, 5, "fp32"),
                                                ((24, 24, 40), 0.4, 3, 5, "fp64")])
def test_dipoles_oscillators_and_strength_function(shape, h, no, nv, prec):
    need_gpu()
    s = system(shape, h, no, nv)
    dip_ref = osp.dipole_matrix(s.phi, s.phi_virt, h)
    ctx = rsx.Context(shape, h, prec)
    dip = ctx.casida_dipoles(to_dev(s.phi, prec), to_dev(s.phi_virt, prec))
    ctx.sync()
    assert rel_max_err(dip.cpu().numpy(), dip_ref) < TOL_DIP[prec]
    # oscillator strengths and S(w) from the same FP64 eigenpairs on both sides
    K = oracle.casida_K(s.phi, s.phi_virt, h)
    A = oracle.tda_matrix(s.eps_occ, s.eps_virt, K, None, 2.0)
    w, X = oracle.tda_solve(A, 4)
    f_ref = osp.oscillator_strengths(w, X, dip_ref)
    wd, Xd, dd = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w, X, dip_ref))
    f = ctx.oscillator_strengths(wd, Xd, dd)
    grid = torch.linspace(0.0, 2.0, 3001, dtype=torch.float64, device="cuda")
    S = ctx.strength_function(wd, f, 0.0005, grid)
    ctx.sync()
    assert np.allclose(f.cpu().numpy(), f_ref, rtol=1e-12, atol=1e-15)
    S_ref = osp.strength_function(grid.cpu().numpy(), w, f_ref, 0.0005)
    assert rel_max_err(S.cpu().numpy(), S_ref) < 1e-12


@pytest.mark.parametrize("no,nv", [(2, 3), (3, 23), (4, 24), (5, 20)])
def test_full_tdhf_matches_oracle(no, nv):
    """Blocked Cholesky over 1..4 blocks of 32 with ragged edges; singlet and triplet."""
    need_gpu()
    s = system((16, 16, 16), 0.5, no, nv, seed=no + nv)
    K = oracle.casida_K(s.phi, s.phi_virt, 0.5)
    Kd = oracle.casida_Kd(s.phi, s.phi_virt, 0.5)
    # widen the gaps so that the triplet ground state is stable (A - B, A + B > 0)
    eo, ev = s.eps_occ - 1.0, s.eps_virt + 0.5
    ctx = rsx.Context((16, 16, 16), 0.5, "fp64")
    Kt, Kdt = torch.from_numpy(K).cuda(), torch.from_numpy(Kd).cuda()
    eot, evt = torch.from_numpy(eo).cuda(), torch.from_numpy(ev).cuda()
    nroots = min(6, no * nv)
    for dm in (2.0, 0.0):
        A, B = osp.tdhf_matrices(eo, ev, K, Kd, dm)
        w_ref, v_ref = osp.tdhf_solve(A, B, nroots)
        w, v = ctx.casida_solve_full(eot, evt, Kt, Kdt, dm, nroots, vectors=True)
        ctx.sync()
        w, v = w.cpu().numpy(), v.cpu().numpy()
        assert np.allclose(w, w_ref, rtol=0, atol=1e-11), (w, w_ref)
        for k in range(nroots):
            sgn = np.sign(v[k] @ v_ref[k])
            assert np.allclose(v[k], sgn * v_ref[k], atol=1e-9)


def test_full_tdhf_at_80_cubed_512_transitions():
    """The Casida workload (80^3, 8 x 64 transitions): K from the tensor-core path, the
    full TDHF roots from the device against numpy on the same K; below the TDA roots."""
    need_gpu()
    s = inputs.casida_system(n=80, h=0.25, nocc=8, nvirt=64)
    ctx = rsx.Context(s.shape, s.h, "fp32")
    K = ctx.casida_K(to_dev(s.phi, "fp32"), to_dev(s.phi_virt, "fp32"))
    eot, evt = torch.from_numpy(s.eps_occ).cuda(), torch.from_numpy(s.eps_virt).cuda()
    w = ctx.casida_solve_full(eot, evt, K, None, 1.0, 10)
    w_tda = ctx.casida_solve(eot, evt, K, None, 1.0, 10)
    ctx.sync()
    A, B = osp.tdhf_matrices(s.eps_occ, s.eps_virt, K.cpu().numpy(), None, 1.0)
    w_ref, _ = osp.tdhf_solve(A, B, 10)
    assert np.allclose(w.cpu().numpy(), w_ref, rtol=0, atol=1e-10)
    assert np.all(w.cpu().numpy() <= w_tda.cpu().numpy() + 1e-12)
