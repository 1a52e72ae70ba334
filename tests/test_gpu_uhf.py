"""GPU parity for the spin-polarised (UHF) Tamm-Dancoff path (Eqs. 4-5 in spin
orbitals): the coupling over alpha and beta transitions from one split-BF16 panel (or
the FP64 plain form) and the FP64 eigen-solve of its matrix, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

TOL_K = {"fp32": 3e-5, "fp64": 1e-11}


def spin_sets(shape, h, noa, nva, nob, nvb):
    a = inputs.casida_system(h=h, nocc=noa, nvirt=nva, shape=shape, radius=1.5, alpha=(0.5, 2.0), seed=1)
    b = inputs.casida_system(h=h, nocc=nob, nvirt=nvb, shape=shape, radius=1.5, alpha=(0.5, 2.0), seed=2)
    return a, b


@pytest.mark.parametrize("shape,h,noa,nva,nob,nvb,prec", [
    ((16, 16, 16), 0.5, 2, 3, 1, 4, "fp32"),
    ((24, 24, 24), 0.45, 3, 5, 2, 6, "fp32"),
    ((24, 24, 40), 0.4, 2, 3, 1, 2, "fp64"),
])
def test_uhf_K_and_roots_vs_oracle(shape, h, noa, nva, nob, nvb, prec):
    need_gpu()
    a, b = spin_sets(shape, h, noa, nva, nob, nvb)
    K_ref = oracle.uhf_K(a.phi, a.phi_virt, b.phi, b.phi_virt, h)
    Kda_ref = oracle.casida_Kd(a.phi, a.phi_virt, h)
    Kdb_ref = oracle.casida_Kd(b.phi, b.phi_virt, h)
    ctx = rsx.Context(shape, h, prec)
    oa, va, ob, vb = (to_dev(x, prec) for x in (a.phi, a.phi_virt, b.phi, b.phi_virt))
    K = ctx.casida_K_uhf(oa, va, ob, vb)
    Kda, Kdb = ctx.casida_Kd(oa, va), ctx.casida_Kd(ob, vb)
    ctx.sync()
    Kh = K.cpu().numpy()
    assert rel_max_err(Kh, K_ref) < TOL_K[prec]
    assert np.allclose(Kh, Kh.T, rtol=0, atol=1e-12 * np.abs(Kh).max())
    eo_a, ev_a = np.sort(np.random.default_rng(3).uniform(-0.8, -0.3, noa)), np.sort(np.random.default_rng(4).uniform(-0.1, 0.5, nva))
    eo_b, ev_b = np.sort(np.random.default_rng(5).uniform(-0.8, -0.3, nob)), np.sort(np.random.default_rng(6).uniform(-0.1, 0.5, nvb))
    nroots = min(6, noa * nva + nob * nvb)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    om = ctx.casida_solve_uhf(dev(eo_a), dev(ev_a), dev(eo_b), dev(ev_b), K, Kda, Kdb, nroots=nroots)
    A_ref = oracle.uhf_tda_matrix(eo_a, ev_a, eo_b, ev_b, Kh, Kda.cpu().numpy(), Kdb.cpu().numpy())
    w_ref = np.linalg.eigvalsh(0.5 * (A_ref + A_ref.T))[:nroots]   # the device symmetrises A
    assert np.max(np.abs(om.cpu().numpy() - w_ref)) < 1e-10
    # the roots against the oracle's own matrix (FP32 K error propagated)
    w_full = np.linalg.eigvalsh(oracle.uhf_tda_matrix(eo_a, ev_a, eo_b, ev_b, K_ref, Kda_ref, Kdb_ref))[:nroots]
    assert np.max(np.abs(om.cpu().numpy() - w_full)) * oracle.HARTREE_EV < (1e-5 if prec == "fp32" else 1e-9)


def test_uhf_closed_shell_equals_singlets_and_triplets():
    """Alpha = beta orbitals: the UHF roots are the RHF singlets (delta_M = 2) and
    triplets (delta_M = 0) of the same orbitals, all from the device."""
    need_gpu()
    shape, h = (16, 16, 16), 0.5
    a, _ = spin_sets(shape, h, 2, 3, 1, 1)
    ctx = rsx.Context(shape, h, "fp32")
    po, pv = to_dev(a.phi, "fp32"), to_dev(a.phi_virt, "fp32")
    eo, ev = torch.tensor([-0.7, -0.45], dtype=torch.float64).cuda(), torch.tensor([0.05, 0.2, 0.4], dtype=torch.float64).cuda()
    K = ctx.casida_K_uhf(po, pv, po, pv)
    Kd = ctx.casida_Kd(po, pv)
    K1 = ctx.casida_K(po, pv)
    w = ctx.casida_solve_uhf(eo, ev, eo, ev, K, Kd, Kd, nroots=12).cpu().numpy()
    sing = ctx.casida_solve(eo, ev, K1, Kd, delta_M=2.0, nroots=6).cpu().numpy()
    trip = ctx.casida_solve(eo, ev, K1, Kd, delta_M=0.0, nroots=6).cpu().numpy()
    assert np.max(np.abs(np.sort(w) - np.sort(np.concatenate([sing, trip])))) < 1e-9


def test_uhf_without_beta_and_bad_arguments():
    need_gpu()
    shape, h = (16, 16, 16), 0.5
    a, _ = spin_sets(shape, h, 1, 4, 1, 1)
    ctx = rsx.Context(shape, h, "fp32")
    po, pv = to_dev(a.phi, "fp32"), to_dev(a.phi_virt, "fp32")
    K = ctx.casida_K_uhf(po, pv)
    K1 = ctx.casida_K(po, pv)
    ctx.sync()
    assert torch.equal(K, K1)
    # beta counts without beta arrays are rejected before any device work
    rc = ctx.lib.rsx_casida_K_uhf(ctx.handle, rsx._ptr(po), 1, rsx._ptr(pv), 4, None, 1, None, 1, rsx._ptr(K),
                                  rsx._stream(None))
    assert rc == rsx.RSX_EINVAL
