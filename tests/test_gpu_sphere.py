"""GPU parity for the spherical domain (Sec. 3.4: a sphere with zero boundary values):
the block eigensolver and the SCF loop restricted to the grid points inside a sphere,
against the FP64 oracle's restricted matrices."""
import numpy as np
import pytest
import torch

import oracle.scf as oscf
from oracle import eigensolver as oe
from paper_2405_01522_gb300 import inputs, precond, rsx
from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,h,radius,free", [(12, 0.5, 2.5, False), (16, 0.5, 3.5, True)])
def test_eigensolver_in_a_sphere(n, h, radius, free):
    need_gpu()
    nb = 4
    V = np.zeros((n, n, n)) if free else inputs.model_potential(n=n, h=h, natoms=2, Z=2.0, rc=0.8, radius=1.0, seed=1)
    m = oe.sphere_mask((n, n, n), h, radius)
    Hm, _ = oe.hamiltonian_masked(V, h, m)
    w_ref = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[:nb]
    psi0 = inputs.starting_orbitals(n=n, h=h, nband=nb, radius=1.0, seed=2)
    es = rsx.Eigensolver(torch.from_numpy(V).float().cuda(), h, nb)
    md = torch.from_numpy(m).float().cuda()
    es.set_mask(md)
    es.init(torch.from_numpy(psi0).float().cuda())
    th = None
    for _ in range(400):
        th = es.step()
    psi = es.orbitals().cpu().numpy()
    es.close()
    assert np.allclose(th, w_ref, rtol=0, atol=2e-5 * np.abs(w_ref).max())
    assert np.abs(psi[:, m == 0]).max() == 0.0          # zero outside the sphere, exactly


def test_scf_in_a_sphere_vs_oracle():
    need_gpu()
    n, h, nocc, radius = 16, 0.5, 2, 3.0
    v = inputs.model_potential(n=n, h=h, natoms=2, Z=2.0, rc=0.8, radius=1.0, seed=3)
    m = oe.sphere_mask(v.shape, h, radius)
    ref = oscf.scf(v, h, nocc, mode="ace", alpha=0.3, tol=1e-10, mask=m)
    ctx = rsx.Context((n, n, n), h, "fp32")
    md = torch.from_numpy(m).float().cuda()
    scf = rsx.SCF(ctx, to_dev(v, "fp32"), nocc, ace=True, alpha=0.3, mask=md)
    scf.init(to_dev(inputs.starting_orbitals(n=n, h=h, nband=nocc, radius=1.0, seed=5), "fp32"))
    hist = []
    for _ in range(80):
        hist.append(scf.step(inner=2))
        if len(hist) > 1 and hist[-1]["reldens"] < 2e-6:
            break
    phi = scf.orbitals().cpu().numpy()
    scf.close()
    assert hist[-1]["reldens"] < 2e-6, [r["reldens"] for r in hist]
    assert abs(hist[-1]["energy"] - ref["energy"]) < 2e-5 * abs(ref["energy"])
    assert np.abs(phi[:, m == 0]).max() == 0.0
