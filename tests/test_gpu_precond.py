"""GPU tests of the plain block eigensolver and the learned-preconditioner network kernels
against the FP64 oracle (forward, loss, gradients; eigenvalues vs a dense eigh)."""
import numpy as np
import pytest
import torch

from oracle import eigensolver as oe
from paper_2405_01522_gb300 import inputs, precond, rsx
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().double().numpy()


def unpack(p):
    """flat parameter vector -> oracle parameter list (weights rounded to bf16 as the kernels use them)."""
    shapes = [(16, 2), (16, 16), (1, 16)]
    out, o = [], 0
    for co, ci in shapes:
        w = p[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = p[o:o + co]
        o += co
        out.append((bf16_round(w), np.asarray(b, dtype=np.float64)))
    return out


@pytest.mark.parametrize("shape", [(2, 12, 10, 9), (1, 8, 8, 8)])
def test_network_forward_loss_and_gradients_vs_oracle(shape):
    need_gpu()
    B, D, H, W = shape
    rng = np.random.default_rng(B * 100 + D)
    p = precond.init_params(seed=3)
    p[:16 * 2 * 27] *= 1.0
    net = rsx.Net(p)
    x = rng.standard_normal((B, 2, D, H, W)).astype(np.float32)
    t = rng.standard_normal((B, D, H, W)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = net.forward(xd).cpu().numpy()
    params = unpack(p)
    border = 1
    loss_ref, g_ref = 0.0, None
    for b in range(B):
        o, _ = oe.net_forward(x[b].astype(np.float64), params)
        assert np.max(np.abs(out[b] - o[0])) <= 2e-5 * max(1e-3, np.max(np.abs(o)))
    # batch loss = mean over all masked voxels of all samples
    mask = np.zeros((D, H, W))
    mask[border:D - border, border:H - border, border:W - border] = 1
    tot = np.zeros(len(p))
    lsum = 0.0
    for b in range(B):
        l_b, g_b = oe.net_loss_and_grads(x[b].astype(np.float64), t[b].astype(np.float64), params, mask)
        lsum += l_b
        flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in g_b])
        tot += flat
    loss_ref, g_ref = lsum / B, tot / B
    loss, g = net.loss_grad(xd, td, border=border)
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_plain_eigensolver_matches_dense_eigenvalues():
    need_gpu()
    n, h, nb = 12, 0.5, 4
    V = inputs.model_potential(n=n, h=h, natoms=2, Z=2.0, rc=0.8, radius=1.0, seed=1)
    w_ref = np.linalg.eigvalsh(oe.hamiltonian_dense(V, h))[:nb]
    psi0 = inputs.starting_orbitals(n=n, h=h, nband=nb, radius=1.0, seed=2)
    res = precond.solve(torch.from_numpy(V).float().cuda(), h, torch.from_numpy(psi0).float().cuda(), nb,
                        tol=1e-9, max_iter=300)
    assert np.allclose(res["theta"], w_ref, rtol=0, atol=2e-5 * np.abs(w_ref).max())


def test_learned_preconditioner_pipeline_small():
    """Plain run -> training pairs -> a few Adam epochs on the GPU -> learned run converges
    to the same energy as the plain run (the gain is measured, not asserted, here)."""
    need_gpu()
    n, h, nb = 24, 0.4, 4
    V = torch.from_numpy(inputs.model_potential(n=n, h=h, natoms=2, Z=3.0, rc=0.6, radius=1.5, seed=4)).float().cuda()
    vscale = float(1.0 / V.abs().max())
    psi0 = torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nb, radius=1.5, seed=5)).float().cuda()
    plain = precond.solve(V, h, psi0, nb, tol=1e-7, vscale=vscale, record_every=2)
    X, Y = precond.make_pairs(V, h, plain, vscale, crop=16, crops_per_sample=4, seed=6)
    net = rsx.Net(precond.init_params(seed=7))
    losses = precond.train(net, X, Y, epochs=3, batch=16, lr=1e-3, border=3)
    assert np.isfinite(losses).all() and losses[-1] < losses[0]
    learned = precond.solve(V, h, psi0, nb, net=net, tol=1e-7, vscale=vscale)
    assert abs(learned["energy"] - plain["energy"]) < 1e-5
