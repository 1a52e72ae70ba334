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
    # the fallback rule ran alongside: either it never fired, or the run went on plain
    fb = learned["fell_back_at"]
    assert fb is None or 1 <= fb <= learned["iters"]
    # with no patience at all the network is dropped after the first step without a new
    # minimum; the run still ends at the plain energy
    quick = precond.solve(V, h, psi0, nb, net=net, tol=1e-7, vscale=vscale, fallback_patience=1)
    assert abs(quick["energy"] - plain["energy"]) < 1e-5


def test_energy64_is_the_rayleigh_ritz_trace_of_the_dense_hamiltonian():
    """rsx_eig_energy64 against the oracle: trace(S^-1 Psi^T H Psi) with the dense FD4
    Hamiltonian and the same FP32 orbitals in FP64 (before convergence, where the block is
    not orthonormal in any precision), and above the sum of the lowest dense eigenvalues by
    less than 1e-9 of it once converged (variational)."""
    need_gpu()
    n, h, nb = 12, 0.5, 4
    V = inputs.model_potential(n=n, h=h, natoms=2, Z=2.0, rc=0.8, radius=1.0, seed=1)
    Hd = oe.hamiltonian_dense(V, h)
    psi0 = inputs.starting_orbitals(n=n, h=h, nband=nb, radius=1.0, seed=2)
    es = rsx.Eigensolver(torch.from_numpy(V).float().cuda(), h, nb)
    es.init(torch.from_numpy(psi0).float().cuda())
    es.step()
    P = es.orbitals().double().cpu().numpy().reshape(nb, -1)
    S, Hs = h ** 3 * (P @ P.T), h ** 3 * (P @ Hd @ P.T)
    e_ref = np.trace(np.linalg.solve(S, Hs))
    assert abs(es.energy64() - e_ref) <= 1e-12 * abs(e_ref)
    for _ in range(300):
        es.step()
    w = np.linalg.eigvalsh(Hd)[:nb]
    e = es.energy64()
    assert -1e-12 * abs(w.sum()) <= e - w.sum() <= 1e-9 * abs(w.sum())
    es.close()


def test_learned_vs_plain_on_an_unseen_system(record_property):
    """The learned preconditioner's gain, measured: train on pairs from plain runs on two
    systems (48^3, 8 bands), then on a third system run the plain and the learned solver
    with FP64 energies after every step against an independent plain reference converged
    to |dE| < 1e-10 Ha.  Both must come (and stay) within 1e-6 Ha of it and end within
    1e-6 Ha of each other; the iterations and solver times to 1e-6 Ha are recorded (the
    measured gain: none so far -- the learned run needs a few more iterations at ~3x the
    cost per iteration), and the learned directions may cost at most 50% more iterations
    than the plain method (they enter a Rayleigh-Ritz next to the plain ones)."""
    need_gpu()
    n, h, nb = 48, 0.25, 8
    pots = [torch.from_numpy(inputs.model_potential(n=n, h=h, natoms=3, Z=4.0, rc=0.6, radius=2.0, seed=s)).float().cuda()
            for s in (51, 52, 53)]
    vscale = float(1.0 / max(float(v.abs().max()) for v in pots))
    psi0 = [torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nb, radius=2.0, seed=60 + s)).float().cuda()
            for s in range(3)]
    Xs, Ys = [], []
    for i in range(2):
        res = precond.solve(pots[i], h, psi0[i], nb, tol=1e-7, vscale=vscale, record_every=2, max_iter=400)
        X, Y = precond.make_pairs(pots[i], h, res, vscale, crop=24, crops_per_sample=6, seed=i)
        Xs.append(X)
        Ys.append(Y)
    X, Y = torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous()
    net = rsx.Net(precond.init_params(seed=0))
    losses = precond.train(net, X, Y, epochs=4, batch=32, lr=1e-3, border=3)
    assert losses[-1] < losses[0]
    ref = precond.solve(pots[2], h, psi0[2], nb, tol=1e-10, vscale=vscale, max_iter=3000, energy64=True)
    plain = precond.solve(pots[2], h, psi0[2], nb, tol=1e-9, vscale=vscale, max_iter=1500, energy64=True)
    learned = precond.solve(pots[2], h, psi0[2], nb, net=net, tol=1e-9, vscale=vscale, max_iter=1500,
                            energy64=True)
    net.close()
    ip, tp = precond.time_to_target(plain, ref["energy"])
    il, tl = precond.time_to_target(learned, ref["energy"])
    record_property("plain_iters_to_1e-6", ip)
    record_property("learned_iters_to_1e-6", il)
    record_property("plain_s_to_1e-6", tp)
    record_property("learned_s_to_1e-6", tl)
    print(f"learned vs plain to 1e-6 Ha: iterations {il} vs {ip}, solver time {tl} vs {tp} s", flush=True)
    assert ip is not None and il is not None, (ip, il)
    assert abs(learned["energy"] - plain["energy"]) < 1e-6
    assert il <= 1.5 * ip, (il, ip, tl, tp)
