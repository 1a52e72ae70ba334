"""GPU tests of the uneven molecule batch (persistent launches under a CUDA graph).

W_m = Vx[phi_m] phi_m and the ACE projectors xi_m of every molecule must match the
single-problem path (rsx_exchange_apply / rsx_ace_build) and the oracle; the captured
graph must replay to the same bits and follow rebinding to new arrays.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import TOL, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu


def molecules(edges, noccs, seed0=11):
    out = []
    for m, (e, k) in enumerate(zip(edges, noccs)):
        s = inputs.batched_system(n=e, h=0.3, nocc=k, ncentres=6, npsi=0, seed=seed0 + m, radius=2.0)
        out.append(s)
    return out


def run_batch(mols, h=0.3):
    b = rsx.Batch([m.shape[0] for m in mols], [m.phi.shape[0] for m in mols], h)
    phi = [to_dev(m.phi, "fp32") for m in mols]
    W = [torch.empty_like(p) for p in phi]
    xi = [torch.empty_like(p) for p in phi]
    b.bind(phi, W, xi)
    b.run()
    b.sync()
    return b, phi, W, xi


def test_batch_matches_single_problem_path_and_oracle():
    need_gpu()
    mols = molecules([48, 64, 48, 80], [3, 2, 1, 4])
    b, phi, W, xi = run_batch(mols)
    for m, s in enumerate(mols):
        ctx = rsx.Context(s.shape, s.h, "fp32")
        if s.shape[0] % 32 == 0:   # the batch runs the 8-lane y/z split at these edges
            ctx.set_tuning(p2_lanes=8, p2_threads=256)
        w1 = ctx.exchange_apply(phi[m], phi[m])
        x1 = ctx.ace_build(phi[m])
        ctx.sync()
        assert torch.equal(W[m], w1), m                      # same kernels, same order
        assert rel_max_err(xi[m].double().cpu().numpy(), x1.double().cpu().numpy()) < 1e-5, m
    # one molecule against the FP64 oracle
    s = mols[2]
    ref = oracle.exchange_apply(s.phi, s.phi, s.h)
    assert rel_max_err(W[2].double().cpu().numpy(), ref) < TOL["fp32"]
    zeta = oracle.ace_build(s.phi, s.h)
    assert rel_max_err(xi[2].double().cpu().numpy(), zeta) < 2e-5


def test_graph_replay_and_rebinding():
    need_gpu()
    mols = molecules([48, 48], [2, 3], seed0=5)
    b, phi, W, xi = run_batch(mols)
    first = [w.clone() for w in W]
    b.run()
    b.sync()
    for a, c in zip(first, W):
        assert torch.equal(a, c)
    # new arrays (swapped orbital sets of equal shape are not available: use scaled inputs)
    phi2 = [2.0 * p for p in phi]
    W2 = [torch.empty_like(p) for p in phi2]
    xi2 = [torch.empty_like(p) for p in phi2]
    b.bind(phi2, W2, xi2)
    b.run()
    b.sync()
    for a, c in zip(first, W2):
        assert rel_max_err(c.double().cpu().numpy(), 8.0 * a.double().cpu().numpy()) < 1e-6


def test_batch_rejects_unsupported_edges():
    need_gpu()
    with pytest.raises(rsx.RsxError):
        rsx.Batch([40], [2], 0.3)


def test_full_size_uneven_batch_every_edge():
    """The 64-molecule batch (edges from {48, 64, 80, 96, 112} at h = 0.2, N_occ U{2..24}):
    every molecule's W against the single-problem path, xi through the ACE identity
    -xi <xi, phi> = W (holds at any size), and for each edge the molecule with the most
    orbitals against the FP64 oracle at sampled points (direct sums, one point at a time)."""
    need_gpu()
    h = 0.2
    desc = inputs.uneven_batch()
    assert {e for e, _, _ in desc} == {48, 64, 80, 96, 112}
    mols = [inputs.batched_system(n=e, h=h, nocc=k, npsi=0, seed=sd) for e, k, sd in desc]
    b, phi, W, xi = run_batch(mols, h=h)
    ctxs = {}
    for m, (e, k, _) in enumerate(desc):
        if e not in ctxs:
            ctxs[e] = rsx.Context((e, e, e), h, "fp32")
            if e % 32 == 0:   # the batch runs the 8-lane y/z split at these edges
                ctxs[e].set_tuning(p2_lanes=8, p2_threads=256)
        ctx = ctxs[e]
        w1 = ctx.exchange_apply(phi[m], phi[m])
        ctx.sync()
        err = rel_max_err(W[m].double().cpu().numpy(), w1.double().cpu().numpy())
        assert torch.equal(W[m], w1), (m, e, k, err)
        # ACE identity on the batch's own xi (FP64 products of the FP32 arrays)
        X = xi[m].double().reshape(k, -1)
        P = phi[m].double().reshape(k, -1)
        C = h ** 3 * (X @ P.T)
        ace = -(C.T @ X)
        Wd = W[m].double().reshape(k, -1)
        assert ((ace - Wd).abs().max() / Wd.abs().max()).item() < 3e-5, (m, e, k)
    for c in ctxs.values():
        c.close()
    rng = np.random.default_rng(11)
    for e in sorted({e for e, _, _ in desc}):
        m = max((i for i, d in enumerate(desc) if d[0] == e), key=lambda i: desc[i][1])
        k = desc[m][1]
        p = k - 1
        # sample points within 2.5 bohr of the box centre, where the orbitals live
        pts = [tuple(int(round(e / 2 + c / h)) for c in rng.uniform(-2.5 / 3 ** 0.5, 2.5 / 3 ** 0.5, 3))
               for _ in range(8)]
        ref = oracle.exchange_apply_at(mols[m].phi, mols[m].phi[p], h, pts)
        got = np.array([W[m][p][q].item() for q in pts])
        assert np.max(np.abs(got - ref)) < TOL["fp32"] * np.max(np.abs(ref)), (m, e, k)
