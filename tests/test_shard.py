"""One exchange apply + ACE build split over ranks (paper_2405_01522_gb300.shard).

CPU: two and three gloo ranks run the sharded driver with the oracle's steps injected
(test infrastructure); the blocks of Vx psi, the reduced M and the all-gathered W and xi
must equal the single-rank oracle.  GPU: one rank (a gloo group of one) with the
library's steps (rsx_exchange_apply, rsx_gram, rsx_ace_factor) against rsx_ace_build and
the oracle.  Every run here has one GPU, so the NCCL form with a GPU per rank is not run.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2405_01522_gb300 import inputs, shard  # noqa: E402


class OracleOps:
    """The sharded driver's local steps by the FP64 oracle, on host tensors."""

    def __init__(self, h):
        self.h = h

    def exchange(self, phi, psi_block):
        return torch.from_numpy(oracle.exchange_apply(phi.numpy(), psi_block.numpy(), self.h))

    def gram(self, a, b):
        return torch.from_numpy(self.h ** 3 * (a.reshape(a.shape[0], -1).numpy() @ b.reshape(b.shape[0], -1).numpy().T))

    def ace_factor(self, M, W):
        m = M.numpy()
        L = np.linalg.cholesky(-0.5 * (m + m.T))
        xi = np.linalg.solve(L, W.reshape(W.shape[0], -1).numpy()).reshape(W.shape)
        return torch.from_numpy(xi)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    return inputs.exchange_system(n=8, h=0.5, nocc=5, npsi=3, radius=1.0, seed=4)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = _system()
    out = shard.exchange_ace_sharded(torch.from_numpy(s.phi), torch.from_numpy(s.psi), OracleOps(s.h))
    q.put((rank, out["psi_range"], out["vx"].numpy(), out["M"].numpy(), out["W"].numpy(), out["xi"].numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_block_ranges_cover_every_item_once():
    for n in (1, 2, 5, 16, 17):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.block_range(n, world, r)
                assert 0 <= lo <= hi <= n
                seen += list(range(lo, hi))
            assert seen == list(range(n))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_exchange_and_ace_match_the_single_rank_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = _system()
    vx_ref = oracle.exchange_apply(s.phi, s.psi, s.h)
    W_ref = oracle.exchange_apply(s.phi, s.phi, s.h)
    M_ref = s.h ** 3 * (s.phi.reshape(5, -1) @ W_ref.reshape(5, -1).T)
    xi_ref = oracle.ace_build(s.phi, s.h)
    vx = np.concatenate([r[2] for r in res])
    assert [r[1] for r in res] == [shard.block_range(3, world, k) for k in range(world)]
    assert np.allclose(vx, vx_ref, rtol=0, atol=1e-13 * np.abs(vx_ref).max())
    for _, _, _, M, W, xi in res:                         # every rank holds the full M, W, xi
        assert np.allclose(M, M_ref, rtol=0, atol=1e-13 * np.abs(M_ref).max())
        assert np.allclose(W, W_ref, rtol=0, atol=1e-13 * np.abs(W_ref).max())
        assert np.allclose(xi, xi_ref, rtol=0, atol=1e-11 * np.abs(xi_ref).max())


@pytest.mark.gpu
def test_sharded_driver_on_the_library_single_rank():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_01522_gb300 import rsx
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        s = inputs.exchange_system(h=0.35, nocc=4, npsi=3, shape=(24, 24, 24), radius=1.5, seed=9)
        ctx = rsx.Context(s.shape, s.h, "fp64")
        phi, psi = torch.from_numpy(s.phi).cuda(), torch.from_numpy(s.psi).cuda()
        out = shard.exchange_ace_sharded(phi, psi, shard.LibraryOps(ctx))
        M_lib = torch.empty((4, 4), dtype=torch.float64, device="cuda")
        xi_lib = ctx.ace_build(phi, M=M_lib)
        ctx.sync()
        assert torch.allclose(out["xi"], xi_lib, rtol=0, atol=1e-12 * xi_lib.abs().max().item())
        assert torch.allclose(out["M"], M_lib, rtol=0, atol=1e-12 * M_lib.abs().max().item())
        ref = oracle.exchange_apply(s.phi, s.psi, s.h)
        assert np.max(np.abs(out["vx"].cpu().numpy() - ref)) < 1e-11 * np.abs(ref).max()
        assert np.max(np.abs(out["xi"].cpu().numpy() - oracle.ace_build(s.phi, s.h))) < 1e-10 * xi_lib.abs().max().item()
    finally:
        dist.destroy_process_group()
