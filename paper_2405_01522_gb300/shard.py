"""One exchange apply and ACE build split over ranks (one GPU per rank).

The pair solves are independent (Sec. 3.1: one Poisson problem per orbital pair), so a
problem of n_occ orbitals and n_psi functions shards by output function: rank r owns a
contiguous block of the psi_p and of the rows W_k of W = Vx[Phi] Phi and solves only their
pairs (Eq. 2, every phi_j against its own outputs); nothing is summed across ranks for
Vx psi_p.  ACE (Eqs. 11-12) needs two exchanges:

* M = h^3 Phi^T W: rank r computes the column block M[:, k0:k1] = h^3 Phi W_block^T of
  its own rows; the zero-padded blocks are summed over the ranks (all-reduce), giving M
  on every rank;
* xi = L^-1 W needs every row of W: the blocks of W are all-gathered (padded to the
  largest block), then every rank factorises -M = L L^T in FP64 and forms xi.

The local steps are supplied by an `ops` object with three methods, so that the same
driver runs on the library (`LibraryOps`, a GPU per rank, NCCL) or on any other
implementation of the steps with torch.distributed on host tensors (gloo):

    ops.exchange(phi, psi_block) -> Vx[phi] psi_block            [n][N]
    ops.gram(a, b)               -> h^3 <a_i, b_j>               [na][nb] float64
    ops.ace_factor(M, W)         -> xi = L^-1 W, -sym(M) = L L^T [nocc][N]
"""
import torch
import torch.distributed as dist


def block_range(n, world, rank):
    """Contiguous block [lo, hi) of n items owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def all_gather_rows(block, n, group=None):
    """Concatenate every rank's row block (ranks in order, block_range layout) into the n
    rows of the full array; blocks are padded to the largest size for the collective."""
    world = dist.get_world_size(group)
    rows = [block_range(n, world, r) for r in range(world)]
    width = max(hi - lo for lo, hi in rows)
    pad = torch.zeros((width,) + tuple(block.shape[1:]), dtype=block.dtype, device=block.device)
    pad[:block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:hi - lo] for p, (lo, hi) in zip(parts, rows)])


def exchange_ace_sharded(phi, psi, ops, group=None):
    """Rank-local share of Vx[phi] psi and the full ACE projectors, see the module notes.

    phi: [nocc][...] and psi: [npsi][...] (every rank holds both; only its blocks are
    solved).  Returns dict(vx=Vx psi for this rank's block, psi_range=(p0, p1),
    W=all rows of Vx[phi] phi, M=h^3 <phi, W> (nocc x nocc, float64), xi=ACE projectors)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    nocc, npsi = phi.shape[0], psi.shape[0]
    p0, p1 = block_range(npsi, world, rank)
    k0, k1 = block_range(nocc, world, rank)
    vx = ops.exchange(phi, psi[p0:p1]) if p1 > p0 else psi[:0].clone()
    w_block = ops.exchange(phi, phi[k0:k1]) if k1 > k0 else phi[:0].clone()
    M = torch.zeros((nocc, nocc), dtype=torch.float64, device=phi.device)
    if k1 > k0:
        M[:, k0:k1] = ops.gram(phi, w_block)
    dist.all_reduce(M, op=dist.ReduceOp.SUM, group=group)
    W = all_gather_rows(w_block, nocc, group)
    xi = ops.ace_factor(M.clone(), W)
    return {"vx": vx, "psi_range": (p0, p1), "W": W, "M": M, "xi": xi}


class LibraryOps:
    """The local steps on one GPU through the library (rsx_exchange_apply, rsx_gram,
    rsx_ace_factor) of a context `ctx`."""

    def __init__(self, ctx):
        self.ctx = ctx

    def exchange(self, phi, psi_block):
        return self.ctx.exchange_apply(phi, psi_block.contiguous())

    def gram(self, a, b):
        return self.ctx.gram(a.contiguous(), b.contiguous())

    def ace_factor(self, M, W):
        return self.ctx.ace_factor(M, W.contiguous())
