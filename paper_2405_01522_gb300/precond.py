"""Learned eigensolver preconditioner: data from the plain solver, training, evaluation.

The plain method is the block eigensolver of the library (rsx_eig_*) with the
kinetic-energy preconditioner.  The learned preconditioner is the library's 3-layer
conv3d network (rsx_net_*), trained on the GPU by the library's own forward/backward
kernels on (residual -> correction) pairs the plain solver generates:

* input  x = (R_i / |R_i|, vscale V) on a 32^3 crop,
* target y = P_perp (Pi* psi_i - psi_i) / |R_i|, where Pi* projects on the converged
  orbitals and P_perp removes the current orbitals' span (the correction that would take
  psi_i into the converged subspace).

In the solver the network adds directions |R_i| net(R_i/|R_i|, vscale V) next to the plain
ones (taking the place of the LOBPCG P block where the basis would not hold both); the
plain preconditioner stays as the reference for convergence (same energy to 1e-6 Ha) and
as the fallback: a learned run whose energy stops falling (no new minimum by more than the
tolerance within `fallback_patience` steps) drops the network and continues plain.
"""
import time

import numpy as np
import torch

from . import inputs, rsx


def init_params(seed=0):
    """He-uniform weights (fan-in ci * 27), zero biases, last layer scaled by 0.1."""
    rng = inputs.SplitMix64(seed)
    layers = [(16, 2), (16, 16), (1, 16)]
    out = []
    for li, (co, ci) in enumerate(layers):
        bound = np.sqrt(6.0 / (ci * 27)) * (0.1 if li == 2 else 1.0)
        w = np.array([rng.uniform(-bound, bound) for _ in range(co * ci * 27)], dtype=np.float32)
        out += [w, np.zeros(co, dtype=np.float32)]
    return np.concatenate(out)


def should_fall_back(trace, patience, tol):
    """True when none of the last `patience` energies is below the best energy before them
    by more than tol (the learned directions have stopped paying for themselves)."""
    if patience <= 0 or len(trace) <= patience:
        return False
    return min(trace[-patience:]) > min(trace[:-patience]) - tol


def solve(V, h, psi0, nband, net=None, tol=1e-6, max_iter=400, sweeps=3, vscale=1.0, record_every=0,
          energy64=False, fallback_patience=8):
    """Run the block eigensolver until |E_k - E_{k-1}| < tol.

    E is the sum of the step's Ritz values, or with energy64 the block's energy evaluated
    in FP64 after every step (rsx_eig_energy64: far below the FP32 noise of the Ritz
    values; its cost is left out of the times).  Returns a dict with iterations, energy,
    Ritz values, solver wall time (s), the energy trace with the elapsed solver time at
    each entry and, with record_every > 0, a list of (psi_it, R_it) device tensors every
    that many iterations (psi before the step, R the residual the step used).  With a
    network, `fell_back_at` is the iteration after which it was dropped (None: never)."""
    es = rsx.Eigensolver(V, h, nband, vscale=vscale, device=V.device.index or 0)
    es.init(psi0)
    torch.cuda.synchronize()
    trace, rec, times, trace32 = [], [], [], []
    elapsed = 0.0
    E_prev, th, it = None, None, 0
    fell_back_at = None
    for it in range(1, max_iter + 1):
        psi_before = es.orbitals() if record_every and it % record_every == 1 else None
        t0 = time.perf_counter()
        th = es.step(net, sweeps)              # each step synchronises the stream
        elapsed += time.perf_counter() - t0
        if psi_before is not None:
            rec.append((psi_before, es.residual()))
        trace32.append(float(sum(th)))
        E = es.energy64() if energy64 else trace32[-1]
        trace.append(E)
        times.append(elapsed)
        if E_prev is not None and abs(E - E_prev) < tol:
            break
        E_prev = E
        if net is not None and should_fall_back(trace, fallback_patience, tol):
            net, fell_back_at = None, it
    torch.cuda.synchronize()
    dt = elapsed
    psi = es.orbitals()
    es.close()
    return {"iters": it, "energy": trace[-1], "theta": th, "time_s": dt, "trace": trace, "times": times,
            "trace32": trace32, "records": rec, "psi": psi, "fell_back_at": fell_back_at}


def time_to_target(res, e_ref, tol=1e-6):
    """First iteration (1-based) and elapsed solver time from which E stays within tol of
    e_ref for the rest of the run; None if the run ends outside it."""
    hit = None
    for i, E in enumerate(res["trace"]):
        if abs(E - e_ref) < tol:
            if hit is None:
                hit = i
        else:
            hit = None
    if hit is None:
        return None, None
    return hit + 1, res["times"][hit]


def make_pairs(V, h, res, vscale, crop=32, crops_per_sample=16, seed=0):
    """Training crops from one converged plain run (res from solve(..., record_every>0))."""
    n = V.shape[0]
    nb = res["psi"].shape[0]
    ctx = rsx.Context((n, n, n), h, "fp32", device=V.device.index or 0)
    star = res["psi"].contiguous()
    rng = inputs.SplitMix64(seed)
    X, Y = [], []
    vch = (V * vscale).contiguous()
    for psi_it, R_it in res["records"]:
        a = ctx.ace_apply(star, psi_it)          # = -Pi* psi_it
        d = -a - psi_it                          # Pi* psi - psi
        t = d + ctx.ace_apply(psi_it, d)         # P_perp d
        s = torch.sqrt((R_it.double() ** 2).sum(dim=(1, 2, 3)) * h ** 3).float().clamp_min(1e-30)
        for b in range(nb):
            for _ in range(crops_per_sample):
                z, y, x = (rng.integer(0, n - crop) for _ in range(3))
                sl = (slice(z, z + crop), slice(y, y + crop), slice(x, x + crop))
                X.append(torch.stack([R_it[b][sl] / s[b], vch[sl]]))
                Y.append(t[b][sl] / s[b])
    ctx.close()
    return torch.stack(X).contiguous(), torch.stack(Y).contiguous()


def train(net, X, Y, epochs=4, batch=32, lr=1e-3, border=3, seed=0):
    """Adam on the library's kernels; returns the per-epoch mean losses."""
    n = X.shape[0]
    rng = inputs.SplitMix64(seed)
    losses = []
    for ep in range(epochs):
        perm = list(range(n))
        for i in range(n - 1, 0, -1):                 # Fisher-Yates with the seeded stream
            j = rng.integer(0, i)
            perm[i], perm[j] = perm[j], perm[i]
        idx = torch.tensor(perm, device=X.device)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            sel = idx[b0:b0 + batch]
            xb, yb = X[sel].contiguous(), Y[sel].contiguous()
            tot += net.train_step(xb, yb, lr, border=border)
            cnt += 1
        losses.append(tot / max(cnt, 1))
    return losses
