"""Failure detection without faulting the GPU (testing aids of the C ABI).

* A bounded device wait made to run out: the grid-wide barrier of the cooperative
  Householder reduction (no asynchronous copies in flight there) with its spin limit set
  to 0, so every CTA but the last arriver gives up at once; rsx_sync_status must report
  RSX_ETIMEOUT and the next call, with the default limit, must be correct again.
* Host-side injection: a workspace allocation that fails (RSX_ENOMEM, nothing launched,
  the context usable afterwards) and an ACE matrix with a flipped sign, whose FP64
  Cholesky meets a non-positive pivot (RSX_ENOTPD deferred to rsx_sync_status).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import TOL, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu


def _tda_case(nt=640, seed=3):
    r = np.random.default_rng(seed)
    B = r.standard_normal((nt, nt)) * 0.02
    K = B @ B.T
    no, nv = 10, nt // 10
    eo = np.sort(r.uniform(-0.8, -0.3, no))
    ev = np.sort(r.uniform(-0.1, 0.5, nv))
    return eo, ev, K


def test_grid_barrier_timeout_is_reported_and_the_context_recovers(monkeypatch):
    need_gpu()
    monkeypatch.setenv("RSX_TRIDIAG_PATH", "coop")
    eo, ev, K = _tda_case()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = rsx.Context((16, 16, 16), 0.4, "fp64")
    ctx.set_wait_limit(0)
    ctx.casida_solve(d(eo), d(ev), d(K), None, 1.0, 10)
    with pytest.raises(rsx.RsxError) as err:
        ctx.sync()
    assert err.value.code == rsx.RSX_ETIMEOUT
    ctx.set_wait_limit(-1)
    w = ctx.casida_solve(d(eo), d(ev), d(K), None, 1.0, 10)
    ctx.sync()
    w_ref, _ = oracle.tda_solve(oracle.tda_matrix(eo, ev, K, None, 1.0), 10)
    assert np.allclose(w.cpu().numpy(), w_ref, rtol=0, atol=1e-12)


def test_injected_allocation_failure_then_recovery():
    need_gpu()
    shape, h = (24, 24, 24), 0.35
    s = inputs.exchange_system(h=h, nocc=2, npsi=3, shape=shape, radius=1.5, seed=2)
    ctx = rsx.Context(shape, h, "fp32")
    phi, psi = to_dev(s.phi, "fp32"), to_dev(s.psi, "fp32")
    out = torch.full_like(psi, float("nan"))
    ctx.inject_fault(rsx.RSX_FAULT_ALLOC, 0)
    with pytest.raises(rsx.RsxError) as err:
        ctx.exchange_apply(phi, psi, out=out)
    assert err.value.code == rsx.RSX_ENOMEM and "injected" in str(err.value)
    ctx.sync()                                   # nothing was launched: no deferred error
    assert torch.isnan(out).all()
    ctx.exchange_apply(phi, psi, out=out)        # the injection fired once
    ctx.sync()
    assert rel_max_err(out.double().cpu().numpy(), oracle.exchange_apply(s.phi, s.psi, h)) < TOL["fp32"]


def test_injected_bad_pivot_is_reported_as_not_positive_definite():
    need_gpu()
    shape, h = (24, 24, 24), 0.35
    s = inputs.exchange_system(h=h, nocc=3, shape=shape, radius=1.5, seed=1)
    ctx = rsx.Context(shape, h, "fp64")
    phi = to_dev(s.phi, "fp64")
    ctx.inject_fault(rsx.RSX_FAULT_PIVOT)
    ctx.ace_build(phi)
    with pytest.raises(rsx.RsxError) as err:
        ctx.sync()
    assert err.value.code == rsx.RSX_ENOTPD
    xi = ctx.ace_build(phi)                      # once only: the next build is correct
    ctx.sync()
    assert rel_max_err(xi.cpu().numpy(), oracle.ace_build(s.phi, h)) < 1e-10


def test_faults_armed_from_the_environment(monkeypatch):
    """RSX_INJECT_FAULT, read by rsx_create: alloc:0 fails the first workspace allocation,
    pivot makes the first ACE build report RSX_ENOTPD; both fire once."""
    need_gpu()
    shape, h = (24, 24, 24), 0.35
    s = inputs.exchange_system(h=h, nocc=3, npsi=2, shape=shape, radius=1.5, seed=4)
    monkeypatch.setenv("RSX_INJECT_FAULT", "alloc:0")
    ctx = rsx.Context(shape, h, "fp32")
    phi, psi = to_dev(s.phi, "fp32"), to_dev(s.psi, "fp32")
    with pytest.raises(rsx.RsxError) as err:
        ctx.exchange_apply(phi, psi)
    assert err.value.code == rsx.RSX_ENOMEM
    out = ctx.exchange_apply(phi, psi)
    ctx.sync()
    assert rel_max_err(out.double().cpu().numpy(), oracle.exchange_apply(s.phi, s.psi, h)) < TOL["fp32"]
    monkeypatch.setenv("RSX_INJECT_FAULT", "pivot")
    ctx2 = rsx.Context(shape, h, "fp32")
    ctx2.ace_build(phi)
    with pytest.raises(rsx.RsxError) as err:
        ctx2.sync()
    assert err.value.code == rsx.RSX_ENOTPD
    ctx2.ace_build(phi)
    ctx2.sync()
