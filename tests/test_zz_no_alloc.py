"""GPU test of rsx_exchange_apply_noalloc, the allocation-free exchange entry point.

Callers whose device memory is owned by their own pool allocator, or who cannot take a
workspace regrow in a latency-critical loop, use this entry point: its FFT scratch is a
fixed array inside the library.  The test works on a fresh context: the first call
(which may load the library's modules, the one allocation the header allows) uses one
set of inputs, the second call another set; the driver's free-memory count must not
change across the second call, and each call's result must match rsx_exchange_apply on
its own inputs within the FP32 parity tolerance of the other GPU tests (so the second
call cannot lean on what the first left in the shared array).  It sits in its own file,
collected last, and passes alone or after the rest of the suite.
"""
import ctypes

import pytest
import torch

from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import TOL, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(lib, ctx, phi, psi, out, stream):
    nocc, npsi = phi.shape[0], psi.shape[0]
    return lib.rsx_exchange_apply_noalloc(ctx.handle, rsx._ptr(phi), nocc, rsx._ptr(psi), npsi, rsx._ptr(out), stream)


def test_noalloc_matches_exchange_apply_twice():
    need_gpu()
    shape, h = (24, 24, 40), 0.3
    first = inputs.exchange_system(h=h, nocc=2, npsi=3, shape=shape, radius=1.5, seed=3)
    second = inputs.exchange_system(h=h, nocc=3, npsi=4, shape=shape, radius=1.5, seed=7)
    ctx = rsx.Context(shape, h, "fp32")             # fresh context: no workspace grown yet
    lib = rsx.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sets = []
    for s in (first, second):
        phi, psi = to_dev(s.phi, "fp32"), to_dev(s.psi, "fp32")
        sets.append((phi, psi, torch.full_like(psi, float("nan"))))
    torch.cuda.synchronize()

    # first call: set-up (module loading, symbol lookup) happens here
    phi, psi, out = sets[0]
    assert _noalloc(lib, ctx, phi, psi, out, stream) == rsx.RSX_OK, lib.rsx_last_error(ctx.handle).decode()
    torch.cuda.synchronize()

    # second call, other inputs: the driver's free device memory must not move
    phi, psi, out = sets[1]
    free_before = torch.cuda.mem_get_info()[0]
    code = _noalloc(lib, ctx, phi, psi, out, stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert code == rsx.RSX_OK, lib.rsx_last_error(ctx.handle).decode()
    assert free_after == free_before, (free_before, free_after)
    assert ctx.lib.rsx_sync_status(ctx.handle, stream) == rsx.RSX_OK

    # only now the reference path (which grows the context workspace)
    for call, (phi, psi, out) in enumerate(sets):
        ref = ctx.exchange_apply(phi, psi)
        ctx.sync()
        assert torch.isfinite(out).all(), call
        assert rel_max_err(out.double().cpu().numpy(), ref.double().cpu().numpy()) < TOL["fp32"], call


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    need_gpu()
    shape, h = (96, 96, 96), 0.2
    ctx = rsx.Context(shape, h, "fp32")
    lib = rsx.load()
    nocc = 10                                       # 10 * 97 * 96 * 96 * 8 B > 64 MiB
    phi = torch.zeros((nocc,) + shape, dtype=torch.float32, device="cuda")
    psi = torch.zeros((1,) + shape, dtype=torch.float32, device="cuda")
    out = torch.empty_like(psi)
    code = lib.rsx_exchange_apply_noalloc(ctx.handle, rsx._ptr(phi), nocc, rsx._ptr(psi), 1, rsx._ptr(out), None)
    assert code == rsx.RSX_EINVAL
    assert "64 MiB" in lib.rsx_last_error(ctx.handle).decode()
