"""GPU test of rsx_exchange_apply_noalloc, the allocation-free exchange entry point.

Callers whose device memory is owned by their own pool allocator, or who cannot take a
workspace regrow in a latency-critical loop, use this entry point: its FFT scratch is a
fixed array inside the library.  The test calls it through the C ABI twice in a row
(the second call reuses the array left by the first) and checks both results against
rsx_exchange_apply within the FP32 parity tolerance of the other GPU tests.  It sits in
its own file, collected last, and passes alone or after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import TOL, need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_exchange_apply_twice():
    need_gpu()
    shape, h = (24, 24, 40), 0.3
    s = inputs.exchange_system(h=h, nocc=3, npsi=4, shape=shape, radius=1.5, seed=7)
    ctx = rsx.Context(shape, h, "fp32")
    lib = rsx.load()
    phi, psi = to_dev(s.phi, "fp32"), to_dev(s.psi, "fp32")
    ref = ctx.exchange_apply(phi, psi)
    ctx.sync()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full_like(psi, float("nan"))
        code = lib.rsx_exchange_apply_noalloc(ctx.handle, rsx._ptr(phi), 3, rsx._ptr(psi), 4, rsx._ptr(out), stream)
        assert code == rsx.RSX_OK, lib.rsx_last_error(ctx.handle).decode()
        ctx.sync()
        assert torch.isfinite(out).all()
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
