"""GPU test of the autotuner: valid choice, cache round trip, identical results."""
import os

import pytest
import torch

from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_autotune_choice_cache_and_bitwise_results(tmp_path):
    need_gpu()
    shape, h = (24, 24, 24), 0.35
    s = inputs.exchange_system(h=h, nocc=3, npsi=5, shape=shape, radius=1.5, seed=4)
    ctx = rsx.Context(shape, h, "fp32")
    phi, psi = to_dev(s.phi, "fp32"), to_dev(s.psi, "fp32")
    ref = ctx.exchange_apply(phi, psi)
    cache = str(tmp_path / "tune.txt")
    t1 = ctx.autotune(3, 5, cache=cache)
    assert t1["p2_threads"] in (256, 384, 512) and t1["chunk_outputs"] in (0, 1, 2, 4)
    assert t1["best_ms"] > 0 and os.path.exists(cache)
    out = ctx.exchange_apply(phi, psi)
    ctx.sync()
    assert torch.equal(out, ref)            # tuning changes scheduling, not arithmetic
    ctx2 = rsx.Context(shape, h, "fp32")
    t2 = ctx2.autotune(3, 5, cache=cache)
    assert t2["best_ms"] == -1.0 and t2["p2_threads"] == t1["p2_threads"]
    assert t2["chunk_outputs"] == t1["chunk_outputs"]
    for p2, ch in ((512, 1), (384, 4), (256, 2), (256, 0)):
        ctx2.set_tuning(p2, ch)
        o2 = ctx2.exchange_apply(phi, psi)
        ctx2.sync()
        assert torch.equal(o2, ref)
