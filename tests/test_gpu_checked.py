"""The bounds-checked build (librsx_checked.so, RSX_CHECKED=1) on small cases of every FFT-pass
mode: FP32 and FP64 exchange (odd A, nx != ny, the largest edge), the Poisson solve, ACE
build and apply, and the Casida K and K_d.  No index of the passes may leave its array
(rsx_sync_status would report RSX_EBOUNDS), and the results still match the oracle.
Runs in a child process, since a process loads one variant of the library."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
from paper_2405_01522_gb300 import inputs, rsx
assert rsx.LIB_PATH.endswith("librsx_checked.so")
def rel(a, b): return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
for shape, h, nocc, npsi, prec in [((24, 24, 24), 0.35, 2, 3, "fp32"), ((56, 56, 24), 0.3, 1, 2, "fp32"),
                                   ((16, 16, 24), 0.4, 2, 2, "fp64"), ((112, 112, 112), 0.25, 1, 1, "fp32")]:
    s = inputs.exchange_system(h=h, nocc=nocc, npsi=npsi, shape=shape, radius=1.5, seed=1)
    dt = torch.float32 if prec == "fp32" else torch.float64
    ctx = rsx.Context(shape, h, prec)
    phi, psi = torch.from_numpy(s.phi).to(dt).cuda(), torch.from_numpy(s.psi).to(dt).cuda()
    v = ctx.exchange_apply(phi, psi)
    ctx.sync()
    e = rel(v.double().cpu().numpy(), oracle.exchange_apply(s.phi, s.psi, h))
    assert e < (1e-5 if prec == "fp32" else 1e-11), (shape, prec, e)
    xi = ctx.ace_build(phi)
    va = ctx.ace_apply(xi, phi)
    w = ctx.exchange_apply(phi, phi)
    ctx.sync()
    assert rel(va.double().cpu().numpy(), w.double().cpu().numpy()) < (3e-5 if prec == "fp32" else 1e-10)
    rho = phi[0] * phi[0]
    pot = ctx.poisson(rho.contiguous())
    ctx.sync()
    assert rel(pot.double().cpu().numpy(), oracle.poisson_fft(rho.double().cpu().numpy(), h)) < 1e-5
    print("ok", shape, prec, flush=True)
for prec in ("fp32", "fp64"):
    c = inputs.casida_system(h=0.45, nocc=2, nvirt=5, shape=(24, 24, 24), radius=1.5, alpha=(0.5, 2.0), seed=0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    ctx = rsx.Context((24, 24, 24), 0.45, prec)
    po, pv = torch.from_numpy(c.phi).to(dt).cuda(), torch.from_numpy(c.phi_virt).to(dt).cuda()
    K, Kd = ctx.casida_K(po, pv), ctx.casida_Kd(po, pv)
    ctx.sync()
    assert rel(K.cpu().numpy(), oracle.casida_K(c.phi, c.phi_virt, 0.45)) < (3e-5 if prec == "fp32" else 1e-11)
    assert rel(Kd.cpu().numpy(), oracle.casida_Kd(c.phi, c.phi_virt, 0.45)) < (1e-5 if prec == "fp32" else 1e-11)
    print("ok casida", prec, flush=True)
print("checked build clean", flush=True)
'''


@pytest.mark.gpu
def test_bounds_checked_build_reports_no_out_of_range_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_01522_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, RSX_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build clean" in r.stdout
