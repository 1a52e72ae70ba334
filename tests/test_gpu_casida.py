"""GPU parity for the Tamm-Dancoff Casida path (Eqs. 6-7): the tcgen05 split-BF16
contraction, K, K_d and the FP64 eigen-solve, all through the C ABI.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_01522_gb300 import inputs, rsx
from gpu_util import need_gpu, rel_max_err, to_dev

pytestmark = pytest.mark.gpu

HA_EV = oracle.HARTREE_EV


def bf16_split(S):
    hi = S.to(torch.bfloat16)
    lo = (S - hi.float()).to(torch.bfloat16)
    return hi.contiguous(), lo.contiguous()


@pytest.mark.parametrize("n,ld", [(128, 64), (128, 64 * 37), (384, 64 * 5), (256, 64 * 3001)])
def test_syrk_bf16x3_matches_torch(n, ld):
    """C = H H^T + H L^T + L H^T against the same products in FP64 by PyTorch."""
    need_gpu()
    g = torch.Generator(device="cuda").manual_seed(n + ld)
    S = torch.randn((n, ld), device="cuda", generator=g)
    hi, lo = bf16_split(S)
    ctx = rsx.Context((16, 16, 16), 0.4, "fp32")
    C = ctx.syrk_bf16x3(hi.view(torch.int16), lo.view(torch.int16))
    ctx.sync()
    H, L = hi.double(), lo.double()
    ref = H @ H.T + H @ L.T + L @ H.T
    # FP32 accumulation over ld / splits terms per partial: error ~ eps32 * sqrt(terms) * |row|^2
    err = (C - ref).abs().max().item() / ref.abs().max().item()
    assert err < 2e-6, err
    assert torch.equal(C, C.T)


CASES = [((16, 16, 16), 0.5, 2, 3, "fp32"), ((24, 24, 24), 0.45, 2, 5, "fp32"), ((24, 24, 40), 0.4, 3, 2, "fp32"),
         ((16, 16, 16), 0.5, 2, 3, "fp64"), ((24, 24, 40), 0.4, 2, 3, "fp64")]
# K tolerance (max |gpu - oracle| / max |oracle|): the FP32 path keeps ~16 mantissa bits
# in the bf16 hi + lo split and drops lo * lo (relative 2^-16 per term, unbiased
# rounding); FP64 plain form: round-off only.
TOL_K = {"fp32": 3e-5, "fp64": 1e-11}
TOL_KD = {"fp32": 1e-5, "fp64": 1e-11}


def casida_system(shape, h, no, nv, seed=0):
    return inputs.casida_system(h=h, nocc=no, nvirt=nv, shape=shape, radius=1.5, alpha=(0.5, 2.0), seed=seed)


@pytest.mark.parametrize("shape,h,no,nv,prec", CASES)
def test_casida_K_and_Kd_parity(shape, h, no, nv, prec):
    need_gpu()
    s = casida_system(shape, h, no, nv)
    K_ref = oracle.casida_K(s.phi, s.phi_virt, h)
    Kd_ref = oracle.casida_Kd(s.phi, s.phi_virt, h)
    ctx = rsx.Context(shape, h, prec)
    po, pv = to_dev(s.phi, prec), to_dev(s.phi_virt, prec)
    K = ctx.casida_K(po, pv)
    Kd = ctx.casida_Kd(po, pv)
    ctx.sync()
    K, Kd = K.cpu().numpy(), Kd.cpu().numpy()
    assert rel_max_err(K, K_ref) < TOL_K[prec]
    assert rel_max_err(Kd, Kd_ref) < TOL_KD[prec]
    assert np.array_equal(K, K.T) or prec == "fp64" and np.allclose(K, K.T, rtol=0, atol=0)


@pytest.mark.parametrize("nt_shape,env", [
    ((1, 1), {}), ((2, 3), {}), ((4, 9), {}), ((4, 16), {}), ((8, 64), {}), ((10, 66), {}),
    ((8, 64), {"RSX_EIG_FP64": "1"}), ((10, 66), {"RSX_EIG_FP64": "1"}),
    ((10, 66), {"RSX_TRIDIAG_PATH": "global"}), ((10, 66), {"RSX_TRIDIAG_PATH": "coop"}),
    ((10, 66), {"RSX_TRIDIAG_PATH": "coop", "RSX_EIG_FP64": "1"}), ((4, 16), {"RSX_TRIDIAG_PATH": "cta"})])
def test_casida_solve_matches_eigh(nt_shape, env, monkeypatch):
    """Device eigen-solve vs numpy eigh on the same matrix, random symmetric K, K_d.
    n >= 96: mixed precision (FP32 reduction and eigenbasis, FP64 Newton corrections and
    Rayleigh-Ritz), else FP64; the reduction on one thread-block cluster with the rows in
    distributed shared memory (default), in global memory, on a cooperative grid or on one
    CTA (forced by RSX_TRIDIAG_PATH); RSX_EIG_FP64 forces the FP64 form."""
    need_gpu()
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    no, nv = nt_shape
    nt = no * nv
    r = np.random.default_rng(nt)
    B = r.standard_normal((nt, nt)) * 0.02
    K = B @ B.T
    Kd = 0.01 * (r.standard_normal((nt, nt)))
    Kd = 0.5 * (Kd + Kd.T)
    eo = np.sort(r.uniform(-0.8, -0.3, no))
    ev = np.sort(r.uniform(-0.1, 0.5, nv))
    ctx = rsx.Context((16, 16, 16), 0.4, "fp64")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    nroots = min(10, nt)
    for dm, use_kd in ((2.0, True), (0.0, True), (1.0, False)):
        w, X = ctx.casida_solve(d(eo), d(ev), d(K), d(Kd) if use_kd else None, dm, nroots, vectors=True)
        ctx.sync()
        A = oracle.tda_matrix(eo, ev, K, Kd if use_kd else None, dm)
        w_ref, _ = oracle.tda_solve(A, nroots)
        assert np.allclose(w.cpu().numpy(), w_ref, rtol=0, atol=1e-12 * max(1.0, np.abs(w_ref).max()))
        Xn = X.cpu().numpy()
        for k in range(nroots):
            assert np.linalg.norm(A @ Xn[k] - w_ref[k] * Xn[k]) < 1e-9
        assert np.allclose(Xn @ Xn.T, np.eye(nroots), atol=1e-8)


def test_casida_ipa_limit_and_one_transition():
    need_gpu()
    ctx = rsx.Context((16, 16, 16), 0.4, "fp64")
    eo = torch.tensor([-0.7, -0.5, -0.35], dtype=torch.float64, device="cuda")
    ev = torch.tensor([-0.05, 0.1, 0.3, 0.45], dtype=torch.float64, device="cuda")
    Z = torch.zeros((12, 12), dtype=torch.float64, device="cuda")
    w = ctx.casida_solve(eo, ev, Z, None, 2.0, 12)
    ctx.sync()
    ipa = np.sort((ev.cpu().numpy()[None, :] - eo.cpu().numpy()[:, None]).ravel())
    assert np.allclose(w.cpu().numpy(), ipa, rtol=0, atol=1e-14)
    # one transition: omega = de + delta_M K - K_d exactly
    s = casida_system((16, 16, 16), 0.5, 1, 1)
    c2 = rsx.Context((16, 16, 16), 0.5, "fp64")
    po, pv = to_dev(s.phi, "fp64"), to_dev(s.phi_virt, "fp64")
    K, Kd = c2.casida_K(po, pv), c2.casida_Kd(po, pv)
    w1 = c2.casida_solve(to_dev(s.eps_occ, "fp64"), to_dev(s.eps_virt, "fp64"), K, Kd, 2.0, 1)
    c2.sync()
    exact = s.eps_virt[0] - s.eps_occ[0] + 2.0 * K.item() - Kd.item()
    assert abs(w1.item() - exact) < 1e-14


def test_config3_full_size_split_bf16_vs_fp64():
    """80^3 at 0.25 bohr, 8 occupied + 64 virtual, 512 transitions: the split-BF16
    tensor-core K against the FP64 plain form, lowest 10 excitation energies to 1e-5 eV;
    sampled K entries against the oracle computed one by one."""
    need_gpu()
    s = inputs.casida_system()
    c32 = rsx.Context(s.shape, s.h, "fp32")
    c64 = rsx.Context(s.shape, s.h, "fp64")
    K32 = c32.casida_K(to_dev(s.phi, "fp32"), to_dev(s.phi_virt, "fp32"))
    K64 = c64.casida_K(to_dev(s.phi, "fp64"), to_dev(s.phi_virt, "fp64"))
    eo, ev = to_dev(s.eps_occ, "fp64"), to_dev(s.eps_virt, "fp64")
    w32 = c64.casida_solve(eo, ev, K32, None, 1.0, 10)
    w64 = c64.casida_solve(eo, ev, K64, None, 1.0, 10)
    c32.sync()
    c64.sync()
    assert np.max(np.abs(w32.cpu().numpy() - w64.cpu().numpy())) * HA_EV < 1e-5
    nv = 64
    K64n = K64.cpu().numpy()
    for (t, u) in ((0, 0), (5, 130), (511, 3)):
        i, a = divmod(t, nv)
        j, b = divmod(u, nv)
        rho_t = s.phi[i] * s.phi_virt[a]
        v_u = oracle.poisson_fft(s.phi[j] * s.phi_virt[b], s.h)
        k_ref = oracle.inner(rho_t, v_u, s.h)
        assert abs(K64n[t, u] - k_ref) <= 1e-10 * abs(K64n).max()


def test_casida_K_multi_tile_vs_oracle():
    """135 transitions (two 128-row tiles of the panel, one of them ragged) at 24^3: the
    split-BF16 tensor-core K element-wise against the FP64 oracle, over ~1800 K blocks of
    the split-K contraction; the FP64 plain form against the same oracle."""
    need_gpu()
    shape, h, no, nv = (24, 24, 24), 0.45, 3, 45
    s = casida_system(shape, h, no, nv, seed=4)
    K_ref = oracle.casida_K(s.phi, s.phi_virt, h)
    for prec in ("fp32", "fp64"):
        ctx = rsx.Context(shape, h, prec)
        K = ctx.casida_K(to_dev(s.phi, prec), to_dev(s.phi_virt, prec))
        ctx.sync()
        K = K.cpu().numpy()
        assert K.shape == (135, 135)
        assert rel_max_err(K, K_ref) < TOL_K[prec], prec
        # the off-diagonal tile block (rows 128.., columns ..127) on its own
        assert np.max(np.abs(K[128:, :128] - K_ref[128:, :128])) < TOL_K[prec] * np.abs(K_ref).max()
        ctx.close()


def test_config3_against_the_oracle_golden():
    """80^3 at 0.25 bohr, 8 occupied + 64 virtual (512 transitions): the split-BF16 K and
    the FP64 plain K against the FP64 oracle's values in tests/golden/casida_80cubed.json
    (written by make_casida_golden.py from the oracle alone): the diagonal, the row sums and
    4096 sampled entries of K, 512 sampled entries of K_d, and the lowest 10 roots of
    diag + K and of the singlet diag + 2K - K_d to 1e-5 eV."""
    import json
    import os
    need_gpu()
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "casida_80cubed.json")))
    c = gold["case"]
    s = inputs.casida_system(n=c["n"], h=c["h"], nocc=c["nocc"], nvirt=c["nvirt"], seed=c["seed"])
    kmax = gold["K_max_abs"]
    samp = np.array(gold["K_samples"])
    ti, ui = samp[:, 0].astype(int), samp[:, 1].astype(int)
    dsamp = np.array(gold["Kd_samples"])
    eo, ev = to_dev(s.eps_occ, "fp64"), to_dev(s.eps_virt, "fp64")
    c64 = rsx.Context(s.shape, s.h, "fp64")
    for prec, tol in (("fp32", TOL_K["fp32"]), ("fp64", 1e-10)):
        ctx = rsx.Context(s.shape, s.h, prec)
        po, pv = to_dev(s.phi, prec), to_dev(s.phi_virt, prec)
        K = ctx.casida_K(po, pv)
        Kd = ctx.casida_Kd(po, pv)
        ctx.sync()
        Kn = K.cpu().numpy()
        assert np.max(np.abs(np.diag(Kn) - np.array(gold["K_diag"]))) < tol * kmax, prec
        assert np.max(np.abs(Kn[ti, ui] - samp[:, 2])) < tol * kmax, prec
        # row sums: 512 terms each, the per-entry bound times sqrt(512) (unbiased rounding)
        assert np.max(np.abs(Kn.sum(axis=1) - np.array(gold["K_row_sums"]))) < tol * kmax * 512 ** 0.5, prec
        Kdn = Kd.cpu().numpy()
        kd_tol = TOL_KD[prec] if prec == "fp32" else 1e-10
        assert np.max(np.abs(Kdn[dsamp[:, 0].astype(int), dsamp[:, 1].astype(int)] - dsamp[:, 2])) \
            < kd_tol * gold["Kd_max_abs"], prec
        w1 = c64.casida_solve(eo, ev, K, None, 1.0, 10)
        w2 = c64.casida_solve(eo, ev, K, Kd, 2.0, 10)
        c64.sync()
        assert np.max(np.abs(w1.cpu().numpy() - np.array(gold["omega_diag_plus_K_ha"]))) * HA_EV < 1e-5, prec
        assert np.max(np.abs(w2.cpu().numpy() - np.array(gold["omega_singlet_ha"]))) * HA_EV < 1e-5, prec
        ctx.close()
