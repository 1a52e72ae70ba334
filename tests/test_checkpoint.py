"""Checkpoint files (paper_2405_01522_gb300.checkpoint): CPU round trips and rejection of
damaged files; on the GPU, resuming the SCF from saved orbitals and the network from
saved parameters."""
import os
import struct

import numpy as np
import pytest
import torch

from paper_2405_01522_gb300 import checkpoint, inputs


def test_round_trip_of_every_dtype_and_shape(tmp_path):
    r = np.random.default_rng(0)
    arrays = {"orb": r.standard_normal((3, 4, 5, 6)).astype(np.float32), "K": r.standard_normal((7, 7)),
              "idx": np.arange(-5, 5, dtype=np.int32), "step": np.array([2 ** 40], dtype=np.int64),
              "empty": np.zeros((0, 3), dtype=np.float64), "scalar": np.array(3.5)}
    bf = torch.randn(5, 3).to(torch.bfloat16)
    p = str(tmp_path / "c.rsx")
    checkpoint.save(p, bf=bf, **arrays)
    back = checkpoint.load(p)
    assert list(back) == ["bf"] + list(arrays)
    for k, v in arrays.items():
        assert back[k].dtype == v.dtype.newbyteorder("<") and back[k].shape == v.shape
        assert np.array_equal(back[k], v)
    t = checkpoint.load(p, device="cpu")
    assert t["bf"].dtype == torch.bfloat16 and torch.equal(t["bf"], bf)


def test_big_endian_input_is_stored_little_endian(tmp_path):
    a = np.arange(6, dtype=">f8").reshape(2, 3)
    p = str(tmp_path / "be.rsx")
    checkpoint.save(p, a=a)
    raw = open(p, "rb").read()
    assert raw[-48:] == np.arange(6, dtype="<f8").tobytes()
    assert np.array_equal(checkpoint.load(p)["a"], a)


def test_damaged_files_are_rejected(tmp_path):
    p = str(tmp_path / "d.rsx")
    checkpoint.save(p, a=np.ones((4, 4), dtype=np.float32))
    raw = open(p, "rb").read()
    for bad in (raw[:-3], b"XXXX" + raw[4:], raw[:4] + struct.pack("<I", 9) + raw[8:]):
        q = str(tmp_path / "bad.rsx")
        open(q, "wb").write(bad)
        with pytest.raises(ValueError):
            checkpoint.load(q)
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "u.rsx"), a=np.ones(3, dtype=np.complex64))


@pytest.mark.gpu
def test_scf_and_network_resume_from_checkpoints(tmp_path):
    """SCF: 8 iterations, save the orbitals, start a new SCF from the saved file -- it
    reaches the uninterrupted run's ground-state energy in fewer iterations than that run
    took from the start.  Network: parameters saved after a few Adam steps reload into a
    fresh network with bit-identical outputs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_01522_gb300 import precond, rsx
    n, h, nocc, radius = 16, 0.4, 2, 1.0
    v = torch.from_numpy(inputs.model_potential(n=n, h=h, natoms=2, Z=2.0, rc=0.8, radius=radius, seed=3)).float().cuda()
    psi0 = torch.from_numpy(inputs.starting_orbitals(n=n, h=h, nband=nocc, radius=radius, seed=5)).float().cuda()
    ctx = rsx.Context((n, n, n), h, "fp32")

    def run(start, iters):
        s = rsx.SCF(ctx, v, nocc, ace=True, alpha=0.3)
        s.init(start)
        hist = []
        for _ in range(iters):
            hist.append(s.step(inner=2))
            if len(hist) > 1 and 0 < hist[-1]["reldens"] < 2e-6:
                break
        return s, hist

    ref, full = run(psi0, 120)
    assert full[-1]["reldens"] < 2e-6
    a, _ = run(psi0, 8)
    p = str(tmp_path / "gs.rsx")
    checkpoint.save_ground_state(p, a.orbitals(), h)
    rec = checkpoint.load(p, device="cuda")
    assert float(rec["h"][0]) == h and torch.equal(rec["orbitals"], a.orbitals())
    b, rest = run(rec["orbitals"].contiguous(), 120)
    assert rest[-1]["reldens"] < 2e-6 and len(rest) < len(full)
    assert abs(rest[-1]["energy"] - full[-1]["energy"]) < 1e-5 * abs(full[-1]["energy"])
    for s in (ref, a, b):
        s.close()
    net = rsx.Net(precond.init_params(seed=1))
    x = torch.randn(2, 2, 12, 12, 12, device="cuda")
    y = torch.randn(2, 12, 12, 12, device="cuda") * 0.01
    for _ in range(3):
        net.train_step(x, y, 1e-3, border=2)
    q = str(tmp_path / "net.rsx")
    checkpoint.save_network(q, net, step=3)
    net2 = rsx.Net(precond.init_params(seed=2))
    assert int(checkpoint.load_network(q, net2)["step"][0]) == 3
    assert torch.equal(net.forward(x), net2.forward(x))
    net.close()
    net2.close()
