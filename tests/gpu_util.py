"""Helpers for the GPU parity tests (inputs to device, tolerance checks)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(a, precision):
    dt = torch.float32 if precision == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def rel_max_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


# Element-wise tolerance (max |gpu - oracle| / max |oracle|).  FP32: the FFT passes
# round each of ~2 log2(M) butterfly levels and the pair product in single precision
# (unit roundoff 6e-8); 1e-5 leaves a margin of ~10x over the observed error growth.
# FP64: same algorithm in double precision against the FP64 oracle.
TOL = {"fp32": 1e-5, "fp64": 1e-11}
# Exchange energies <psi, Vx psi> and E_x: 1e-6 relative for FP32 (stated target).
TOL_ENERGY = {"fp32": 1e-6, "fp64": 1e-12}
