"""Writes casida_80cubed.json: the FP64 oracle's Tamm-Dancoff coupling for the 80^3 case
(h = 0.25 bohr padded to 160^3, 8 occupied + 64 virtual orthonormal Gaussian-sum
orbitals, 512 transitions; Eqs. 6-7), the expected values of the full-size GPU Casida
test.  Calls only the oracle and the seeded inputs.

Stored (a text fixture, not the whole 512 x 512 matrix):
  * the lowest 10 roots of diag(eps_a - eps_i) + K (the TDA form with the coupling alone)
    and of the RHF singlet diag + 2K - K_d (Eq. 7), in Hartree;
  * K on its diagonal, its row sums, and 4096 entries at seeded random positions;
  * K_d at 512 seeded random positions;
  * max |K|, for the relative tolerances.

    python tests/golden/make_casida_golden.py
"""
import functools
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2405_01522_gb300 import inputs  # noqa: E402

CASE = {"n": 80, "h": 0.25, "nocc": 8, "nvirt": 64, "seed": 0, "nsample_K": 4096, "nsample_Kd": 512,
        "sample_seed": 2405}


def main():
    c = CASE
    t0 = time.time()
    s = inputs.casida_system(n=c["n"], h=c["h"], nocc=c["nocc"], nvirt=c["nvirt"], seed=c["seed"])
    ghat = oracle.kernel_spectrum(tuple(2 * x for x in s.shape), s.h)
    poisson = functools.partial(oracle.poisson_fft, ghat=ghat)     # the kernel spectrum computed once
    K = oracle.casida_K(s.phi, s.phi_virt, s.h, poisson=poisson)
    print(f"K done {time.time() - t0:.0f} s", flush=True)
    Kd = oracle.casida_Kd(s.phi, s.phi_virt, s.h, poisson=poisson)
    print(f"K_d done {time.time() - t0:.0f} s", flush=True)
    nt = K.shape[0]
    w_k, _ = oracle.tda_solve(oracle.tda_matrix(s.eps_occ, s.eps_virt, K, None, delta_M=1.0), 10)
    w_s, _ = oracle.tda_solve(oracle.tda_matrix(s.eps_occ, s.eps_virt, K, Kd, delta_M=2.0), 10)
    rng = np.random.default_rng(c["sample_seed"])
    idx = rng.integers(0, nt, size=(c["nsample_K"], 2))
    idd = rng.integers(0, nt, size=(c["nsample_Kd"], 2))
    out = {
        "_doc": "FP64 oracle values (oracle.casida_K / casida_Kd / tda_solve) for the 80^3 Casida case; "
                "written by tests/golden/make_casida_golden.py, which calls only the oracle and the seeded inputs. "
                "K_{ia,jb} = (ia|jb) and K_d = (ab|ji) of Eqs. 6-7 (Sec. 2), transition t = i * nvirt + a.",
        "case": c,
        "omega_diag_plus_K_ha": [float(x) for x in w_k],
        "omega_singlet_ha": [float(x) for x in w_s],
        "K_max_abs": float(np.abs(K).max()),
        "K_diag": [float(x) for x in np.diag(K)],
        "K_row_sums": [float(x) for x in K.sum(axis=1)],
        "K_samples": [[int(t), int(u), float(K[t, u])] for t, u in idx],
        "Kd_max_abs": float(np.abs(Kd).max()),
        "Kd_samples": [[int(t), int(u), float(Kd[t, u])] for t, u in idd],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "casida_80cubed.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(f"written in {time.time() - t0:.0f} s; omega (diag + K) = {w_k}", flush=True)


if __name__ == "__main__":
    main()
