"""Writes scf_16cubed.json: the converged closed-shell HF SCF of the oracle (FP64, dense
diagonalisation, Sec. 3.1-3.2) with ACE and with exact exchange on a 16^3 box, the
expected values of the GPU SCF tests.  Calls only the oracle and the seeded inputs.

    python tests/golden/make_scf_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.scf as oscf  # noqa: E402
from paper_2405_01522_gb300 import inputs  # noqa: E402

CASE = {"n": 16, "h": 0.5, "natoms": 2, "Z": 2.0, "rc": 0.8, "radius": 1.0, "seed": 3, "nocc": 2, "alpha": 0.3}


def main():
    c = CASE
    v = inputs.model_potential(n=c["n"], h=c["h"], natoms=c["natoms"], Z=c["Z"], rc=c["rc"], radius=c["radius"],
                               seed=c["seed"])
    out = {"case": c, "tol": 1e-10}
    for mode in ("ace", "exact"):
        r = oscf.scf(v, c["h"], c["nocc"], mode=mode, alpha=c["alpha"], tol=out["tol"])
        out[mode] = {k: (float(r[k]) if k != "eps_orb" else [float(x) for x in r[k]])
                     for k in ("energy", "one_body", "hartree", "exchange", "reldens", "eps_orb")}
        out[mode]["iters"] = int(r["iters"])
        print(mode, out[mode], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "scf_16cubed.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
