"""Writes born_ion_5120.json: the dense-LU oracle's polar solvation energy
of the Born ion on the 5,120-triangle icosphere (radius 2 A, +1 e at the
centre, eps 4 / 80, kappa 0.125 1/A, 3-point rule, P0, Eq. direct), the
reference the benchmark's mixed and all-FP64 GPU solves are measured
against.  Calls only oracle/ (and the seeded mesh generator); run from the
repository root:  python tests/golden/make_born_ion.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402
from oracle import bem, closed_forms  # noqa: E402


def main():
    V, F = synthetic.icosphere(4, 2.0)
    eps_in, eps_out, kappa = 4.0, 80.0, 0.125
    t0 = time.time()
    e, *_ = bem.solve_energy(V, F, 3, np.zeros((1, 3)), np.array([1.0]), eps_in, eps_out, kappa)
    out = {"what": "dense-LU oracle dG of Eq. direct (P0, 3-point rule) for the Born ion",
           "mesh": "synthetic.icosphere(4, 2.0): 5120 triangles, radius 2 A", "charge": 1.0,
           "position": [0.0, 0.0, 0.0], "eps_in": eps_in, "eps_out": eps_out, "kappa": kappa, "nquad": 3,
           "energy_kcal_mol": e,
           "born_closed_form_kcal_mol": closed_forms.born_energy(1.0, 2.0, eps_in, eps_out, kappa),
           "oracle_seconds": round(time.time() - t0, 1),
           "script": "tests/golden/make_born_ion.py"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "born_ion_5120.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
