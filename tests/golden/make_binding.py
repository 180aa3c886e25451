"""Writes binding_small.json: polar binding energies (Eq. bind) of three
small synthetic receptor-ligand complexes, every solvation energy by the
oracle's matrix-free FP64 GMRES (direct point sums, exact singular
corrections, relative residual 1e-10) on the complex, receptor and ligand
surfaces, with the paper's binding parameters (eps_in 1, eps_out 80,
kappa 0.10265 1/A; Sec. "Binding energy calculations").  The reference of the
batched GPU solve's binding energies.  Calls only oracle/ (and the seeded
generators); run from the repository root:
    python tests/golden/make_binding.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402
from oracle import bem  # noqa: E402
from oracle.closed_forms import KCAL  # noqa: E402

EPS_IN, EPS_OUT, KAPPA = 1.0, 80.0, 0.10265
CASES = [(20, 5), (30, 6), (40, 8)]          # (receptor atoms, ligand atoms)
SPACING = 1.0


def mesh_hash(V, T):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(V, np.float64).tobytes())
    h.update(np.ascontiguousarray(T, np.int32).tobytes())
    return h.hexdigest()[:16]


def main():
    out = {"what": "polar binding energies (Eq. bind) of small synthetic complexes, oracle matrix-free GMRES",
           "eps_in": EPS_IN, "eps_out": EPS_OUT, "kappa": KAPPA, "nquad": 3, "tol": 1e-10,
           "generator": "synthetic.binding_complex(n_rec, n_lig, seed=10 + n_rec, spacing=1.0)",
           "script": "tests/golden/make_binding.py", "complexes": []}
    for n_rec, n_lig in CASES:
        cx = synthetic.binding_complex(n_rec, n_lig, seed=10 + n_rec, spacing=SPACING)
        rec = {"n_rec": n_rec, "n_lig": n_lig}
        for k in ("cplx", "rec", "lig"):
            V, T = cx["surf"][k]
            xyz, _, q = cx[k]
            t0 = time.time()
            e, _, _, it, res = bem.solve_energy_free(V, T, 3, xyz, q, EPS_IN, EPS_OUT, KAPPA, tol=1e-10)
            rec[k] = {"triangles": int(len(T)), "mesh_sha256_16": mesh_hash(V, T), "dG_kcal_mol": e,
                      "iterations": it, "residual": res, "seconds": round(time.time() - t0, 1)}
            print(n_rec, k, len(T), e, it, res, round(time.time() - t0, 1), flush=True)
        xr, xl = cx["rec"][0], cx["lig"][0]
        r = np.linalg.norm(xr[:, None, :] - xl[None, :, :], axis=2)
        coul = KCAL * (cx["rec"][2][:, None] * cx["lig"][2][None, :] / (EPS_IN * r)).sum()
        rec["dG_coul_kcal_mol"] = coul
        rec["dG_bind_kcal_mol"] = rec["cplx"]["dG_kcal_mol"] - rec["rec"]["dG_kcal_mol"] - \
            rec["lig"]["dG_kcal_mol"] - coul
        out["complexes"].append(rec)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "binding_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
