"""Batched binding energies against the oracle (Eq. bind).

Three small synthetic receptor-ligand complexes (20/5, 30/6 and 40/8 atoms;
complex, receptor and ligand surfaces of 1,300-7,800 triangles) with the
paper's binding parameters (eps_in 1, eps_out 80, kappa 0.10265 1/A): the nine
meshes solved together by pb_solve_batch (mixed precision, tol 1e-8), each
solvation energy against the oracle's matrix-free FP64 GMRES value and the
binding energies against the oracle's (tests/golden/binding_small.json,
written by tests/golden/make_binding.py).  Solvation energies within the 1e-4
target; a binding energy is a small difference of large solvation energies,
so its bound is 1e-4 of the largest of them.
"""
import json
import os

import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "binding_small.json")


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.mark.skipif(not os.path.exists(GOLD), reason="golden binding energies not written")
def test_batched_binding_energies_vs_oracle(pb):
    gold = json.load(open(GOLD))
    eps = (gold["eps_in"], gold["eps_out"], gold["kappa"])
    ctx = pb.pb_create(0, None)
    meshes, atoms, charges = [], [], []
    try:
        cxs = []
        for c in gold["complexes"]:
            cx = synthetic.binding_complex(c["n_rec"], c["n_lig"], seed=10 + c["n_rec"], spacing=1.0)
            cxs.append(cx)
            for k in ("cplx", "rec", "lig"):
                V, T = cx["surf"][k]
                assert len(T) == c[k]["triangles"]
                meshes.append(pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 6, 64))
                atoms.append(cx[k][0])
                charges.append(cx[k][2])
        res, st, rc = pb.pb_solve_batch(ctx, meshes, atoms, charges, *eps, 1e-8, 500)
        assert rc == pb.PB_OK
        es = []
        for r in res:
            es.append(pb.pb_solvation_energy(ctx, r))
            pb.pb_result_destroy(r)
    finally:
        for m in meshes:
            pb.pb_mesh_destroy(m)
        pb.pb_destroy(ctx)
    for ci, c in enumerate(gold["complexes"]):
        e3 = es[3 * ci: 3 * ci + 3]
        ref3 = [c[k]["dG_kcal_mol"] for k in ("cplx", "rec", "lig")]
        for e, ref in zip(e3, ref3):
            assert abs(e - ref) < 1e-4 * abs(ref), (ci, e, ref)
        bind = e3[0] - e3[1] - e3[2] - c["dG_coul_kcal_mol"]
        print(f"complex {ci}: dG_bind {bind:.6f} oracle {c['dG_bind_kcal_mol']:.6f} kcal/mol")
        assert abs(bind - c["dG_bind_kcal_mol"]) < 1e-4 * max(abs(r) for r in ref3)
