"""Off-centre-charge sphere refinement study (Sec. "Mesh refinement study
using an analytical solution"): radius 4 A, unit charge at (1, 1, 1),
eps 4 / 80, kappa 0.125 1/A, octahedral sphere meshes of 512, 2,048 and
8,192 elements with the 6-point rule.  The GPU solvation energies match the
dense oracle on the smallest mesh and approach Kirkwood's analytic value
(tests/golden/kirkwood_sphere.json) at first order in 1/N.
"""
import json
import os

import numpy as np
import pytest

import synthetic
from oracle import bem, closed_forms as cf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def golden():
    return json.load(open(os.path.join(HERE, "golden", "kirkwood_sphere.json")))


@pytest.fixture(scope="module")
def energies(golden):
    import paper_2103_01048_gb300 as pb
    ctx = pb.pb_create(0, None)
    out = {}
    try:
        for lev in (3, 4, 5):
            V, F = synthetic.octasphere(lev, golden["radius"])
            m = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 6, 8, 64)
            try:
                res, st = pb.pb_solve(ctx, m, np.array([golden["position"]]), np.array([golden["q"]]),
                                      golden["eps_in"], golden["eps_out"], golden["kappa"], 1e-7, 500)
                assert st == pb.PB_OK
                out[lev] = pb.pb_solvation_energy(ctx, res)
                pb.pb_result_destroy(res)
            finally:
                pb.pb_mesh_destroy(m)
    finally:
        pb.pb_destroy(ctx)
    return out


def test_smallest_mesh_matches_oracle(golden, energies):
    V, F = synthetic.octasphere(3, golden["radius"])
    E_ref, *_ = bem.solve_energy(V, F, 6, np.array([golden["position"]]), np.array([golden["q"]]),
                                 golden["eps_in"], golden["eps_out"], golden["kappa"])
    assert abs(energies[3] - E_ref) / abs(E_ref) < 1e-4


def test_first_order_convergence_to_kirkwood(golden, energies):
    E_k = cf.kirkwood_energy([golden["q"]], [golden["position"]], golden["radius"], golden["eps_in"],
                             golden["eps_out"], golden["kappa"])
    err = [abs(energies[lev] - E_k) / abs(E_k) for lev in (3, 4, 5)]
    assert err[0] > err[1] > err[2]
    # N grows 4x per level: order 1 in 1/N means the error falls ~4x per level
    orders = [np.log(err[i] / err[i + 1]) / np.log(4.0) for i in range(2)]
    assert all(0.85 < o < 1.15 for o in orders), orders
    assert err[2] < 1e-3
