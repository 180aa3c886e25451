"""GPU adjoint gradients vs the oracle: dE/dq against 1/2 (R + R^T) q from
the dense matrices, dE/dx against central differences of the dense-LU
energy (surface fixed); mixed and FP64 paths; and the torch.autograd
wrapper against the C-ABI gradients."""
import numpy as np
import pytest

import synthetic
from oracle import bem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = (4.0, 80.0, 0.125)


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def ctx(pb):
    c = pb.pb_create(0, None)
    yield c
    pb.pb_destroy(c)


@pytest.fixture(scope="module")
def system():
    V, F = synthetic.icosphere(3, 3.0)
    mats = bem.assemble_p0(V, F, 3, EPS[2])
    atoms = np.array([[0.5, -0.3, 0.2], [-0.8, 0.4, 0.6], [0.1, 0.9, -0.7], [1.2, 0.2, -0.4]])
    q = np.array([0.6, -0.5, 0.3, -0.4])
    gq = bem.energy_grad_q(V, F, 3, atoms, q, *EPS, mats)
    gx = bem.energy_grad_x_fd(V, F, 3, atoms, q, *EPS, mats, h=1e-4)
    return V, F, atoms, q, gq, gx


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_gradients_vs_oracle(pb, ctx, system, precision):
    V, F, atoms, q, gq_ref, gx_ref = system
    prec = pb.PB_MIXED if precision == "mixed" else pb.PB_FP64
    mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6 if precision == "mixed" else 8, 64)
    try:
        res, st = pb.pb_solve(ctx, mesh, atoms, q, *EPS, 1e-9, 400, precision=prec)
        assert st == pb.PB_OK
        gq, gx, st2 = pb.pb_energy_grad(ctx, res, len(q), tol=1e-9, max_iter=400)
        assert st2 == pb.PB_OK
        pb.pb_result_destroy(res)
    finally:
        pb.pb_mesh_destroy(mesh)
    assert np.abs(gq - gq_ref).max() < 1e-4 * np.abs(gq_ref).max()
    gxr = np.array([[gx_ref[(k, c)] for c in range(3)] for k in range(len(q))])
    assert np.abs(gx - gxr).max() < 1e-3 * np.abs(gxr).max()


def test_autograd_function(pb, ctx, system):
    from paper_2103_01048_gb300.autograd import solvation_energy
    V, F, atoms, q, gq_ref, _ = system
    mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6, 64)
    try:
        qt = torch.tensor(q, dtype=torch.float64, requires_grad=True)
        xt = torch.tensor(atoms, dtype=torch.float64, requires_grad=True)
        e = solvation_energy(qt, xt, ctx, mesh, *EPS, tol=1e-9)
        e.backward()
        res, _ = pb.pb_solve(ctx, mesh, atoms, q, *EPS, 1e-9, 400)
        gq, gx, _ = pb.pb_energy_grad(ctx, res, len(q), tol=1e-9)
        e2 = pb.pb_solvation_energy(ctx, res)
        pb.pb_result_destroy(res)
    finally:
        pb.pb_mesh_destroy(mesh)
    assert abs(float(e.detach()) - e2) < 1e-6 * abs(e2)
    assert np.allclose(qt.grad.numpy(), gq, rtol=1e-5, atol=1e-9)
    assert np.allclose(xt.grad.numpy(), gx, rtol=1e-5, atol=1e-9)
    assert np.abs(qt.grad.numpy() - gq_ref).max() < 1e-4 * np.abs(gq_ref).max()
