"""A non-spherical surface against the dense-LU oracle.

The geometry of the protein-like configurations: the Gaussian-density
isosurface of 24 atoms (jittered FCC, radii U[1.2, 2], charges U[-0.8, 0.8]
with zero net charge), marching tetrahedra at 1.1 A spacing, ~4,000
triangles (3-point rule, P0).  The oracle assembles the four Galerkin
matrices densely and solves Eq. direct by LU; the GPU solves by FMM-GMRES.
Checks: the energy (Eq. energy) within the 1e-4 relative target for mixed
and FP64 arithmetic, in deterministic mode and in a batched solve; the
reaction potential at every atom; dE/dq against 1/2 (R + R^T) q from the
oracle's charge-response matrix.
"""
import numpy as np
import pytest

import synthetic
from oracle import bem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = (4.0, 80.0, 0.125)
TOL_E = 1e-4


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
    xyz, radii, q = synthetic.fcc_ball_atoms(24, 6.5, 2.85, 0.1, seed=4)
    V, T = synthetic.gaussian_surface(xyz, radii, 1.1)
    assert 3500 <= len(T) <= 4500
    mats = bem.assemble_p0(V, T, 3, EPS[2])
    e, phi, dphi, _ = bem.solve_energy(V, T, 3, xyz, q, *EPS, mats=mats)
    phir = bem.phi_reac(V, T, 3, phi, dphi, xyz)
    gq = bem.energy_grad_q(V, T, 3, xyz, q, *EPS, mats)
    return V, T.astype(np.int32), xyz, q, e, phir, gq


@pytest.mark.parametrize("prec,p", [("mixed", 6), ("fp64", 6), ("fp64", 8)])
def test_gaussian_surface_energy(pb, ctx, system, prec, p):
    V, T, xyz, q, e_ref, phir_ref, _ = system
    mesh = pb.pb_mesh_setup(ctx, V, T, 3, p, 64)
    try:
        res, st = pb.pb_solve(ctx, mesh, xyz, q, *EPS, 1e-8, 500,
                              precision=pb.PB_FP64 if prec == "fp64" else pb.PB_MIXED)
        assert st == pb.PB_OK
        e, phir = pb.pb_solvation_energy(ctx, res, len(q))
        pb.pb_result_destroy(res)
    finally:
        pb.pb_mesh_destroy(mesh)
    print(f"gaussian surface {prec} p={p}: dG {e:.8f} oracle {e_ref:.8f} rel {abs(e - e_ref) / abs(e_ref):.2e}")
    assert abs(e - e_ref) < TOL_E * abs(e_ref)
    assert np.abs(phir - phir_ref).max() < 2e-4 * np.abs(phir_ref).max()


def test_gaussian_surface_deterministic(pb, ctx, system):
    V, T, xyz, q, e_ref, _, _ = system
    pb.pb_set_option(ctx, pb.PB_OPT_DETERMINISTIC, 1)
    mesh = pb.pb_mesh_setup(ctx, V, T, 3, 6, 64)
    try:
        es = []
        for _ in range(2):
            res, st = pb.pb_solve(ctx, mesh, xyz, q, *EPS, 1e-8, 500)
            assert st == pb.PB_OK
            es.append(pb.pb_solvation_energy(ctx, res))
            pb.pb_result_destroy(res)
    finally:
        pb.pb_mesh_destroy(mesh)
        pb.pb_set_option(ctx, pb.PB_OPT_DETERMINISTIC, 0)
    assert es[0] == es[1]
    assert abs(es[0] - e_ref) < TOL_E * abs(e_ref)


def test_gaussian_surface_gradient_q(pb, ctx, system):
    V, T, xyz, q, _, _, gq_ref = system
    mesh = pb.pb_mesh_setup(ctx, V, T, 3, 6, 64)
    try:
        res, _ = pb.pb_solve(ctx, mesh, xyz, q, *EPS, 1e-9, 500)
        gq, gx, st = pb.pb_energy_grad(ctx, res, len(q), tol=1e-9)
        pb.pb_result_destroy(res)
    finally:
        pb.pb_mesh_destroy(mesh)
    assert st == pb.PB_OK
    assert np.abs(gq - gq_ref).max() < 1e-4 * np.abs(gq_ref).max()


def test_batch_against_oracle(pb, ctx, system):
    """pb_solve_batch on three systems of different size (the Gaussian
    surface, a Born ion, an off-centre charge in a coarse sphere), each
    energy against its own dense-LU oracle solve."""
    V, T, xyz, q, e_ref, _, _ = system
    Vb, Fb = synthetic.icosphere(3, 2.0)
    Vk, Fk = synthetic.octasphere(3, 4.0)
    sys = [(V, T, xyz, q, e_ref),
           (Vb, Fb.astype(np.int32), np.zeros((1, 3)), np.array([1.0]), None),
           (Vk, Fk.astype(np.int32), np.array([[1.0, 1.0, 1.0]]), np.array([1.0]), None)]
    refs = []
    for Vs, Ts, a, c, er in sys:
        if er is None:
            er, *_ = bem.solve_energy(Vs, Ts, 3, a, c, *EPS)
        refs.append(er)
    meshes = [pb.pb_mesh_setup(ctx, Vs, Ts, 3, 6, 64) for Vs, Ts, *_ in sys]
    try:
        res, st, rc = pb.pb_solve_batch(ctx, meshes, [s[2] for s in sys], [s[3] for s in sys], *EPS, 1e-8, 500)
        assert rc == pb.PB_OK and all(s == pb.PB_OK for s in st)
        for r, er in zip(res, refs):
            e = pb.pb_solvation_energy(ctx, r)
            pb.pb_result_destroy(r)
            assert abs(e - er) < TOL_E * abs(er), (e, er)
    finally:
        for m in meshes:
            pb.pb_mesh_destroy(m)
