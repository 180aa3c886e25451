"""The synthetic-protein configuration: 2,000 atoms (jittered FCC in a 20 A
ball, radii U[1.2, 2], charges U[-0.8, 0.8] with zero net charge) inside the
~80,000-triangle Gaussian surface, mixed-precision FMM with FP64 GMRES.

No dense oracle fits this size; checks: convergence, the energy at p = 6
against p = 8 (the FMM's own convergence), dE/dq against central differences
in q (the energy is quadratic in q, so the difference is exact up to the
solve's noise) and dE/dx against central differences in the positions with
the surface held fixed (h = 1e-2 A: the FP32 FMM's run-to-run noise swamps
differences at h = 1e-4)."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = (4.0, 80.0, 0.125)


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def protein():
    V, T, xyz, radii, q, h = synthetic.synthetic_protein()
    assert 72000 <= len(T) <= 88000
    return V, T, xyz, q


def test_protein_solve_and_gradients(pb, protein):
    V, T, xyz, q = protein
    ctx = pb.pb_create(0, None)
    m6 = pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 6, 128)
    m8 = pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 8, 128)
    try:
        def energy(mesh, x, qq, tol=1e-8):
            res, st = pb.pb_solve(ctx, mesh, x, qq, *EPS, tol, 1000)
            assert st == pb.PB_OK
            e = pb.pb_solvation_energy(ctx, res)
            return e, res

        e6, res = energy(m6, xyz, q, 1e-5)
        it6, rr6, _ = pb.pb_result_get(res)
        pb.pb_result_destroy(res)
        e8, res8 = energy(m8, xyz, q, 1e-5)
        pb.pb_result_destroy(res8)
        assert np.isfinite(e6) and e6 < 0 and it6 > 0 and rr6 <= 1e-5
        assert abs(e6 - e8) / abs(e8) < 1e-4
        # gradients at a tight tolerance
        e, res = energy(m6, xyz, q)
        gq, gx, st = pb.pb_energy_grad(ctx, res, len(q), tol=1e-8, max_iter=1000)
        pb.pb_result_destroy(res)
        assert st == pb.PB_OK and gq.shape == (2000,) and gx.shape == (2000, 3)
        rng = np.random.default_rng(7)
        ks = rng.choice(len(q), 5, replace=False)
        hq = 0.05
        for k in ks:
            qp, qm = q.copy(), q.copy()
            qp[k] += hq
            qm[k] -= hq
            fd = (energy(m6, xyz, qp)[0] - energy(m6, xyz, qm)[0]) / (2 * hq)
            assert abs(fd - gq[k]) < 1e-3 * np.abs(gq).max(), (k, fd, gq[k])
        hx = 1e-2
        comps = [(int(k), int(c)) for k, c in zip(rng.choice(len(q), 5, replace=False), rng.integers(0, 3, 5))]
        for k, c in comps:
            xp, xm = xyz.copy(), xyz.copy()
            xp[k, c] += hx
            xm[k, c] -= hx
            fd = (energy(m6, xp, q)[0] - energy(m6, xm, q)[0]) / (2 * hx)
            assert abs(fd - gx[k, c]) < 1e-2 * np.abs(gx).max(), (k, c, fd, gx[k, c])
    finally:
        pb.pb_mesh_destroy(m6)
        pb.pb_mesh_destroy(m8)
        pb.pb_destroy(ctx)
