"""Batched solves (one stream and one captured mat-vec graph per system,
lockstep GMRES) against one-at-a-time pb_solve, and the ncrit autotuner."""
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


def systems():
    out = []
    V, F = synthetic.icosphere(3, 2.0)
    out.append((V, F, np.zeros((1, 3)), np.array([1.0])))
    V, F = synthetic.icosphere(2, 3.0)
    out.append((V, F, np.array([[0.5, 0.2, -0.3], [-0.7, 0.1, 0.4], [0.0, -0.8, 0.2]]), np.array([0.5, -0.6, 0.1])))
    xyz, r, q = synthetic.fcc_ball_atoms(20, 5.5, 2.85, 0.1, seed=5)
    V, F = synthetic.gaussian_surface(xyz, r, 0.45)
    out.append((V, F, xyz, q))
    V, F = synthetic.icosphere(4, 4.0)
    out.append((V, F, np.array([[1.0, 1.0, 1.0]]), np.array([1.0])))
    return out


def test_batch_matches_single_solves(pb):
    ctx = pb.pb_create(0, None)
    sysl = systems()
    meshes = [pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6, 64) for V, F, _, _ in sysl]
    try:
        single = []
        for m, (_, _, a, q) in zip(meshes, sysl):
            res, st = pb.pb_solve(ctx, m, a, q, *EPS, 1e-7, 400)
            assert st == pb.PB_OK
            it, _, _ = pb.pb_result_get(res)
            single.append((pb.pb_solvation_energy(ctx, res), it))
            pb.pb_result_destroy(res)
        for _ in range(2):   # twice: graphs are rebuilt per call
            results, sts, rc = pb.pb_solve_batch(ctx, meshes, [s[2] for s in sysl], [s[3] for s in sysl],
                                                 *EPS, 1e-7, 400)
            assert rc == pb.PB_OK and np.all(sts == pb.PB_OK)
            for res, (e_ref, it_ref) in zip(results, single):
                e = pb.pb_solvation_energy(ctx, res)
                it, rr, _ = pb.pb_result_get(res)
                assert rr <= 1e-7
                assert abs(it - it_ref) <= 2
                assert abs(e - e_ref) <= 1e-5 * abs(e_ref)
                pb.pb_result_destroy(res)
        with pytest.raises(pb.PBError):
            pb.pb_solve_batch(ctx, [meshes[0], meshes[0]], [sysl[0][2]] * 2, [sysl[0][3]] * 2, *EPS, 1e-7)
    finally:
        for m in meshes:
            pb.pb_mesh_destroy(m)
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("m", [5, 12])
def test_batch_restarted_gmres(pb, m):
    """GMRES(m) in the batch (PB_OPT_RESTART): every system converges to
    the same energy as the unrestarted batch (the restart recomputes the
    true residual, so the final residual is the true one at tol), with at
    least as many iterations, and restarts run within max_iter."""
    ctx = pb.pb_create(0, None)
    sysl = systems()
    meshes = [pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6, 64) for V, F, _, _ in sysl]
    try:
        args = ([s[2] for s in sysl], [s[3] for s in sysl], *EPS, 1e-7, 400)
        full, sts, rc = pb.pb_solve_batch(ctx, meshes, *args)
        assert rc == pb.PB_OK
        ref = [(pb.pb_solvation_energy(ctx, r_), pb.pb_result_get(r_)[0]) for r_ in full]
        for r_ in full:
            pb.pb_result_destroy(r_)
        pb.pb_set_option(ctx, pb.PB_OPT_RESTART, m)
        res, sts, rc = pb.pb_solve_batch(ctx, meshes, *args)
        assert rc == pb.PB_OK and np.all(sts == pb.PB_OK)
        for r_, (e_ref, it_ref) in zip(res, ref):
            e = pb.pb_solvation_energy(ctx, r_)
            it, rr, _ = pb.pb_result_get(r_)
            print(f"GMRES({m}): {it} iterations (full GMRES {it_ref}), dG {e:.9f} vs {e_ref:.9f}")
            assert rr <= 1e-7 and it >= it_ref
            assert abs(e - e_ref) <= 1e-5 * abs(e_ref)
            pb.pb_result_destroy(r_)
        # a cap below the need: PB_ENOCONV with the iterations at the cap
        res, sts, rc = pb.pb_solve_batch(ctx, meshes, [s[2] for s in sysl], [s[3] for s in sysl], *EPS, 1e-12, 2 * m)
        assert rc == pb.PB_ENOCONV
        for r_ in res:
            assert pb.pb_result_get(r_)[0] <= 2 * m
            pb.pb_result_destroy(r_)
    finally:
        for mm in meshes:
            pb.pb_mesh_destroy(mm)
        pb.pb_destroy(ctx)


def test_ncrit_autotuner(pb):
    ctx = pb.pb_create(0, None)
    try:
        x, _ = synthetic.bumpy_sphere_points(200000, seed=1)
        best, ms = pb.pb_tune_ncrit(ctx, torch.from_numpy(x).cuda(), 6, [32, 64, 128, 256])
        assert best in (32, 64, 128, 256) and ms > 0
    finally:
        pb.pb_destroy(ctx)


def test_tile_autotuner(pb):
    """pb_tune picks ncrit and the leaf / M2L tile shapes on the paired apply,
    leaves the winning tile options on the context, and an apply with them
    still matches the FP64 direct sum."""
    ctx = pb.pb_create(0, None)
    try:
        x, nrm = synthetic.bumpy_sphere_points(200000, seed=1)
        X = torch.from_numpy(x).cuda()
        best, nt, tile, ms = pb.pb_tune(ctx, X, 6, [64, 128])
        assert best in (64, 128) and nt in (2, 4) and tile in (0, 1) and ms > 0
        # the options on the context are the tuner's choice: setting them again is accepted
        pb.pb_set_option(ctx, pb.PB_OPT_LEAF_NT, nt)
        pb.pb_set_option(ctx, pb.PB_OPT_M2L_TILE, tile)
        with pytest.raises(pb.PBError):
            pb.pb_set_option(ctx, pb.PB_OPT_M2L_TILE, 2)
        # parity of every tile combination on a 20k-point case
        xs, ns = synthetic.bumpy_sphere_points(20000, seed=3)
        q = synthetic.uniform_densities(len(xs), seed=4)
        d = synthetic.uniform_densities(len(xs), seed=5)
        from oracle import kernels as ok
        refL = ok.direct_sum(ok.LAPLACE, 0.0, xs, q=q, dip=d, src_n=ns)
        refY = ok.direct_sum(ok.YUKAWA, 0.125, xs, q=q, dip=d, src_n=ns)
        h = pb.fmm_tree_build(ctx, torch.from_numpy(xs).cuda(), 64)
        try:
            for nt_ in (2, 4):
                for tile_ in (0, 1):
                    pb.pb_set_option(ctx, pb.PB_OPT_LEAF_NT, nt_)
                    pb.pb_set_option(ctx, pb.PB_OPT_M2L_TILE, tile_)
                    oL = torch.empty(len(xs), device="cuda")
                    oY = torch.empty(len(xs), device="cuda")
                    Q = torch.from_numpy(q).cuda()
                    pb.fmm_apply_pair(ctx, h, 0.125, 6, oL, oY, q_lap=Q, q_yuk=Q, dip=torch.from_numpy(d).cuda(),
                                      src_n=torch.from_numpy(ns).cuda())
                    pb.pb_sync(ctx)
                    for o, r in ((oL.cpu().numpy(), refL), (oY.cpu().numpy(), refY)):
                        assert np.linalg.norm(o - r) / np.linalg.norm(r) < 1e-5
        finally:
            pb.fmm_tree_destroy(h)
    finally:
        pb.pb_destroy(ctx)
