"""Charge <-> surface couplings through the FMM against the direct sums,
and the deterministic mode."""
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


def test_fmm_coupling_matches_direct(pb):
    V, T, xyz, radii, q, h = synthetic.synthetic_protein(natoms=250, target_tris=20000, ball_radius=11.0, seed=4)
    out = {}
    for mode in (1, 2):
        ctx = pb.pb_create(0, None)
        pb.pb_set_option(ctx, pb.PB_OPT_COUPLING, mode)
        mesh = pb.pb_mesh_setup(ctx, V, T.astype(np.int32), 3, 6, 64)
        try:
            res, st = pb.pb_solve(ctx, mesh, xyz, q, *EPS, 1e-8, 500)
            assert st == pb.PB_OK
            e, phir = pb.pb_solvation_energy(ctx, res, len(q))
            gq, gx, _ = pb.pb_energy_grad(ctx, res, len(q), tol=1e-8, max_iter=500)
            pb.pb_result_destroy(res)
        finally:
            pb.pb_mesh_destroy(mesh)
            pb.pb_destroy(ctx)
        out[mode] = (e, phir, gq)
    e1, p1, g1 = out[1]
    e2, p2, g2 = out[2]
    assert abs(e1 - e2) < 1e-5 * abs(e1)
    assert np.abs(p1 - p2).max() < 1e-4 * np.abs(p1).max()
    assert np.abs(g1 - g2).max() < 1e-4 * np.abs(g1).max()


def test_deterministic_mode_is_bitwise_reproducible(pb):
    ctx = pb.pb_create(0, None)
    pb.pb_set_option(ctx, pb.PB_OPT_DETERMINISTIC, 1)
    try:
        x, nrm = synthetic.bumpy_sphere_points(200000, seed=2)
        qd = synthetic.uniform_densities(200000, seed=3)
        tree = pb.fmm_tree_build(ctx, torch.from_numpy(x).cuda(), 64)
        outs = []
        for _ in range(2):
            o = torch.zeros(200000, device="cuda")
            pb.fmm_apply(ctx, tree, pb.FMM_YUKAWA, 0.125, 6, o, q=torch.from_numpy(qd).cuda(),
                         dip=torch.from_numpy(qd).cuda(), src_n=torch.from_numpy(nrm).cuda())
            torch.cuda.synchronize()
            outs.append(o.cpu().numpy())
        pb.fmm_tree_destroy(tree)
        assert np.array_equal(outs[0], outs[1])
        with pytest.raises(pb.PBError):
            pb.pb_set_option(ctx, 99, 1)
    finally:
        pb.pb_destroy(ctx)
