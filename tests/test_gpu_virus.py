"""Virus-scale shell (1.6M atoms, 9,984,600 triangles): the FMM apply over
its 29,953,800 quadrature points against the FP64 direct sum.

The full solve at this size has no affordable oracle; what is pinned is the
FMM that every GMRES iteration applies (Sec. "Fast multipole method";
direct-sum definition of the potentials, Eq. direct): the paired Laplace +
Yukawa single+double-layer apply over all quadrature points, checked on a
seeded sample of 1,000 targets against the oracle's FP64 sum over all
sources, at p = 4 (the order of the paper's virus run, "4 digits"), 6 and
8, and with the all-FP64 path.
"""
import numpy as np
import pytest

import synthetic
from oracle.bem import quad_points
from oracle.kernels import LAPLACE, YUKAWA, direct_sum, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = 0.125


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def shell():
    V, T, _, _, _ = synthetic.virus_shell()
    P, _, nrm, _ = quad_points(V, T, 3)
    x = P.astype(np.float32)
    n = nrm.astype(np.float32)
    q = synthetic.uniform_densities(len(x), seed=31)
    d = synthetic.uniform_densities(len(x), seed=32)
    idx = synthetic.random_subsample(len(x), 1000, seed=33)
    refL = direct_sum(LAPLACE, 0.0, x, q=q, dip=d, src_n=n, tgt=x[idx])
    refY = direct_sum(YUKAWA, KAPPA, x, q=q, dip=d, src_n=n, tgt=x[idx])
    return x, n, q, d, idx, refL, refY


def test_virus_shell_apply_sampled(pb, shell):
    """Mixed path at p = 4, 6, 8 and the all-FP64 path at p = 6, 8.

    Measured (GB300): mixed Laplace 2.65e-4 / 1.12e-5 / 1.15e-5 and Yukawa
    3.49e-4 / 5.98e-6 / 2.04e-6 at p = 4 / 6 / 8; FP64 at p = 6 3.43e-6 /
    5.55e-6.  The mixed Laplace error stops falling at 1.1e-5 from p = 6 on:
    with densities of random sign the potential is a small remainder of sums
    over 30M sources, and the FP32 rounding of those sums (the far field of
    the whole shell does not decay for Laplace as it does for Yukawa) sets a
    floor that p does not move, while the FP64 path on the same tree shows
    the FMM approximation itself well inside 1e-5.  Asserted: Yukawa within
    1e-5 at p = 8; Laplace at p = 8 within 2e-5 (the FP32 floor above, with
    margin); p = 4 within 5e-4 (the paper's "4 digits" at p = 4); errors
    decreasing from p = 4 to 6; FP64 within 1e-5 at p = 6 and 1e-6 at p = 8."""
    x, n, q, d, idx, refL, refY = shell
    assert len(x) == 29_953_800
    ctx = pb.pb_create(0, None)
    err = {}
    try:
        X = torch.from_numpy(x).cuda()
        Q, D, N = (torch.from_numpy(a).cuda() for a in (q, d, n))
        sel = torch.from_numpy(idx).cuda()
        h = pb.fmm_tree_build(ctx, X, 128)
        try:
            oL = torch.empty(len(x), device="cuda")
            oY = torch.empty(len(x), device="cuda")
            for p in (4, 6, 8):
                pb.fmm_apply_pair(ctx, h, KAPPA, p, oL, oY, q_lap=Q, q_yuk=Q, dip=D, src_n=N)
                pb.pb_sync(ctx)
                err[p] = (rel_l2(oL[sel].cpu().numpy(), refL), rel_l2(oY[sel].cpu().numpy(), refY))
                print(f"virus shell p={p}: rel L2 Laplace {err[p][0]:.2e}, Yukawa {err[p][1]:.2e}")
            del oL, oY
            oL = torch.empty(len(x), dtype=torch.float64, device="cuda")
            oY = torch.empty(len(x), dtype=torch.float64, device="cuda")
            Q64, D64, N64 = (t.double() for t in (Q, D, N))
            e64 = {}
            for p in (6, 8):
                pb.fmm_apply_pair(ctx, h, KAPPA, p, oL, oY, q_lap=Q64, q_yuk=Q64, dip=D64, src_n=N64,
                                  precision=pb.PB_FP64)
                pb.pb_sync(ctx)
                e64[p] = (rel_l2(oL[sel].cpu().numpy(), refL), rel_l2(oY[sel].cpu().numpy(), refY))
                print(f"virus shell FP64 p={p}: rel L2 Laplace {e64[p][0]:.2e}, Yukawa {e64[p][1]:.2e}")
        finally:
            pb.fmm_tree_destroy(h)
    finally:
        pb.pb_destroy(ctx)
    assert err[8][1] < 1e-5 and err[8][0] < 2e-5
    assert max(err[4]) < 5e-4
    assert err[6][0] < err[4][0] and err[6][1] < err[4][1]
    assert max(e64[6]) < 1e-5 and max(e64[8]) < 1e-6
