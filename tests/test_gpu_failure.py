"""Failure paths, reached without faulting or hanging the GPU.

* Bounded device waits: the tensor-core box-operator kernel's mbarrier waits
  are shortened to a few cycles (test hook), so they give up; the kernel then
  stops its roles, drains its own MMAs and copies, frees its tensor memory
  and flags the error, and pb_sync reports PB_ETIMEOUT.  The context stays
  usable: with the default limit restored the same apply matches the FP64
  direct sum again.
* Device-allocation failure: the nth allocation of a call is made to fail on
  the host (test hook) as a failed cudaMallocAsync would.  The call returns
  PB_ENOMEM, gives back every byte it took from the memory pool, leaves no
  half-built cache behind, and the same call afterwards succeeds with the
  right numbers.
"""
import numpy as np
import pytest

import synthetic
from oracle.kernels import LAPLACE, YUKAWA, direct_sum, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KAPPA = 0.125


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def ctx(pb):
    c = pb.pb_create(0, None)
    yield c
    pb._test_fail_alloc(0)
    pb._test_wait_limit(0)
    pb.pb_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def case(pb):
    x, nrm = synthetic.bumpy_sphere_points(20000, seed=5)
    q = synthetic.uniform_densities(20000, seed=6)
    d = synthetic.uniform_densities(20000, seed=7)
    ref_l = direct_sum(LAPLACE, 0.0, x, q=q, dip=d, src_n=nrm)
    ref_y = direct_sum(YUKAWA, KAPPA, x, q=q, dip=d, src_n=nrm)
    return x, nrm, q, d, ref_l, ref_y


def paired(pb, ctx, tree, case, p=6):
    x, nrm, q, d, _, _ = case
    n = len(x)
    oL = torch.zeros(n, dtype=torch.float32, device="cuda")
    oY = torch.zeros(n, dtype=torch.float32, device="cuda")
    qd, dd, nd = dev(q), dev(d), dev(nrm)
    pb.fmm_apply_pair(ctx, tree, KAPPA, p, oL, oY, q_lap=qd, q_yuk=qd, dip=dd, src_n=nd)
    return oL, oY


def test_bounded_wait_gives_up_with_etimeout(pb, ctx, case):
    x = case[0]
    tree = pb.fmm_tree_build(ctx, dev(x), 64)
    try:
        paired(pb, ctx, tree, case)          # operators built, tensor-core path warm
        pb.pb_sync(ctx)
        got = None
        for _ in range(3):                   # a wait that happens to succeed at once cannot time out
            pb._test_wait_limit(1)
            try:
                paired(pb, ctx, tree, case)
                pb.pb_sync(ctx)
            except pb.PBError as e:
                got = e.code
            finally:
                pb._test_wait_limit(0)
            if got is not None:
                break
        assert got == pb.PB_ETIMEOUT
        # the error was reported once and cleared; the context works again
        pb.pb_sync(ctx)
        oL, oY = paired(pb, ctx, tree, case)
        pb.pb_sync(ctx)
        assert rel_l2(oL.cpu().numpy(), case[4]) < 1e-5
        assert rel_l2(oY.cpu().numpy(), case[5]) < 1e-5
    finally:
        pb.fmm_tree_destroy(tree)


def _expect_enomem_without_leak(pb, ctx, nth, call):
    """Run `call` with its nth allocation failing; True if it failed with
    PB_ENOMEM (pool usage unchanged), False if it needed fewer allocations."""
    torch.cuda.synchronize()
    pb.pb_sync(ctx)
    used0 = pb._test_pool_used(0)
    pb._test_fail_alloc(nth)
    try:
        r = call()
    except pb.PBError as e:
        assert e.code == pb.PB_ENOMEM, e
        pb.pb_sync(ctx)
        assert pb._test_pool_used(0) == used0, f"allocation {nth}: pool usage changed"
        return True
    finally:
        pb._test_fail_alloc(0)
    return r


def test_allocation_failure_tree_build(pb, ctx, case):
    x = dev(case[0])
    n_fail = 0
    for nth in range(1, 200):
        r = _expect_enomem_without_leak(pb, ctx, nth, lambda: pb.fmm_tree_build(ctx, x, 64))
        if r is True:
            n_fail += 1
            continue
        pb.fmm_tree_destroy(r)              # nth beyond the call's allocations: it succeeded
        break
    assert n_fail >= 10


def _tree_footprint(pb, ctx, x, case, fail_at):
    """Pool bytes a fresh tree holds after (optionally) one apply whose
    allocation `fail_at` fails and then one apply that succeeds; the
    successful apply's results are checked against the direct sum."""
    torch.cuda.synchronize()
    pb.pb_sync(ctx)
    u0 = pb._test_pool_used(0)
    tree = pb.fmm_tree_build(ctx, x, 64)
    try:
        failed = False
        if fail_at:
            pb._test_fail_alloc(fail_at)
            try:
                paired(pb, ctx, tree, case)
                pb.pb_sync(ctx)
            except pb.PBError as e:
                assert e.code == pb.PB_ENOMEM
                failed = True
            finally:
                pb._test_fail_alloc(0)
        oL, oY = paired(pb, ctx, tree, case)
        pb.pb_sync(ctx)
        assert rel_l2(oL.cpu().numpy(), case[4]) < 1e-5
        assert rel_l2(oY.cpu().numpy(), case[5]) < 1e-5
        del oL, oY
        torch.cuda.synchronize()
        pb.pb_sync(ctx)
        return pb._test_pool_used(0) - u0, failed
    finally:
        pb.fmm_tree_destroy(tree)


def test_allocation_failure_apply_and_solve(pb, ctx, case):
    x = dev(case[0])
    # the first apply on a tree builds and caches the operator sets of both
    # kernels: a failure part-way may leave a finished set cached (as a
    # successful call would), never a half-built one and nothing else, so
    # after one more successful apply the tree holds exactly the bytes of a
    # tree that never saw a failure
    ref, _ = _tree_footprint(pb, ctx, x, case, 0)
    n_fail = 0
    for nth in (1, 2, 3, 5, 9, 17, 33, 65):
        got, failed = _tree_footprint(pb, ctx, x, case, nth)
        n_fail += failed
        assert got == ref, f"allocation {nth}: {got} bytes held, {ref} without the failure"
    assert n_fail >= 6
    # mesh set-up and a solve
    V, F = synthetic.icosphere(2, 2.0)
    F = F.astype(np.int32)
    atoms = np.array([[0.1, 0.2, -0.3]])
    q = np.array([1.0])
    for nth in (1, 2, 4, 8, 16, 32):
        r = _expect_enomem_without_leak(pb, ctx, nth, lambda: pb.pb_mesh_setup(ctx, V, F, 3, 6, 64))
        if r is not True:
            pb.pb_mesh_destroy(r)
            break
    mesh = pb.pb_mesh_setup(ctx, V, F, 3, 6, 64)
    try:
        # two solves first: the second captures the mesh's mat-vec graph, a
        # cache the mesh keeps; later solves only take per-call workspace
        for _ in range(2):
            res, _ = pb.pb_solve(ctx, mesh, atoms, q, 4.0, 80.0, KAPPA, 1e-8, 200)
            e_ref = pb.pb_solvation_energy(ctx, res)
            pb.pb_result_destroy(res)
        failed = 0
        for nth in (1, 2, 3, 5, 8, 13, 21, 34):
            r = _expect_enomem_without_leak(
                pb, ctx, nth, lambda: pb.pb_solve(ctx, mesh, atoms, q, 4.0, 80.0, KAPPA, 1e-8, 200))
            if r is True:
                failed += 1
                continue
            pb.pb_result_destroy(r[0])
            break
        assert failed >= 3
        res, st = pb.pb_solve(ctx, mesh, atoms, q, 4.0, 80.0, KAPPA, 1e-8, 200)
        assert st == pb.PB_OK
        e = pb.pb_solvation_energy(ctx, res)
        pb.pb_result_destroy(res)
        # the mixed path's FMM reductions run in a run-dependent order (~1e-7)
        assert abs(e - e_ref) <= 1e-7 * abs(e_ref)
    finally:
        pb.pb_mesh_destroy(mesh)
