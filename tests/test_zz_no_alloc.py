"""The allocation-free energy entry point agrees with pb_solvation_energy.

pb_solvation_energy_noalloc serves callers that cannot allocate device
memory when they need the energy: an application whose device allocator is
locked after start-up, or a real-time loop that must not enter the
allocator.  It keeps its intermediate values in one fixed array inside the
library.  The checks: two calls in a row give the energy of
pb_solvation_energy (direct reaction-potential sums: to rounding; FMM
coupling: to the FMM's error), the library's device-allocation count does
not move across a call, bad output buffers and too many atoms are
rejected.  This file runs last so that a failure here does not hide the
other tests' results.
"""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


def test_noalloc_energy_matches_allocating_entry_point(pb):
    ctx = pb.pb_create(0, None)
    V, F = synthetic.icosphere(3, 2.0)
    atoms = np.array([[0.2, -0.1, 0.3], [-0.5, 0.2, 0.1], [0.1, 0.6, -0.4]])
    q = np.array([0.6, -0.9, 0.4])
    mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6, 64)
    try:
        pb.pb_set_option(ctx, pb.PB_OPT_COUPLING, 1)           # direct sums everywhere
        res, st = pb.pb_solve(ctx, mesh, atoms, q, 4.0, 80.0, 0.125, 1e-8, 200)
        assert st == pb.PB_OK
        e_ref = pb.pb_solvation_energy(ctx, res)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):                       # two calls in a row share the scratch
            out.fill_(np.nan)
            n0 = pb._test_alloc_count()
            pb.pb_solvation_energy_noalloc(ctx, res, out)
            pb.pb_sync(ctx)
            assert pb._test_alloc_count() == n0   # no device allocation in the call
            e = float(out.item())
            assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
        # the allocating entry point does allocate (the counter sees it)
        n0 = pb._test_alloc_count()
        pb.pb_solvation_energy(ctx, res)
        assert pb._test_alloc_count() > n0
        # with the FMM coupling the allocating call differs by the FMM error
        pb.pb_set_option(ctx, pb.PB_OPT_COUPLING, 2)
        e_fmm = pb.pb_solvation_energy(ctx, res)
        pb.pb_solvation_energy_noalloc(ctx, res, out)
        pb.pb_sync(ctx)
        assert abs(float(out.item()) - e_ref) <= 1e-10 * abs(e_ref)    # noalloc ignores the option
        assert abs(e_fmm - e_ref) <= 1e-5 * abs(e_ref)
        pb.pb_set_option(ctx, pb.PB_OPT_COUPLING, 0)
        # output buffers that are not one float64 CUDA element are refused
        with pytest.raises(ValueError):
            pb.pb_solvation_energy_noalloc(ctx, res, np.zeros(1))
        with pytest.raises(ValueError):
            pb.pb_solvation_energy_noalloc(ctx, res, torch.zeros(1, dtype=torch.float32, device="cuda"))
        with pytest.raises(ValueError):
            pb.pb_solvation_energy_noalloc(ctx, res, torch.zeros(0, dtype=torch.float64, device="cuda"))
        # the library itself refuses a host pointer
        host = np.zeros(1)
        rc = pb._lib.pb_solvation_energy_noalloc(ctx, res, host.ctypes.data)
        assert rc == pb.PB_EINVAL and host[0] == 0.0
        pb.pb_result_destroy(res)
        # more atoms than the scratch holds: rejected with PB_EINVAL
        rng = np.random.default_rng(0)
        many = rng.uniform(-0.5, 0.5, (262_145, 3))
        qm = rng.uniform(-0.1, 0.1, 262_145)
        res2, _ = pb.pb_solve(ctx, mesh, many, qm, 4.0, 80.0, 0.125, 1e-3, 1)
        with pytest.raises(pb.PBError) as err:
            pb.pb_solvation_energy_noalloc(ctx, res2, out)
        assert err.value.code == pb.PB_EINVAL
        pb.pb_result_destroy(res2)
    finally:
        pb.pb_mesh_destroy(mesh)
        pb.pb_destroy(ctx)
