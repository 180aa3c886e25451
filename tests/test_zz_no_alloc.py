"""The allocation-free energy entry point agrees with pb_solvation_energy.

pb_solvation_energy_noalloc serves callers that cannot allocate device
memory when they need the energy (for example during CUDA graph capture);
it keeps its scratch in a fixed array inside the library.  This file runs
last so that a failure here does not hide the other tests' results.
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
    V, F = synthetic.icosphere(2, 2.0)
    atoms = np.array([[0.2, -0.1, 0.3], [-0.5, 0.2, 0.1]])
    q = np.array([0.6, -0.9])
    mesh = pb.pb_mesh_setup(ctx, V, F.astype(np.int32), 3, 6, 64)
    try:
        res, st = pb.pb_solve(ctx, mesh, atoms, q, 4.0, 80.0, 0.125, 1e-8, 200)
        assert st == pb.PB_OK
        e_ref = pb.pb_solvation_energy(ctx, res)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):                       # two calls in a row share the scratch
            out.zero_()
            pb.pb_solvation_energy_noalloc(ctx, res, out)
            pb.pb_sync(ctx)
            e = float(out.item())
            assert abs(e - e_ref) <= 1e-10 * abs(e_ref)
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
