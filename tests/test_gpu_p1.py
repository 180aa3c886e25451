"""P1 basis and the derivative formulations on the GPU against the oracle.

* the mat-vec of every formulation (direct, exterior Eq. lu, interior
  Eq. juffer) against the dense P1 Galerkin matrices of the oracle
  (oracle/bem_p1.py), mixed and FP64, with and without the lumped-mass
  preconditioner, on a sphere and on a Gaussian surface;
* solves: the energy against the oracle's dense LU solve of the same system
  (within the 1e-4 target), interior = exterior, and the exterior
  formulation converging in fewer iterations than the interior one
  (Sec. "Matrix conditioning of two derivative formulations");
* the exterior formulation's iteration count stays flat under mesh
  refinement while the direct formulation's grows (the paper's performance
  tables), with the Born energy at first order in N;
* argument checks: derivative formulations need a P1 mesh; gradients,
  batches and the allocation-free energy take P0 results only.
"""
import numpy as np
import pytest

import synthetic
from oracle import bem_p1, closed_forms as cf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = (4.0, 80.0, 0.125)
FORMS = {"direct": 0, "exterior": 1, "interior": 2}


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


@pytest.fixture(scope="module")
def ctx(pb):
    c = pb.pb_create(0, None)
    yield c
    pb.pb_destroy(c)


def _systems():
    V, F = synthetic.icosphere(2, 2.0)
    yield "sphere320", V, F.astype(np.int32)
    xyz, radii, q = synthetic.fcc_ball_atoms(4, 3.5, 2.85, 0.1, seed=4)
    Vg, Fg = synthetic.gaussian_surface(xyz, radii, 1.3)
    yield "gaussian648", Vg, Fg.astype(np.int32)


@pytest.fixture(scope="module")
def oracle_mats():
    return {name: (V, F, bem_p1.assemble_p1(V, F, 3, EPS[2])) for name, V, F in _systems()}


@pytest.mark.parametrize("name", ["sphere320", "gaussian648"])
def test_p1_singular_blocks(pb, ctx, oracle_mats, name):
    """The P1 singular blocks (minus their regular-rule part) of every
    vertex-sharing pair against the oracle's with the same graded outer rule
    (5 levels, the GPU's FP64 rule): the Laplace blocks equal to rounding;
    the Yukawa blocks add the smooth remainder, which the GPU integrates with
    a 2-level rule (measured 5e-7 of the largest block).  Against the
    oracle's default 6 levels they differ by the rule's own convergence
    (measured: 3.7e-6 of the largest V block, 4.4e-5 of the largest K
    block, exactly the oracle's own 5-versus-6-level difference)."""
    V, F, _ = oracle_mats[name]
    mesh = pb.pb_mesh_setup(ctx, V, F, 3, 6, 32, basis=pb.PB_P1)
    try:
        off, ids, S = pb.pb_mesh_export_singular(ctx, mesh, EPS[2], p1=True)
    finally:
        pb.pb_mesh_destroy(mesh)
    pairs = [(i, int(ids[e])) for i in range(len(F)) for e in range(off[i], off[i + 1])]
    ref5 = bem_p1.pair_blocks(V, F, pairs, 3, EPS[2], minus_regular=True, L_outer=5)
    ref6 = bem_p1.pair_blocks(V, F, pairs, 3, EPS[2], minus_regular=True, L_outer=6)
    for op in range(4):
        err5 = np.abs(S[:, op] - ref5[:, op]).max() / np.abs(ref5[:, op]).max()
        err6 = np.abs(S[:, op] - ref6[:, op]).max() / np.abs(ref6[:, op]).max()
        print(f"P1 singular blocks {name} op {op}: max rel {err5:.2e} (same rule), {err6:.2e} (6 levels)")
        assert err5 < (1e-10 if op in (0, 1) else 2e-6), op
        assert err6 < (1e-5 if op in (0, 2) else 1e-4), op


@pytest.mark.parametrize("name", ["sphere320", "gaussian648"])
@pytest.mark.parametrize("form", ["direct", "exterior", "interior"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_p1_matvec_vs_dense(pb, ctx, oracle_mats, name, form, prec):
    V, F, m = oracle_mats[name]
    nv = len(V)
    A = bem_p1.system_matrix(m, *EPS[:2], form)
    lm = bem_p1.lumped_mass(V, F)
    mesh = pb.pb_mesh_setup(ctx, V, F, 3, 6, 32, basis=pb.PB_P1)
    try:
        assert pb.pb_mesh_unknowns(mesh) == nv
        rng = np.random.default_rng(3)
        x = rng.uniform(-1, 1, 2 * nv)
        for precond in (False, True):
            y = np.zeros(2 * nv)
            pb.pb_mesh_matvec(ctx, mesh, x, y, *EPS, precision=pb.PB_FP64 if prec == "fp64" else pb.PB_MIXED,
                              precond=precond, formulation=FORMS[form])
            ref = A @ x
            if precond:
                ref = ref / np.concatenate([lm, lm])
            err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
            print(f"P1 mat-vec {name} {form} {prec} precond={precond}: rel L2 {err:.2e}")
            # the GPU's singular rule is 5 graded levels deep, the oracle's 6:
            # 3.7e-6 of the V blocks, 4.4e-5 of the (smaller) K blocks, so
            # the FP64 mat-vec agrees to a few 1e-6
            assert err < (2e-5 if prec == "mixed" else 1e-5)
    finally:
        pb.pb_mesh_destroy(mesh)


def test_p1_solves_vs_oracle(pb, ctx, oracle_mats):
    """Energies of the three P1 formulations against the dense LU oracle
    (Born ion and an off-centre charge pair in the Gaussian surface)."""
    cases = {"sphere320": (np.zeros((1, 3)), np.array([1.0])),
             "gaussian648": (None, None)}
    its = {}
    for name, (V, F, m) in oracle_mats.items():
        atoms, q = cases[name]
        if atoms is None:
            xyz, radii, qq = synthetic.fcc_ball_atoms(4, 3.5, 2.85, 0.1, seed=4)
            atoms, q = xyz, qq
        mesh = pb.pb_mesh_setup(ctx, V, F, 3, 6, 32, basis=pb.PB_P1)
        try:
            es = {}
            for form, code in FORMS.items():
                e_ref, *_ = bem_p1.solve_energy(V, F, 3, atoms, q, *EPS, form, mats=m)
                for prec in (pb.PB_MIXED, pb.PB_FP64):
                    res, st = pb.pb_solve(ctx, mesh, atoms, q, *EPS, 1e-9, 500, precision=prec, formulation=code)
                    assert st == pb.PB_OK
                    e = pb.pb_solvation_energy(ctx, res)
                    it, rr, _ = pb.pb_result_get(res)
                    pb.pb_result_destroy(res)
                    its[(name, form, prec)] = it
                    print(f"P1 solve {name} {form} prec={prec}: dG {e:.8f} oracle {e_ref:.8f} "
                          f"rel {abs(e - e_ref) / abs(e_ref):.2e}, {it} iterations")
                    assert abs(e - e_ref) < 1e-4 * abs(e_ref)
                    es[(form, prec)] = e
            assert abs(es[("exterior", pb.PB_FP64)] - es[("interior", pb.PB_FP64)]) < 1e-7 * abs(es[("exterior", 1)])
        finally:
            pb.pb_mesh_destroy(mesh)
    for name in oracle_mats:
        assert its[(name, "exterior", pb.PB_FP64)] < its[(name, "interior", pb.PB_FP64)]


def test_exterior_iterations_flat_under_refinement(pb, ctx):
    """Born ion on icospheres of 320 ... 20,480 triangles: the exterior
    derivative formulation (P1, lumped mass) converges in about the same
    number of iterations at every size, the direct one (P0, block
    diagonal) in more and more; both energies approach the Born value at
    first order in N."""
    born = cf.born_energy(1.0, 2.0, *EPS)
    rows = []
    for lev in (2, 3, 4, 5):
        V, F = synthetic.icosphere(lev, 2.0)
        F = F.astype(np.int32)
        row = {"nt": len(F)}
        for label, basis, form in (("ext", pb.PB_P1, 1), ("dir", pb.PB_P0, 0)):
            mesh = pb.pb_mesh_setup(ctx, V, F, 3, 6, 64, basis=basis)
            res, st = pb.pb_solve(ctx, mesh, np.zeros((1, 3)), np.array([1.0]), *EPS, 1e-6, 500, formulation=form)
            assert st == pb.PB_OK
            row[label + "_e"] = abs(pb.pb_solvation_energy(ctx, res) - born) / abs(born)
            row[label + "_it"] = pb.pb_result_get(res)[0]
            pb.pb_result_destroy(res)
            pb.pb_mesh_destroy(mesh)
        rows.append(row)
        print("refinement", row)
    ext = [r["ext_it"] for r in rows]
    assert max(ext) - min(ext) <= 3
    for a, b in zip(rows, rows[1:]):
        assert 3.0 < a["ext_e"] / b["ext_e"] < 5.0
    assert rows[-1]["dir_it"] > rows[0]["dir_it"]


def test_p1_argument_checks(pb, ctx):
    V, F = synthetic.icosphere(1, 2.0)
    F = F.astype(np.int32)
    m0 = pb.pb_mesh_setup(ctx, V, F, 3, 6, 32)
    m1 = pb.pb_mesh_setup(ctx, V, F, 3, 6, 32, basis=pb.PB_P1)
    try:
        with pytest.raises(pb.PBError) as e:
            pb.pb_solve(ctx, m0, np.zeros((1, 3)), np.array([1.0]), *EPS, 1e-6, 100, formulation=1)
        assert e.value.code == pb.PB_EINVAL
        res, _ = pb.pb_solve(ctx, m1, np.zeros((1, 3)), np.array([1.0]), *EPS, 1e-6, 100, formulation=1)
        with pytest.raises(pb.PBError) as e:
            pb.pb_energy_grad(ctx, res, 1)
        assert e.value.code == pb.PB_EINVAL
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(pb.PBError) as e:
            pb.pb_solvation_energy_noalloc(ctx, res, out)
        assert e.value.code == pb.PB_EINVAL
        pb.pb_result_destroy(res)
        with pytest.raises(pb.PBError) as e:       # a derivative formulation on a P0 mesh
            pb.pb_solve_batch(ctx, [m1, m0], [np.zeros((1, 3))] * 2, [np.array([1.0])] * 2, *EPS, 1e-6, 100,
                              formulation=FORMS["exterior"])
        assert e.value.code == pb.PB_EINVAL
    finally:
        pb.pb_mesh_destroy(m0)
        pb.pb_mesh_destroy(m1)


@pytest.mark.parametrize("form", ["exterior", "direct"])
def test_p1_batch_vs_single_and_oracle(pb, ctx, oracle_mats, form):
    """pb_solve_batch_ex on P1 meshes (the two oracle systems and a finer
    sphere): every energy equals the one-at-a-time pb_solve_ex result up to
    the FMM's summation order, and the oracle systems match the dense LU
    oracle within the 1e-4 target."""
    Vs, Fs = synthetic.icosphere(3, 2.0)
    xyz, radii, qq = synthetic.fcc_ball_atoms(4, 3.5, 2.85, 0.1, seed=4)
    systems = [(oracle_mats["sphere320"], np.zeros((1, 3)), np.array([1.0])),
               (oracle_mats["gaussian648"], xyz, qq),
               ((Vs, Fs.astype(np.int32), None), np.array([[0.5, -0.3, 0.2]]), np.array([-1.0]))]
    meshes = [pb.pb_mesh_setup(ctx, V, F, 3, 6, 32, basis=pb.PB_P1) for (V, F, _), _, _ in systems]
    try:
        res, st, rc = pb.pb_solve_batch(ctx, meshes, [a for _, a, _ in systems], [q for _, _, q in systems], *EPS,
                                        1e-9, 500, formulation=FORMS[form])
        assert rc == pb.PB_OK and all(s_ == pb.PB_OK for s_ in st)
        eb = [pb.pb_solvation_energy(ctx, r_) for r_ in res]
        itb = [pb.pb_result_get(r_)[0] for r_ in res]
        for r_ in res:
            pb.pb_result_destroy(r_)
        for k, (m, ((V, F, mats), a, q)) in enumerate(zip(meshes, systems)):
            r1, s1 = pb.pb_solve(ctx, m, a, q, *EPS, 1e-9, 500, formulation=FORMS[form])
            e1 = pb.pb_solvation_energy(ctx, r1)
            it1 = pb.pb_result_get(r1)[0]
            pb.pb_result_destroy(r1)
            print(f"P1 batch {form} system {k}: dG {eb[k]:.9f} single {e1:.9f}, iterations {itb[k]} / {it1}")
            assert abs(eb[k] - e1) < 1e-7 * abs(e1)
            if mats is not None:
                e_ref, *_ = bem_p1.solve_energy(V, F, 3, a, q, *EPS, form, mats=mats)
                assert abs(eb[k] - e_ref) < 1e-4 * abs(e_ref)
    finally:
        for m in meshes:
            pb.pb_mesh_destroy(m)
