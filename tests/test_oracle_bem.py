"""Pins of the P0 Galerkin BEM oracle (no GPU).

* analytic triangle integrals vs brute-force quadrature away from the
  triangle, and the solid angle of a closed surface (Gauss: -4 pi inside, 0
  outside);
* Galerkin matrices vs the sphere identities V_L[1] = a, V_Y[1] =
  (1 - e^{-2 k a})/(2k), K_L[1] = -1/2 on the surface (to discretisation
  order), and K_L = 0 on identical flat triangles;
* the direct-formulation energy of a Born ion converging to the closed form
  at the paper's 1/N rate, and of the paper's off-centre Kirkwood sphere;
* the Kirkwood series against the paper's printed -12.258363 kcal/mol
  (golden fixture tests/golden/kirkwood_sphere.json).
"""
import ctypes
import json
import os

import numpy as np
import pytest

import synthetic
from oracle import bem, closed_forms as cf
from oracle._lib import lib

HERE = os.path.dirname(os.path.abspath(__file__))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def tri_sl(x, v):
    return lib().or_tri_sl(_p(np.ascontiguousarray(x, float)), *[_p(np.ascontiguousarray(t, float)) for t in v])


def tri_dl(x, v):
    return lib().or_tri_dl(_p(np.ascontiguousarray(x, float)), *[_p(np.ascontiguousarray(t, float)) for t in v])


def brute(x, v, f, n=400):
    # midpoint rule on an n x n split of the triangle (no singularity: x away)
    v0, v1, v2 = [np.asarray(t, float) for t in v]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m = i + j < n
    pts, wts = [], []
    # upright and inverted sub-triangles, centroid rule
    for up in (True, False):
        mm = m if up else (i + j < n - 1)
        a = (i[mm] + (1 / 3 if up else 2 / 3)) / n
        b = (j[mm] + (1 / 3 if up else 2 / 3)) / n
        pts.append(v0 + a[:, None] * (v1 - v0) + b[:, None] * (v2 - v0))
        wts.append(np.full(mm.sum(), 1.0))
    P = np.concatenate(pts)
    w = np.concatenate(wts)
    area = 0.5 * np.linalg.norm(np.cross(v1 - v0, v2 - v0))
    return area * (w * f(np.asarray(x, float) - P)).sum() / w.sum()


TRI = ([0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.2])


@pytest.mark.parametrize("x", [[0.4, 0.3, 1.0], [2.0, -1.0, 0.5], [0.5, 0.4, -0.6]])
def test_triangle_integrals_brute(x):
    sl = tri_sl(x, TRI)
    dl = tri_dl(x, TRI)
    n = np.cross(np.subtract(TRI[1], TRI[0]), np.subtract(TRI[2], TRI[0]))
    n /= np.linalg.norm(n)
    bsl = brute(x, TRI, lambda r: 1 / np.linalg.norm(r, axis=1))
    bdl = brute(x, TRI, lambda r: (r @ n) / np.linalg.norm(r, axis=1) ** 3)
    assert abs(sl - bsl) < 1e-5 * abs(bsl)
    assert abs(dl - bdl) < 1e-4 * abs(bdl)


def test_solid_angle_closed_surface():
    V, F = synthetic.icosphere(2, 1.3)
    for x, ref in [([0.1, 0.2, -0.3], -4 * np.pi), ([2.0, 0.1, 0.0], 0.0), ([0.0, 0.0, 0.0], -4 * np.pi)]:
        s = sum(tri_dl(x, V[f]) for f in F)
        assert abs(s - ref) < 1e-9


def test_in_plane_potential_limit():
    # continuity of the single-layer potential across the plane
    x = np.array([0.4, 0.3, 0.0])
    eps = 1e-7
    n = np.cross(np.subtract(TRI[1], TRI[0]), np.subtract(TRI[2], TRI[0]))
    n /= np.linalg.norm(n)
    x = np.asarray(TRI[0]) + 0.3 * np.subtract(TRI[1], TRI[0]) + 0.3 * np.subtract(TRI[2], TRI[0])
    a = tri_sl(x, TRI)
    b = tri_sl(x + eps * n, TRI)
    assert abs(a - b) < 1e-5
    # solid angle jump of 4 pi across the triangle
    assert abs(tri_dl(x + eps * n, TRI) - tri_dl(x - eps * n, TRI) - 4 * np.pi) < 1e-4


def test_sphere_operator_identities():
    a, k = 2.0, 0.125
    V, F = synthetic.icosphere(3, a)
    n, area = bem.geometry(V, F)
    VL, KL, VY, KY = bem.assemble_p0(V, F, 3, k)
    rows_vl = VL.sum(axis=1) / area
    rows_kl = KL.sum(axis=1) / area
    rows_vy = VY.sum(axis=1) / area
    assert abs(rows_vl.mean() - a) < 5e-3 * a
    assert abs(rows_kl.mean() + 0.5) < 5e-3
    assert abs(rows_vy.mean() - (1 - np.exp(-2 * k * a)) / (2 * k)) < 5e-3 * a
    assert np.all(np.abs(np.diag(KL)) < 1e-14)
    assert np.all(np.abs(np.diag(KY)) < 1e-14)
    assert np.all(np.diag(VL) > 0)


def test_singular_rule_converged():
    """The graded outer rule of the singular entries is converged well below
    the 1e-4 energy tolerance: the default rule agrees with a much finer one
    to 2e-6 relative on every identical or vertex-sharing pair."""
    V, F = synthetic.icosphere(1, 2.0)
    nt = len(F)
    adj = np.array([[len(set(F[i]) & set(F[j])) > 0 for j in range(nt)] for i in range(nt)])
    m1 = bem.assemble_p0(V, F, 3, 0.125)
    m2 = bem.assemble_p0(V, F, 3, 0.125, L_outer=8, n_outer=6, n_inner=6)
    for A, B in zip(m1, m2):
        d = np.abs((A - B)[adj]).max() / np.abs(B[adj]).max()
        assert d < 2e-6
        assert np.array_equal(A[~adj], B[~adj])


def test_born_ion_convergence():
    born = cf.born_energy(1.0, 2.0, 4.0, 80.0, 0.125)
    errs = []
    for lev in (1, 2, 3):
        V, F = synthetic.icosphere(lev, 2.0)
        E, phi, dphi, _ = bem.solve_energy(V, F, 3, np.zeros((1, 3)), np.array([1.0]), 4.0, 80.0, 0.125)
        errs.append(abs(E - born))
        assert phi.std() < 1e-2 * abs(phi.mean())     # symmetry: near-constant
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4            # 1/N convergence
    assert errs[-1] / abs(born) < 5e-3


def test_kirkwood_golden():
    g = json.load(open(os.path.join(HERE, "golden", "kirkwood_sphere.json")))
    E = cf.kirkwood_energy([g["q"]], [g["position"]], g["radius"], g["eps_in"], g["eps_out"], g["kappa"])
    assert abs(E - g["energy_kcal_mol"]) < 5e-7 * abs(g["energy_kcal_mol"])
    # Born is the n = 0 term of Kirkwood's series with the charge at the centre
    assert abs(cf.kirkwood_energy([1.0], [[0, 0, 0]], 2.0, 4.0, 80.0, 0.125)
               - cf.born_energy(1.0, 2.0, 4.0, 80.0, 0.125)) < 1e-12


def test_kirkwood_discrete_off_centre():
    """Discrete direct-formulation energy of the paper's off-centre sphere
    problem approaches the analytic value at first order in 1/N."""
    g = json.load(open(os.path.join(HERE, "golden", "kirkwood_sphere.json")))
    errs = []
    for lev in (1, 2, 3):
        V, F = synthetic.icosphere(lev, g["radius"])
        E, *_ = bem.solve_energy(V, F, 3, np.array([g["position"]]), np.array([g["q"]]),
                                 g["eps_in"], g["eps_out"], g["kappa"])
        errs.append(abs(E - g["energy_kcal_mol"]))
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert 3.0 < errs[1] / errs[2] < 5.0
    assert errs[-1] / abs(g["energy_kcal_mol"]) < 1e-2


def _monomial_exact(a, b):
    """int over the reference triangle (area 1/2) of l1^a l2^b, divided by
    its area: 2 a! b! / (a + b + 2)!  (Dirichlet integral)."""
    from math import factorial
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


@pytest.mark.parametrize("nq,degree", [(3, 2), (6, 4)])
def test_regular_rule_exact_degree(nq, degree):
    """The regular rules integrate every monomial l1^a l2^b with a + b <= the
    rule's degree exactly (interior degree-2 3-point rule, Dunavant's degree-4
    6-point rule; weights normalised to sum to 1), and are not exact one
    degree higher.  The published constants are given to 15 digits, so
    'exact' is 1e-13 here."""
    L, W = bem.regular_rule(nq)
    assert abs(W.sum() - 1.0) < 1e-14
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-15)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            got = (W * L[:, 1] ** a * L[:, 2] ** b).sum()
            assert abs(got - _monomial_exact(a, b)) < 1e-13, (nq, a, b)
    # one degree higher the rule is no longer exact for some monomial
    errs = [abs((W * L[:, 1] ** a * L[:, 2] ** (degree + 1 - a)).sum() - _monomial_exact(a, degree + 1 - a))
            for a in range(degree + 2)]
    assert max(errs) > 1e-6
    # symmetric under permutations of the barycentric coordinates
    for perm in ([1, 2, 0], [2, 0, 1], [1, 0, 2]):
        Lp = L[:, perm]
        for a in range(degree + 1):
            for b in range(degree + 1 - a):
                assert abs((W * Lp[:, 1] ** a * Lp[:, 2] ** b).sum() - _monomial_exact(a, b)) < 1e-13


def test_born_ion_golden_file():
    """The stored dense-LU energy of the 5,120-triangle Born ion (written by
    tests/golden/make_born_ion.py, oracle only) lies within the P0
    discretisation error of the Born closed form: the 1/N convergence pinned
    above gives about 7e-4 relative at this size."""
    g = json.load(open(os.path.join(HERE, "golden", "born_ion_5120.json")))
    born = cf.born_energy(1.0, 2.0, g["eps_in"], g["eps_out"], g["kappa"])
    assert abs(g["born_closed_form_kcal_mol"] - born) < 1e-12
    rel = abs(g["energy_kcal_mol"] - born) / abs(born)
    assert 1e-4 < rel < 2e-3


@pytest.mark.slow
def test_matrix_free_gmres_matches_dense_lu():
    """The matrix-free FP64 GMRES of the oracle (direct point sums, exact
    singular corrections; for sizes beyond the dense LU) gives the dense LU's
    energy on an off-centre charge in a 320-triangle sphere."""
    V, F = synthetic.icosphere(2, 2.0)
    atoms, q = np.array([[0.3, 0.2, -0.1]]), np.array([1.0])
    e_lu, *_ = bem.solve_energy(V, F, 3, atoms, q, 4.0, 80.0, 0.125)
    e_f, _, _, it, res = bem.solve_energy_free(V, F, 3, atoms, q, 4.0, 80.0, 0.125)
    assert res <= 1e-10 and it < 100
    assert abs(e_f - e_lu) < 1e-9 * abs(e_lu)
