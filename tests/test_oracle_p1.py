"""Pins of the P1 Galerkin oracle and the derivative formulations (no GPU).

* linear-density analytic inner integrals against brute-force quadrature,
  and their sums against the uniform-density closed forms;
* the P1 matrices of V, K and the hypersingular W of both kernels against the
  sphere eigen-relations (Laplace: V Y_l = a/(2l+1), K Y_l = -1/(2(2l+1)),
  W Y_l = l(l+1)/(a(2l+1)); Yukawa, z = kappa a, with the modified spherical
  Bessel functions i_l, k_l (k_0(z) = e^-z / z): V = kappa a^2 i_l k_l,
  K = -1/2 + kappa^2 a^2 i_l' k_l, W = -kappa^3 a^2 i_l' k_l'), to the
  discretisation error, and W_L annihilating constants exactly;
* the integrated-by-parts (curl) form of W used by the oracle against the
  hypersingular kernel -d2g/dn_x dn_y of Eq. adj_hyp (itself pinned by finite
  differences in test_oracle_kernels) on hat functions with disjoint
  supports, and K' against the target-normal-derivative kernel;
* Born ion energies of the interior (Eq. juffer) and exterior (Eq. lu)
  derivative formulations and of the direct formulation in P1: the Born
  closed form at the paper's first order in N, interior = exterior;
* the paper's conditioning argument: the mass-preconditioned interior
  operator has two eigenvalue clusters, at (1 + eps2/eps1)/2 and
  (1 + eps1/eps2)/2, the exterior one a single cluster at the latter.
"""
import numpy as np
import pytest

import synthetic
from oracle import bem, bem_p1, closed_forms as cf
from oracle.kernels import LAPLACE, YUKAWA, direct_sum

EPS_IN, EPS_OUT, KAPPA = 4.0, 80.0, 0.125
TRI = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.1, 0.0]), np.array([0.3, 0.9, 0.2])]


def brute_lin(x, v, n=800):
    """Midpoint rule on an n x n split (upright and inverted sub-triangles)."""
    v0, v1, v2 = v
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts, lam = [], []
    for up in (True, False):
        mm = (i + j < n) if up else (i + j < n - 1)
        a = (i[mm] + (1 / 3 if up else 2 / 3)) / n
        b = (j[mm] + (1 / 3 if up else 2 / 3)) / n
        pts.append(v0 + a[:, None] * (v1 - v0) + b[:, None] * (v2 - v0))
        lam.append(np.stack([1 - a - b, a, b], 1))
    P, L = np.concatenate(pts), np.concatenate(lam)
    nrm = np.cross(v1 - v0, v2 - v0)
    area = 0.5 * np.linalg.norm(nrm)
    nrm /= 2 * area
    d = x - P
    r = np.linalg.norm(d, axis=1)
    return area * (L / r[:, None]).mean(0), area * (L * ((d @ nrm) / r ** 3)[:, None]).mean(0)


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.5], [2.0, -1.0, 0.3], [-0.5, 0.4, 0.05], [0.5, 0.45, -0.02],
                               [1.2, 1.3, 0.4]])
def test_linear_inner_integrals_brute_force(x):
    x = np.asarray(x, float)
    sl, dl = bem_p1.tri_lin(x, TRI)
    bs, bd = brute_lin(x, TRI)
    assert np.abs(sl - bs).max() < 3e-6 * np.abs(bs).max()
    assert np.abs(dl - bd).max() < 5e-6 * np.abs(bd).max()
    # partition of unity: the three linear densities add up to the uniform one
    from tests.test_oracle_bem import tri_dl, tri_sl
    assert abs(sl.sum() - tri_sl(x, TRI)) < 1e-12 * abs(sl.sum())
    assert abs(dl.sum() - tri_dl(x, TRI)) < 1e-12 * max(abs(dl.sum()), 1e-3)


def test_linear_inner_integrals_in_plane():
    """Points in the triangle's plane outside it (where the double layer
    vanishes), one of them on the extension of an edge (distance 0 from the
    edge line): finite single layer matching brute force, zero double layer."""
    n = np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0])
    for x in ([1.5, 0.15, 0.0], [-0.4, -0.3, 0.0], list(TRI[0] + 1.5 * (TRI[1] - TRI[0]))):
        x = np.asarray(x, float)
        x = x - ((x - TRI[0]) @ n) / (n @ n) * n          # project into the plane
        sl, dl = bem_p1.tri_lin(x, TRI)
        bs, _ = brute_lin(x, TRI)
        assert np.all(np.isfinite(sl)) and np.abs(dl).max() < 1e-9
        assert np.abs(sl - bs).max() < 3e-6 * np.abs(bs).max()


def _bessel(l, z):
    from scipy.special import spherical_in, spherical_kn
    i, ip = spherical_in(l, z), spherical_in(l, z, derivative=True)
    k, kp = 2 / np.pi * spherical_kn(l, z), 2 / np.pi * spherical_kn(l, z, derivative=True)
    return i, ip, k, kp


@pytest.fixture(scope="module")
def sphere2():
    a = 2.0
    V, F = synthetic.icosphere(2, a)
    return a, V, F, bem_p1.assemble_p1(V, F, 3, KAPPA)


def test_sphere_eigen_relations(sphere2):
    """Rayleigh quotients <A u, u>/<M u, u> of the constant (l = 0) and of
    z/a (l = 1) against the continuous eigenvalues, to the 320-triangle
    discretisation error (about 1%; 2.5% allowed).  The Yukawa W at l = 0 is
    the kappa^2 (n.n) term alone: its sign is pinned here."""
    a, V, F, m = sphere2
    M = m["M"]
    z = KAPPA * a
    fs = {0: np.ones(len(V)), 1: V[:, 2] / a}
    for l, f in fs.items():
        i, ip, k, kp = _bessel(l, z)
        exact = {"VL": a / (2 * l + 1), "KL": -1 / (2 * (2 * l + 1)), "VY": KAPPA * a * a * i * k,
                 "KY": -0.5 + KAPPA ** 2 * a * a * ip * k, "WY": -KAPPA ** 3 * a * a * ip * kp,
                 "KpL": -1 / (2 * (2 * l + 1)), "KpY": -0.5 + KAPPA ** 2 * a * a * ip * k}
        if l > 0:
            exact["WL"] = l * (l + 1) / (a * (2 * l + 1))
        for name, val in exact.items():
            got = (f @ m[name] @ f) / (f @ M @ f)
            assert abs(got - val) < 0.025 * abs(val), (name, l, got, val)
    one = np.ones(len(V))
    assert np.abs(m["WL"] @ one).max() < 1e-12 * np.abs(m["WL"]).max()


def _refined_points(V, F, tris, levels=3):
    """6-point rule on a 4^levels midpoint subdivision of the given
    triangles: points, weights, normals, hat values of each triangle's
    vertices (the owning triangle's barycentrics)."""
    L, W = bem.regular_rule(6)
    P, w, nrm, owner, lam = [], [], [], [], []
    for t in tris:
        v = V[F[t]]
        n = np.cross(v[1] - v[0], v[2] - v[0])
        area = 0.5 * np.linalg.norm(n)
        n /= 2 * area
        subs = [np.eye(3)]
        for _ in range(levels):
            nxt = []
            for s in subs:
                m01, m12, m20 = (s[0] + s[1]) / 2, (s[1] + s[2]) / 2, (s[2] + s[0]) / 2
                nxt += [np.array([s[0], m01, m20]), np.array([m01, s[1], m12]), np.array([m20, m12, s[2]]),
                        np.array([m12, m20, m01])]
            subs = nxt
        for s in subs:
            bary = L @ s                     # barycentrics of the sub-rule points in t
            P.append(bary @ v)
            w.append(W * area / len(subs))
            nrm.append(np.repeat(n[None], len(W), 0))
            owner.append(np.full(len(W), t))
            lam.append(bary)
    return (np.concatenate(P), np.concatenate(w), np.concatenate(nrm), np.concatenate(owner),
            np.concatenate(lam))


def _hat_at(F, owner, lam, vertex):
    """Hat function of `vertex` at refined points (0 where it is not a vertex)."""
    val = np.zeros(len(owner))
    for a in range(3):
        sel = F[owner, a] == vertex
        val[sel] = lam[sel, a]
    return val


def test_hypersingular_curl_form_and_adjoint_double_layer(sphere2):
    """For hat functions with disjoint supports the curl form equals the
    hypersingular kernel: W_ij = -int int phi_i(x) d2g/dn_x dn_y phi_j(y)
    (Eq. adj_hyp); and K'_ij = int int phi_i(x) dg/dn_x phi_j(y).  Both
    sides with a fine rule (pins the curl form, the sign of its kappa^2
    term and the transpose); the assembled 3-point-rule entries within that
    rule's error at this separation."""
    a, V, F, m = sphere2
    F = np.asarray(F)
    i = int(np.argmax(V[:, 2]))
    d = np.linalg.norm(V - V[i], axis=1)
    j = int(np.argsort(np.abs(d - 1.6))[0])          # a vertex about 1.6 A away
    ti = [t for t in range(len(F)) if i in F[t]]
    tj = [t for t in range(len(F)) if j in F[t]]
    assert not set(F[ti].ravel()) & set(F[tj].ravel())
    Px, wx, nx, ox, lx = _refined_points(V, F, ti)
    Py, wy, ny, oy, ly = _refined_points(V, F, tj)
    phx = _hat_at(F, ox, lx, i)
    phy = _hat_at(F, oy, ly, j)
    for kernel, kappa, name in ((LAPLACE, 0.0, "L"), (YUKAWA, KAPPA, "Y")):
        # hypersingular kernel: dn[x] = sum_y d2g/dn_x dn_y d_y, d_y = w phi_j
        _, dn = direct_sum(kernel, kappa, Py, dip=wy * phy, src_n=ny, tgt=Px, tgt_n=nx, want_dn=True)
        w_hyp = -(wx * phx) @ dn
        # curl form: curl phi (constant per triangle) and the kappa^2 (n.n) term
        cx = np.zeros((len(Px), 3))
        cy = np.zeros((len(Py), 3))
        for pts, c, own, vert in ((Px, cx, ox, i), (Py, cy, oy, j)):
            for t in set(own):
                v = V[F[t]]
                area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
                aa = list(F[t]).index(vert)
                c[own == t] = (v[(aa + 1) % 3] - v[(aa + 2) % 3]) / (2 * area)
        w_curl = 0.0
        for k in range(3):
            w_curl += (wx * cx[:, k]) @ direct_sum(kernel, kappa, Py, q=wy * cy[:, k], tgt=Px)
        if kernel == YUKAWA:
            for k in range(3):
                w_curl += KAPPA ** 2 * (wx * phx * nx[:, k]) @ direct_sum(kernel, kappa, Py,
                                                                          q=wy * phy * ny[:, k], tgt=Px)
        assert abs(w_curl - w_hyp) < 1e-7 * abs(w_hyp), (name, w_curl, w_hyp)
        assert abs(m["W" + name][i, j] - w_hyp) < 2e-3 * abs(w_hyp), (name, m["W" + name][i, j], w_hyp)
        # adjoint double layer: target-normal derivative of the single layer
        _, kp = direct_sum(kernel, kappa, Py, q=wy * phy, tgt=Px, tgt_n=nx, want_dn=True)
        kp_ij = (wx * phx) @ kp
        assert abs(m["Kp" + name][i, j] - kp_ij) < 2e-3 * abs(kp_ij), (name, m["Kp" + name][i, j], kp_ij)


def test_born_ion_derivative_formulations(sphere2):
    """Interior (Eq. juffer), exterior (Eq. lu) and direct (Eq. direct)
    formulations in P1 converge to the Born energy at first order in N
    (errors fall by about 4 per icosphere refinement, the paper's 1/N), and
    the two derivative formulations (a row and unknown scaling of each
    other) give the same energy."""
    born = cf.born_energy(1.0, 2.0, EPS_IN, EPS_OUT, KAPPA)
    errs = {}
    a, V2, F2, m2 = sphere2
    V1, F1 = synthetic.icosphere(1, 2.0)
    m1 = bem_p1.assemble_p1(V1, F1, 3, KAPPA)
    for lev, V, F, m in ((1, V1, F1, m1), (2, V2, F2, m2)):
        es = {}
        for form in bem_p1.FORMULATIONS:
            e, *_ = bem_p1.solve_energy(V, F, 3, np.zeros((1, 3)), np.array([1.0]), EPS_IN, EPS_OUT, KAPPA,
                                        form, mats=m)
            es[form] = e
            errs[(form, lev)] = abs(e - born) / abs(born)
        assert abs(es["interior"] - es["exterior"]) < 1e-11 * abs(born)
    for form in bem_p1.FORMULATIONS:
        assert errs[(form, 2)] < 0.015
        assert 3.0 < errs[(form, 1)] / errs[(form, 2)] < 5.0, form


def test_spectrum_clusters():
    """Sec. "Matrix conditioning of two derivative formulations": with the
    P1 mass matrix as preconditioner the interior operator's eigenvalues
    gather at (1 + eps2/eps1)/2 = 10.5 and at (1 + eps1/eps2)/2 = 0.525,
    the exterior operator's at 0.525 only (a non-spherical 4-atom Gaussian
    surface, ~650 triangles).  Mass lumping keeps the exterior spectrum
    inside a narrow band as well."""
    xyz, radii, q = synthetic.fcc_ball_atoms(4, 3.5, 2.85, 0.1, seed=4)
    V, F = synthetic.gaussian_surface(xyz, radii, 1.3)
    m = bem_p1.assemble_p1(V, F, 3, KAPPA)
    c_hi, c_lo = 0.5 * (1 + EPS_OUT / EPS_IN), 0.5 * (1 + EPS_IN / EPS_OUT)
    ev_i = bem_p1.preconditioned_spectrum(m, V, F, EPS_IN, EPS_OUT, "interior")
    ev_e = bem_p1.preconditioned_spectrum(m, V, F, EPS_IN, EPS_OUT, "exterior")
    near = lambda ev, c: np.mean(np.abs(ev - c) < 0.25 * c)
    assert near(ev_i, c_hi) > 0.4 and near(ev_i, c_lo) > 0.4
    assert near(ev_e, c_lo) > 0.85 and near(ev_e, c_hi) == 0.0
    spread = lambda ev: np.abs(ev).max() / np.abs(ev).min()
    assert spread(ev_e) < 5.0 < 20.0 < spread(ev_i)
    ev_el = bem_p1.preconditioned_spectrum(m, V, F, EPS_IN, EPS_OUT, "exterior", lumped=True)
    ev_il = bem_p1.preconditioned_spectrum(m, V, F, EPS_IN, EPS_OUT, "interior", lumped=True)
    assert ev_el.real.max() < 1.0 < 10.0 < ev_il.real.max()
