"""P1 Galerkin oracle of the derivative formulations (and the direct one).

Test infrastructure only.

Continuous piecewise-linear (P1) trial and test functions phi_i (hat
functions of the vertices) on flat triangles (Sec. "Matrix conditioning of
two derivative formulations": both spaces P1).  Dense matrices from
oracle.c (or_assemble_p1): V, K of both kernels and the hypersingular W in
its integrated-by-parts form; the adjoint double layer K' (Eq. adj_hyp, the
target-normal derivative, reading: the garbled dg/dn is d g / d n_x) is the
transpose of K in this Galerkin setting, <K' u, v> = <u, K v>.  M is the P1
mass matrix, M_ij = sum_T |T| (1 + delta_ij) / 12.

Interior derivative formulation (Eq. juffer), unknowns x = [phi_1; dphi_1/dn]:
  [ (1+e21)/2 M - (e21 K_Y - K_L)    V_Y - V_L                   ]
  [ W_Y - W_L                        (1+e12)/2 M + e12 K'_Y - K'_L ]
  rhs = [int phi_i f; int phi_i df/dn],  f = sum_k q_k / (4 pi eps1 |x - r_k|)
with e21 = eps2/eps1, e12 = eps1/eps2.
Exterior derivative formulation (Eq. lu), unknowns x = [phi_2; dphi_2/dn]:
  [ (1+e12)/2 M - (K_Y - e12 K_L)    V_Y - V_L                   ]
  [ e12 (W_Y - W_L)                  (1+e12)/2 M + e12 K'_Y - K'_L ]
  rhs with eps2 in place of eps1 (reading of the garbled "phi_2/dn": the
  normal derivative d phi_2 / dn); then phi_1 = phi_2, dphi_1/dn =
  e21 dphi_2/dn on the surface.
Direct formulation (Eq. direct) in P1:
  [ M/2 + K_L    -V_L     ]
  [ M/2 - K_Y    e12 V_Y  ],  rhs [int phi_i f; 0].
Reaction potential (Eq. phi_reac) and energy (Eq. energy) as in bem.py, with
the P1 fields evaluated at the quadrature points.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import lib
from .bem import geometry, kahan_sum, regular_rule
from .closed_forms import KCAL
from .kernels import LAPLACE, direct_sum


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def tri_lin(x, v):
    """(int_T lambda_b / |x - y|, int_T lambda_b (x - y).n / |x - y|^3), b = 0..2."""
    sl = np.zeros(3)
    dl = np.zeros(3)
    lib().or_tri_lin(_p(np.ascontiguousarray(x, float)), *[_p(np.ascontiguousarray(t, float)) for t in v],
                     _p(sl), _p(dl))
    return sl, dl


def assemble_p1(verts, tris, nq, kappa, L_outer=6, n_outer=4, n_inner=4):
    """Dense P1 Galerkin matrices, dict with VL, KL, VY, KY, WL, WY, KpL, KpY
    (K' = K^T) and the mass matrix M, each [nv, nv]."""
    V = np.ascontiguousarray(verts, dtype=np.float64)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    nv = len(V)
    names = ("VL", "KL", "VY", "KY", "WL", "WY")
    mats = {k: np.zeros((nv, nv)) for k in names}
    rc = lib().or_assemble_p1(nv, _p(V), len(F), _p(F), int(nq), float(kappa), int(L_outer), int(n_outer),
                              int(n_inner), *[_p(mats[k]) for k in names])
    if rc != 0:
        raise ValueError("assembly failed")
    mats["KpL"] = mats["KL"].T.copy()
    mats["KpY"] = mats["KY"].T.copy()
    mats["M"] = mass_p1(V, F)
    return mats


def pair_blocks(verts, tris, pairs, nq, kappa, minus_regular=True, L_outer=6):
    """P1 blocks [npairs][4][3][3] (V_L, K_L, V_Y, K_Y; test vertex, trial
    vertex) of the triangle pairs (i, j), optionally minus their regular
    product-rule part (oracle.c or_pair_p1)."""
    V = np.ascontiguousarray(verts, dtype=np.float64)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    out = np.zeros((len(pairs), 4, 3, 3))
    buf = np.zeros(36)
    for k, (i, j) in enumerate(pairs):
        ti = np.ascontiguousarray(F[i])
        tj = np.ascontiguousarray(F[j])
        if lib().or_pair_p1(_p(V), _p(ti), _p(tj), int(nq), float(kappa), int(L_outer), 4, 4,
                            1 if minus_regular else 0, _p(buf)) != 0:
            raise ValueError("pair block failed")
        out[k] = buf.reshape(4, 3, 3)
    return out


def mass_p1(verts, tris):
    """P1 mass matrix: sum over triangles of |T| (1 + delta_ab) / 12."""
    _, area = geometry(verts, tris)
    nv = len(verts)
    M = np.zeros((nv, nv))
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for t, f in enumerate(np.asarray(tris)):
        M[np.ix_(f, f)] += area[t] * loc
    return M


def lumped_mass(verts, tris):
    """Row sums of the P1 mass matrix (|T|/3 per incident triangle)."""
    return mass_p1(verts, tris).sum(axis=1)


def quad_p1(verts, tris, nq):
    """Quadrature points, weights w_k |T|, unit normals, triangle index and
    the barycentric coordinates (weights of the triangle's three vertices)."""
    V = np.asarray(verts, dtype=np.float64)
    F = np.asarray(tris)
    L, W = regular_rule(nq)
    n, area = geometry(V, F)
    P = np.einsum("kc,icd->ikd", L, V[F]).reshape(-1, 3)
    w = (W[None, :] * area[:, None]).ravel()
    nrm = np.repeat(n, nq, axis=0)
    tri = np.repeat(np.arange(len(F)), nq)
    lam = np.tile(L, (len(F), 1))
    return P, w, nrm, tri, lam


def to_points(verts, tris, nq, u):
    """Values of the P1 function with vertex values u at the quadrature points."""
    P, w, nrm, tri, lam = quad_p1(verts, tris, nq)
    F = np.asarray(tris)
    return (lam * np.asarray(u)[F[tri]]).sum(axis=1)


def test_integrals(verts, tris, nq, fpts):
    """int phi_i f over the surface with the nq-point rule (f at the points)."""
    P, w, nrm, tri, lam = quad_p1(verts, tris, nq)
    F = np.asarray(tris)
    b = np.zeros(len(verts))
    for a in range(3):
        np.add.at(b, F[tri, a], w * lam[:, a] * fpts)
    return b


def coulomb_rhs(verts, tris, nq, atoms, charges, eps):
    """[int phi_i f; int phi_i df/dn_x], f = sum_k q_k / (4 pi eps |x - r_k|)."""
    P, w, nrm, tri, lam = quad_p1(verts, tris, nq)
    f, dfdn = direct_sum(LAPLACE, 0.0, atoms, q=np.asarray(charges, dtype=np.float64) / eps, tgt=P,
                         tgt_n=nrm, want_dn=True)
    return test_integrals(verts, tris, nq, f), test_integrals(verts, tris, nq, dfdn)


FORMULATIONS = ("direct", "exterior", "interior")


def system_matrix(mats, eps_in, eps_out, formulation):
    """The 2x2 block Galerkin matrix of the formulation."""
    e12 = eps_in / eps_out
    e21 = eps_out / eps_in
    M = mats["M"]
    if formulation == "interior":
        return np.block([[0.5 * (1 + e21) * M - (e21 * mats["KY"] - mats["KL"]), mats["VY"] - mats["VL"]],
                         [mats["WY"] - mats["WL"], 0.5 * (1 + e12) * M + e12 * mats["KpY"] - mats["KpL"]]])
    if formulation == "exterior":
        return np.block([[0.5 * (1 + e12) * M - (mats["KY"] - e12 * mats["KL"]), mats["VY"] - mats["VL"]],
                         [e12 * (mats["WY"] - mats["WL"]), 0.5 * (1 + e12) * M + e12 * mats["KpY"] - mats["KpL"]]])
    if formulation == "direct":
        return np.block([[0.5 * M + mats["KL"], -mats["VL"]], [0.5 * M - mats["KY"], e12 * mats["VY"]]])
    raise ValueError(formulation)


def system_rhs(verts, tris, nq, atoms, charges, eps_in, eps_out, formulation):
    if formulation == "direct":
        b0, _ = coulomb_rhs(verts, tris, nq, atoms, charges, eps_in)
        return np.concatenate([b0, np.zeros(len(verts))])
    eps = eps_in if formulation == "interior" else eps_out
    b0, b1 = coulomb_rhs(verts, tris, nq, atoms, charges, eps)
    return np.concatenate([b0, b1])


def interior_fields(x, eps_in, eps_out, formulation):
    """(phi_1, dphi_1/dn) at the vertices from the solution vector."""
    nv = len(x) // 2
    phi, dphi = x[:nv], x[nv:]
    if formulation == "exterior":
        dphi = dphi * (eps_out / eps_in)
    return phi, dphi


def phi_reac(verts, tris, nq, phi, dphi, atoms):
    """Eq. phi_reac at the atoms: -K_L[phi_1] + V_L[dphi_1] with the nq-point rule."""
    P, w, nrm, tri, lam = quad_p1(verts, tris, nq)
    ph = to_points(verts, tris, nq, phi)
    dp = to_points(verts, tris, nq, dphi)
    return direct_sum(LAPLACE, 0.0, P, q=w * dp, dip=-w * ph, src_n=nrm, tgt=atoms)


def solve_energy(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, formulation, mats=None):
    """Dense LU solve of the formulation; (energy kcal/mol, phi_1, dphi_1, x, mats)."""
    if mats is None:
        mats = assemble_p1(verts, tris, nq, kappa)
    A = system_matrix(mats, eps_in, eps_out, formulation)
    b = system_rhs(verts, tris, nq, atoms, charges, eps_in, eps_out, formulation)
    x = np.linalg.solve(A, b)
    phi, dphi = interior_fields(x, eps_in, eps_out, formulation)
    pr = phi_reac(verts, tris, nq, phi, dphi, np.asarray(atoms, dtype=np.float64).reshape(-1, 3))
    e = 0.5 * kahan_sum(np.asarray(charges) * pr) * 4.0 * np.pi * KCAL
    return e, phi, dphi, x, mats


def preconditioned_spectrum(mats, verts, tris, eps_in, eps_out, formulation, lumped=False):
    """Eigenvalues of M^{-1} A with M = diag(M1, M1) the P1 mass matrix (or its
    lumped diagonal), the matrix whose clustering the paper discusses."""
    A = system_matrix(mats, eps_in, eps_out, formulation)
    nv = len(verts)
    if lumped:
        d = np.concatenate([lumped_mass(verts, tris)] * 2)
        B = A / d[:, None]
    else:
        Mb = np.block([[mats["M"], np.zeros((nv, nv))], [np.zeros((nv, nv)), mats["M"]]])
        B = np.linalg.solve(Mb, A)
    return np.linalg.eigvals(B)
