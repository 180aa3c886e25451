"""P0 Galerkin boundary-element oracle for the direct formulation.

Test infrastructure only.

Discretisation (Sec. "An introduction to Bempp"): piecewise-constant (P0)
trial and test functions on flat triangles, A_ij = int_Ti int_Tj k(x,y),
b_i = int_Ti f.  Regular pairs use the product of the nq-point triangle rule
(the G entries of Eq. bempp_fmm_matvec); identical or vertex-sharing pairs use
a semi-analytic rule (analytic inner integral, fine outer rule), see oracle.c.

Direct formulation (Eq. direct), Galerkin form with M the P0 mass matrix
(diagonal of the triangle areas):
    [ M/2 + K_L        -V_L          ] [phi ]   [ b ]
    [ M/2 - K_Y   (eps1/eps2) V_Y    ] [dphi] = [ 0 ],
    b_i = int_Ti sum_k q_k / (4 pi eps1 |x - r_k|).
Reaction potential (Eq. phi_reac): phi_reac(r) = -K_L[phi](r) + V_L[dphi](r),
energy (Eq. energy): dG = 1/2 sum_k q_k phi_reac(r_k), times 4 pi C for
kcal/mol (C = 332.0637).

Readings: the 3-point rule is the interior degree-2 rule (2/3,1/6,1/6),
the 6-point rule is Dunavant's degree-4 rule; "adjacent" means sharing at
least one vertex.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import lib
from .kernels import LAPLACE, direct_sum
from .closed_forms import KCAL


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def geometry(verts, tris):
    """Unit normals n = (v1-v0)x(v2-v0)/|.| and areas of each triangle."""
    V = np.asarray(verts, dtype=np.float64)
    F = np.asarray(tris)
    e1 = V[F[:, 1]] - V[F[:, 0]]
    e2 = V[F[:, 2]] - V[F[:, 0]]
    c = np.cross(e1, e2)
    a = np.linalg.norm(c, axis=1)
    return c / a[:, None], 0.5 * a


def regular_rule(nq):
    L = np.zeros(3 * nq)
    W = np.zeros(nq)
    if lib().or_regular_rule(int(nq), _p(L), _p(W)) != 0:
        raise ValueError("nq must be 1, 3 or 6")
    return L.reshape(nq, 3), W


def quad_points(verts, tris, nq):
    """Quadrature points x_a (a = i*nq + k), their weights w_k |T_i|, normals
    of their triangle, and the triangle index."""
    V = np.asarray(verts, dtype=np.float64)
    F = np.asarray(tris)
    L, W = regular_rule(nq)
    n, area = geometry(V, F)
    P = np.einsum("kc,icd->ikd", L, V[F]).reshape(-1, 3)
    w = (W[None, :] * area[:, None]).ravel()
    nrm = np.repeat(n, nq, axis=0)
    tri = np.repeat(np.arange(len(F)), nq)
    return P, w, nrm, tri


def assemble_p0(verts, tris, nq, kappa, L_outer=6, n_outer=4, n_inner=4):
    """Dense P0 Galerkin matrices (V_L, K_L, V_Y, K_Y), each [nt, nt]."""
    V = np.ascontiguousarray(verts, dtype=np.float64)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    nt = len(F)
    mats = [np.zeros((nt, nt)) for _ in range(4)]
    rc = lib().or_assemble_p0(len(V), _p(V), nt, _p(F), int(nq), float(kappa),
                              int(L_outer), int(n_outer), int(n_inner), *[_p(m) for m in mats])
    if rc != 0:
        raise ValueError("assembly failed")
    return tuple(mats)


def direct_matrix(mats, area, eps_in, eps_out):
    """The 2x2 block matrix of Eq. direct in P0 Galerkin form."""
    VL, KL, VY, KY = mats
    M = np.diag(area)
    return np.block([[0.5 * M + KL, -VL], [0.5 * M - KY, (eps_in / eps_out) * VY]])


def rhs(verts, tris, nq, atoms, charges, eps_in):
    """b_i = int_Ti sum_k q_k/(4 pi eps1 |x - r_k|) with the nq-point rule."""
    P, w, _, tri = quad_points(verts, tris, nq)
    f = direct_sum(LAPLACE, 0.0, atoms, q=np.asarray(charges, dtype=np.float64) / eps_in, tgt=P)
    b = np.zeros(len(tris))
    np.add.at(b, tri, w * f)
    return b


def solve_direct(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, mats=None):
    """Dense LU solve of Eq. direct; returns (phi, dphi, mats)."""
    _, area = geometry(verts, tris)
    if mats is None:
        mats = assemble_p0(verts, tris, nq, kappa)
    A = direct_matrix(mats, area, eps_in, eps_out)
    nt = len(tris)
    b = np.concatenate([rhs(verts, tris, nq, atoms, charges, eps_in), np.zeros(nt)])
    x = np.linalg.solve(A, b)
    return x[:nt], x[nt:], mats


def phi_reac(verts, tris, nq, phi, dphi, atoms):
    """Eq. phi_reac at the atoms: -K_L[phi] + V_L[dphi] with the nq-point rule."""
    P, w, nrm, tri = quad_points(verts, tris, nq)
    return direct_sum(LAPLACE, 0.0, P, q=w * np.asarray(dphi)[tri], dip=-w * np.asarray(phi)[tri],
                      src_n=nrm, tgt=atoms)


def kahan_sum(v):
    s = 0.0
    c = 0.0
    for x in np.asarray(v, dtype=np.float64).ravel():
        y = x - c
        t = s + y
        c = (t - s) - y
        s = t
    return s


def solvation_energy(charges, phir):
    """Eq. energy in kcal/mol: 1/2 sum q phi_reac * 4 pi C (Kahan sum)."""
    return 0.5 * kahan_sum(np.asarray(charges) * phir) * 4.0 * np.pi * KCAL


def solve_energy(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, mats=None):
    phi, dphi, mats = solve_direct(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, mats)
    pr = phi_reac(verts, tris, nq, phi, dphi, atoms)
    return solvation_energy(charges, pr), phi, dphi, mats


def charge_response(verts, tris, nq, atoms, eps_in, eps_out, kappa, mats):
    """Matrix R with phi_reac(r_k) = sum_l R_kl q_l (Eq. phi_reac after
    Eq. direct), built column by column from its definition
    R = E A^{-1} B: B maps charges to the right-hand side, E maps the surface
    solution to the reaction potential at the atoms."""
    atoms = np.asarray(atoms, dtype=np.float64).reshape(-1, 3)
    na = len(atoms)
    nt = len(tris)
    P, w, nrm, tri = quad_points(verts, tris, nq)
    _, area = geometry(verts, tris)
    A = direct_matrix(mats, area, eps_in, eps_out)
    B = np.zeros((2 * nt, na))
    E = np.zeros((na, 2 * nt))
    for k in range(na):
        d = P - atoms[k]
        r = np.linalg.norm(d, axis=1)
        g = 1.0 / (4 * np.pi * r)
        np.add.at(B[:nt, k], tri, w * g / eps_in)
        # dg/dn_y at y = x_b for target r_k: (r_k - x_b).n_b / (4 pi r^3)
        dgdn = ((atoms[k] - P) * nrm).sum(axis=1) / (4 * np.pi * r ** 3)
        np.add.at(E[k, :nt], tri, -w * dgdn)
        np.add.at(E[k, nt:], tri, w * g)
    return E @ np.linalg.solve(A, B)


def energy_grad_q(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, mats):
    """dE/dq = 1/2 (R + R^T) q in kcal/mol/e (E = 1/2 q^T R q * 4 pi C)."""
    R = charge_response(verts, tris, nq, atoms, eps_in, eps_out, kappa, mats)
    q = np.asarray(charges, dtype=np.float64)
    return 0.5 * (R + R.T) @ q * 4.0 * np.pi * KCAL


def energy_grad_x_fd(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, mats, h=1e-4, idx=None):
    """dE/dr_k by central finite differences of the dense-LU energy, the
    surface held fixed; idx selects (atom, axis) components (default all)."""
    atoms = np.asarray(atoms, dtype=np.float64).reshape(-1, 3)
    comps = idx if idx is not None else [(k, c) for k in range(len(atoms)) for c in range(3)]
    out = {}
    for k, c in comps:
        ap = atoms.copy(); ap[k, c] += h
        am = atoms.copy(); am[k, c] -= h
        ep, *_ = solve_energy(verts, tris, nq, ap, charges, eps_in, eps_out, kappa, mats=mats)
        em, *_ = solve_energy(verts, tris, nq, am, charges, eps_in, eps_out, kappa, mats=mats)
        out[(k, c)] = (ep - em) / (2 * h)
    return out


# ---------------------------------------------------------------------------
# Matrix-free solve (sizes beyond the dense LU)
# ---------------------------------------------------------------------------

def vertex_sharing_pairs(tris):
    """All ordered pairs (i, j) of triangles sharing at least one vertex
    (i == j included), as two index arrays."""
    F = np.asarray(tris)
    from collections import defaultdict
    inc = defaultdict(list)
    for t, f in enumerate(F):
        for v in f:
            inc[int(v)].append(t)
    I, J = [], []
    for i, f in enumerate(F):
        js = sorted(set(t for v in f for t in inc[int(v)]))
        I += [i] * len(js)
        J += js
    return np.array(I), np.array(J)


def singular_corrections(verts, tris, nq, kappa, L_outer=6):
    """Sparse P0 corrections of the vertex-sharing pairs, one scipy CSR
    matrix per kernel (V_L, K_L, V_Y, K_Y): the semi-analytic entry (as in
    assemble_p0) minus the same entry under the nq x nq regular product rule
    (what the point sums already hold); oracle.c or_corrections_p0."""
    import scipy.sparse as sp
    V = np.ascontiguousarray(verts, dtype=np.float64)
    F = np.ascontiguousarray(tris, dtype=np.int32)
    I, J = vertex_sharing_pairs(F)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.zeros((len(I), 4))
    if lib().or_corrections_p0(len(V), _p(V), len(F), _p(F), len(I), _p(I), _p(J), int(nq), float(kappa),
                               int(L_outer), 4, 4, _p(out)) != 0:
        raise ValueError("corrections failed")
    nt = len(F)
    return [sp.csr_matrix((out[:, op], (I, J)), shape=(nt, nt)) for op in range(4)]


def matvec_free(verts, tris, nq, kappa, eps_in, eps_out, corr=None):
    """The direct-formulation matrix of Eq. direct as a function x -> A x:
    point sums of the kernels over all quadrature-point pairs (FP64 direct
    sums, r = 0 excluded) tested with the P0 functions, plus the sparse
    singular corrections, plus the mass terms."""
    from .kernels import YUKAWA
    P, w, nrm, tri = quad_points(verts, tris, nq)
    _, area = geometry(verts, tris)
    nt = len(tris)
    if corr is None:
        corr = singular_corrections(verts, tris, nq, kappa)
    cVL, cKL, cVY, cKY = corr
    e12 = eps_in / eps_out

    def test(f):
        out = np.zeros(nt)
        np.add.at(out, tri, w * f)
        return out

    def A(x):
        phi, dphi = x[:nt], x[nt:]
        # V_L dphi and K_L phi from one Laplace sum, V_Y and K_Y from one Yukawa sum
        pL = direct_sum(LAPLACE, 0.0, P, q=-w * dphi[tri], dip=w * phi[tri], src_n=nrm)
        pY = direct_sum(YUKAWA, kappa, P, q=e12 * w * dphi[tri], dip=-w * phi[tri], src_n=nrm)
        r1 = test(pL) + cKL @ phi - cVL @ dphi + 0.5 * area * phi
        r2 = test(pY) - cKY @ phi + e12 * (cVY @ dphi) + 0.5 * area * phi
        return np.concatenate([r1, r2])
    return A


def gmres(A, b, tol=1e-10, max_iter=500, M=None):
    """Unrestarted GMRES from x0 = 0 (Arnoldi with modified Gram-Schmidt,
    Givens rotations), left preconditioner M (a function) if given; stops at
    ||M(b - A x)|| <= tol ||M b||.  Returns (x, iterations, relative residual)."""
    Mf = M if M is not None else (lambda v: v)
    r0 = Mf(b)
    beta = np.linalg.norm(r0)
    n = len(b)
    if beta == 0.0:
        return np.zeros(n), 0, 0.0
    Vb = [r0 / beta]
    H = np.zeros((max_iter + 1, max_iter))
    cs, sn = np.zeros(max_iter), np.zeros(max_iter)
    g = np.zeros(max_iter + 1)
    g[0] = beta
    k = 0
    for k in range(max_iter):
        w_ = Mf(A(Vb[k]))
        for i in range(k + 1):
            H[i, k] = np.dot(Vb[i], w_)
            w_ = w_ - H[i, k] * Vb[i]
        H[k + 1, k] = np.linalg.norm(w_)
        for i in range(k):
            a_, b_ = H[i, k], H[i + 1, k]
            H[i, k], H[i + 1, k] = cs[i] * a_ + sn[i] * b_, -sn[i] * a_ + cs[i] * b_
        rr = np.hypot(H[k, k], H[k + 1, k])
        cs[k], sn[k] = H[k, k] / rr, H[k + 1, k] / rr
        H[k, k], H[k + 1, k] = rr, 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        if H[k + 1, k] == 0.0 and rr == 0.0:
            break
        Vb.append(w_ / np.linalg.norm(w_) if np.linalg.norm(w_) > 0 else w_)
        if abs(g[k + 1]) <= tol * beta:
            k += 1
            break
    else:
        k = max_iter
    y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
    x = np.zeros(n)
    for i in range(k):
        x += y[i] * Vb[i]
    return x, k, abs(g[k]) / beta


def solve_energy_free(verts, tris, nq, atoms, charges, eps_in, eps_out, kappa, tol=1e-10, max_iter=500):
    """Eq. direct by matrix-free GMRES (direct sums, exact singular
    corrections), preconditioned by the per-triangle 2x2 blocks of the
    diagonal entries; then Eq. phi_reac and Eq. energy.  Returns
    (energy, phi, dphi, iterations, residual)."""
    nt = len(tris)
    corr = singular_corrections(verts, tris, nq, kappa)
    A = matvec_free(verts, tris, nq, kappa, eps_in, eps_out, corr)
    _, area = geometry(verts, tris)
    e12 = eps_in / eps_out
    d11 = corr[1].diagonal() + 0.5 * area
    d12 = -corr[0].diagonal()
    d21 = -corr[3].diagonal() + 0.5 * area
    d22 = e12 * corr[2].diagonal()
    # (the self corrections stand in for the diagonal entries: only a
    # preconditioner, it does not change the solution)
    det = d11 * d22 - d12 * d21

    def M(v):
        a, c = v[:nt], v[nt:]
        return np.concatenate([(d22 * a - d12 * c) / det, (-d21 * a + d11 * c) / det])
    b = np.concatenate([rhs(verts, tris, nq, atoms, charges, eps_in), np.zeros(nt)])
    x, it, res = gmres(A, b, tol=tol, max_iter=max_iter, M=M)
    phi, dphi = x[:nt], x[nt:]
    pr = phi_reac(verts, tris, nq, phi, dphi, atoms)
    return solvation_energy(charges, pr), phi, dphi, it, res
