"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: point clouds, meshes, densities and atom
layouts.  It contains none of the method's arithmetic (no Green's functions,
no quadrature, no tree, no operators), so that the oracle and the CUDA path
stay independent while being fed identical arrays.

Workload shapes follow the paper's experiments (Sec. "Performance study",
Table of 1A7M meshes; the Zika capsid; the Kirkwood sphere of Sec. "Mesh
refinement study using an analytical solution"), with synthetic geometry
standing in for the PDB/Nanoshaper meshes, which are not available here.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "bumpy_sphere_points",
    "uniform_densities",
    "icosphere",
    "random_subsample",
    "fcc_ball_atoms",
]


def bumpy_sphere_points(n: int, amp: float = 0.05, nbumps: int = 32,
                        width: float = 0.3, seed: int = 0):
    """Points on a unit sphere with an additive smooth random radial bump.

    Direction u = normalised Gaussian 3-vector; radius r = 1 + amp * f(u) with
    f(u) = sum_k w_k exp(-|u - c_k|^2 / (2 width^2)), c_k uniform on the
    sphere, w_k ~ U[-1, 1], normalised so that max |f| over the points is 1.

    Returns (xyz float32 [n,3], normals float32 [n,3]); the normals are the
    radial unit vectors u (the kernels only need unit normals).
    """
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = rng.standard_normal((nbumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    w = rng.uniform(-1.0, 1.0, nbumps)
    f = np.zeros(n)
    for k in range(nbumps):
        d2 = ((u - c[k]) ** 2).sum(axis=1)
        f += w[k] * np.exp(-d2 / (2.0 * width * width))
    fmax = np.abs(f).max() if n else 1.0
    if fmax > 0:
        f /= fmax
    r = 1.0 + amp * f
    xyz = (u * r[:, None]).astype(np.float32)
    nrm = u.astype(np.float32)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(nrm)


def uniform_densities(n: int, seed: int = 1, lo: float = -1.0, hi: float = 1.0):
    """FP32 densities uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n).astype(np.float32)


def random_subsample(n: int, k: int, seed: int = 2):
    """Sorted indices of a seeded subsample of k out of n (without replacement)."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


def octasphere(level: int, radius: float = 1.0):
    """Octahedron subdivided `level` times (each triangle into four at its
    edge midpoints), vertices projected to the sphere: nt = 8 * 4**level
    (512, 2,048, 8,192, 32,768, 131,072 for levels 3-7, the element counts of
    the off-centre-charge sphere refinement study).  Returns (verts float64
    [nv,3], tris int32 [nt,3]), counter-clockwise seen from outside."""
    v = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    f = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    verts = [np.array(q, dtype=np.float64) for q in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius
    F = np.array(faces, dtype=np.int32)
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    flip = (nrm * (p0 + p1 + p2)).sum(axis=1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return np.ascontiguousarray(V), np.ascontiguousarray(F)


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron subdivided `level` times, vertices projected to the sphere.

    Returns (verts float64 [nv,3], tris int32 [nt,3]) with counter-clockwise
    ordering seen from outside (outward normals).  nt = 20 * 4**level and
    nv = 10 * 4**level + 2.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius
    F = np.array(faces, dtype=np.int32)
    # orient outward: the centroid direction must agree with the face normal
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    flip = (nrm * (p0 + p1 + p2)).sum(axis=1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return np.ascontiguousarray(V), np.ascontiguousarray(F)


def fcc_ball_atoms(natoms: int, ball_radius: float, nn_dist: float,
                   jitter: float, seed: int = 3,
                   rmin: float = 1.2, rmax: float = 2.0, qmax: float = 0.8,
                   shell: tuple | None = None):
    """Atoms on a jittered FCC lattice clipped to a ball (or a spherical shell).

    A seeded random subset of exactly `natoms` lattice sites is taken, each
    moved by a uniform jitter of at most `jitter` per axis.  Radii are uniform
    in [rmin, rmax]; charges uniform in [-qmax, qmax] shifted to zero net
    charge.  Returns (xyz float64 [n,3], radii float64 [n], q float64 [n]).
    """
    rng = np.random.default_rng(seed)
    a = nn_dist * 2.0 ** 0.5           # cubic cell edge of the FCC lattice
    outer = ball_radius if shell is None else shell[1]
    m = int(np.ceil(outer / a)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) * a
    offs = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    sites = (base[:, None, :] + offs[None, :, :]).reshape(-1, 3)
    rho = np.linalg.norm(sites, axis=1)
    if shell is None:
        keep = rho <= ball_radius
    else:
        keep = (rho >= shell[0]) & (rho <= shell[1])
    sites = sites[keep]
    if len(sites) < natoms:
        raise ValueError(f"only {len(sites)} lattice sites for {natoms} atoms")
    idx = rng.choice(len(sites), size=natoms, replace=False)
    xyz = sites[np.sort(idx)] + rng.uniform(-jitter, jitter, (natoms, 3))
    radii = rng.uniform(rmin, rmax, natoms)
    q = rng.uniform(-qmax, qmax, natoms)
    q -= q.mean()
    return xyz, radii, q


def gaussian_surface(xyz, radii, spacing, level=1.0, cutoff=3.0, pad=None):
    """Closed triangulation of the isosurface F(x) = level of the Gaussian
    density F(x) = sum_k exp(-(|x - r_k|^2 / R_k^2 - 1)), terms cut off beyond
    cutoff * R_k, by marching tetrahedra on a regular grid of the given
    spacing (each cube split into six tetrahedra around its main diagonal, so
    neighbouring cubes share faces and the surface is watertight).  Grid
    values within 1e-6 of `level` are nudged off it so that no vertex sits on
    a grid node.  Triangles are oriented with normals pointing to lower F
    (out of the molecule).  Returns (verts float64 [nv,3], tris int32 [nt,3]).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    if pad is None:
        pad = 2.0 * radii.max() + 2 * spacing
    lo = xyz.min(axis=0) - pad
    hi = xyz.max(axis=0) + pad
    n = np.ceil((hi - lo) / spacing).astype(int) + 1
    gx = [lo[a] + spacing * np.arange(n[a]) for a in range(3)]
    F = np.zeros(tuple(n))
    for k in range(len(xyz)):
        rc = cutoff * radii[k]
        sl = []
        for a in range(3):
            i0 = max(0, int(np.floor((xyz[k, a] - rc - lo[a]) / spacing)))
            i1 = min(n[a], int(np.ceil((xyz[k, a] + rc - lo[a]) / spacing)) + 1)
            sl.append(slice(i0, i1))
        X, Y, Z = np.meshgrid(gx[0][sl[0]], gx[1][sl[1]], gx[2][sl[2]], indexing="ij")
        d2 = (X - xyz[k, 0]) ** 2 + (Y - xyz[k, 1]) ** 2 + (Z - xyz[k, 2]) ** 2
        term = np.exp(-(d2 / radii[k] ** 2 - 1.0))
        term[d2 > rc * rc] = 0.0
        F[sl[0], sl[1], sl[2]] += term
    G = F - level
    G[np.abs(G) < 1e-6] = 1e-6
    inside = G > 0
    # six tetrahedra of the unit cube sharing the diagonal (0,0,0)-(1,1,1)
    corners = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                        [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]])
    tets = [(0, 1, 3, 7), (0, 3, 2, 7), (0, 2, 6, 7), (0, 6, 4, 7), (0, 4, 5, 7), (0, 5, 1, 7)]
    ci = np.stack(np.meshgrid(np.arange(n[0] - 1), np.arange(n[1] - 1), np.arange(n[2] - 1),
                              indexing="ij"), axis=-1).reshape(-1, 3)
    # keep cubes crossed by the surface
    cin = np.stack([inside[ci[:, 0] + c[0], ci[:, 1] + c[1], ci[:, 2] + c[2]] for c in corners], axis=1)
    cross = cin.any(axis=1) & ~cin.all(axis=1)
    ci = ci[cross]
    stride = np.array([n[1] * n[2], n[2], 1])
    vert_of_edge = {}
    verts = []
    tris = []

    def edge_vertex(a, b):
        key = (a, b) if a < b else (b, a)
        v = vert_of_edge.get(key)
        if v is None:
            ia = np.array(np.unravel_index(a, n))
            ib = np.array(np.unravel_index(b, n))
            ga, gb = G[tuple(ia)], G[tuple(ib)]
            # linear interpolation, kept off the grid nodes (no sliver triangles)
            t = min(0.98, max(0.02, ga / (ga - gb)))
            p = lo + spacing * (ia + t * (ib - ia))
            v = len(verts)
            verts.append(p)
            vert_of_edge[key] = v
        return v

    flat = G.ravel()
    for c in ci:
        base = c @ stride
        ids = [base + corners[m] @ stride for m in range(8)]
        for tet in tets:
            node = [ids[m] for m in tet]
            ins = [flat[v] > 0 for v in node]
            m = sum(ins)
            if m == 0 or m == 4:
                continue
            I = [v for v, s in zip(node, ins) if s]
            O = [v for v, s in zip(node, ins) if not s]
            if m == 1:
                faces = [(edge_vertex(I[0], O[0]), edge_vertex(I[0], O[1]), edge_vertex(I[0], O[2]))]
                ref = [(I[0], O[0])]
            elif m == 3:
                faces = [(edge_vertex(O[0], I[0]), edge_vertex(O[0], I[1]), edge_vertex(O[0], I[2]))]
                ref = [(I[0], O[0])]
            else:
                a, b = edge_vertex(I[0], O[0]), edge_vertex(I[0], O[1])
                c2, d = edge_vertex(I[1], O[1]), edge_vertex(I[1], O[0])
                faces = [(a, b, c2), (a, c2, d)]
                ref = [(I[0], O[0])]
            ia = np.array(np.unravel_index(ref[0][0], n), dtype=float)
            io = np.array(np.unravel_index(ref[0][1], n), dtype=float)
            outward = io - ia                      # from inside to outside
            for f in faces:
                p0, p1, p2 = verts[f[0]], verts[f[1]], verts[f[2]]
                nr = np.cross(p1 - p0, p2 - p0)
                tris.append(f if nr @ outward >= 0 else (f[0], f[2], f[1]))
    V = np.array(verts)
    T = np.array(tris, dtype=np.int32)
    return V, T


def synthetic_protein(natoms=2000, target_tris=80000, seed=3, ball_radius=20.0):
    """Atoms (jittered FCC in a ball, radii U[1.2, 2.0], charges U[-0.8, 0.8]
    with zero net charge) and their Gaussian surface with the grid spacing
    tuned so the triangle count is within 10% of target_tris.  Returns
    (verts, tris, xyz, radii, q, spacing)."""
    xyz, radii, q = fcc_ball_atoms(natoms, ball_radius, 2.85, 0.1, seed=seed)
    h = 0.7 * (80000.0 / target_tris) ** 0.5 * (ball_radius / 20.0)
    for _ in range(6):
        V, T = gaussian_surface(xyz, radii, h)
        ratio = len(T) / target_tris
        if 0.9 <= ratio <= 1.1:
            break
        h *= ratio ** 0.5
    return V, T, xyz, radii, q, h


def fcc_fill_radius(natoms, nn_dist=2.85, step=0.05):
    """Ball radius (a multiple of `step`, at most `step` beyond the
    natoms-th nearest site) whose FCC lattice of nearest-neighbour distance
    nn_dist holds at least natoms sites."""
    a = nn_dist * 2.0 ** 0.5
    r = (3 * natoms * (a ** 3 / 4) / (4 * np.pi)) ** (1 / 3) * 0.9
    m = int(np.ceil(2 * r / a)) + 2
    g = np.arange(-m, m + 1, dtype=np.float64)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) * a
    offs = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    rho = np.sort(np.linalg.norm((base[:, None, :] + offs[None, :, :]).reshape(-1, 3), axis=1))
    return float((np.floor(rho[natoms - 1] / step) + 1) * step)      # strictly beyond the natoms-th site


def binding_complex(n_rec, n_lig, seed=0, gap=4.5, spacing=0.7, dense=False):
    """A synthetic receptor-ligand complex: receptor atoms on a jittered FCC
    lattice in a ball sized for n_rec atoms, ligand in a small ball placed
    along a seeded random direction so that the closest receptor-ligand
    atom-centre distance is `gap` A.  Returns dict with the atoms, radii and
    charges of the receptor, the ligand and the complex, and the three
    Gaussian surfaces (verts, tris).  dense=False: balls 10% wider than the
    atoms need (a porous receptor, ~60% of the sites taken); dense=True: the
    smallest balls that hold the atoms (compact bodies like the synthetic
    protein's)."""
    rng = np.random.default_rng(seed)
    per_atom = 2.85 ** 3 / 2 ** 0.5          # FCC volume per site
    if dense:
        rr, rl = fcc_fill_radius(n_rec), fcc_fill_radius(n_lig)
    else:
        rr = (3 * n_rec * per_atom / (4 * np.pi)) ** (1 / 3) * 1.1 + 1.0
        rl = (3 * n_lig * per_atom / (4 * np.pi)) ** (1 / 3) * 1.1 + 1.0
    xr, radr, qr = fcc_ball_atoms(n_rec, rr, 2.85, 0.1, seed=seed + 1)
    xl, radl, ql = fcc_ball_atoms(n_lig, rl, 2.85, 0.1, seed=seed + 2)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    shift = rr + rl
    for _ in range(60):
        d = np.min(np.linalg.norm((xl + shift * u)[:, None, :] - xr[None, :, :], axis=2))
        shift += gap - d
        if abs(gap - d) < 1e-3:
            break
    xl = xl + shift * u
    xc = np.concatenate([xr, xl])
    radc = np.concatenate([radr, radl])
    qc = np.concatenate([qr, ql])
    out = dict(rec=(xr, radr, qr), lig=(xl, radl, ql), cplx=(xc, radc, qc))
    out["surf"] = {k: gaussian_surface(v[0], v[1], spacing) for k, v in
                   (("rec", out["rec"]), ("lig", out["lig"]), ("cplx", out["cplx"]))}
    return out


def cube_sphere(n, radius, outward=True, amp=0.0, seed=0):
    """Closed triangulated sphere from a cube with n x n cells per face,
    vertices projected radially (welded along the cube edges), radius
    modulated by 1 + amp * f(u) with the bump field of bumpy_sphere_points.
    12 n^2 triangles; normals point away from the centre if `outward`, else
    towards it.  Returns (verts float64 [nv,3], tris int32 [nt,3])."""
    g = np.arange(n + 1)
    I, J = np.meshgrid(g, g, indexing="ij")
    I = I.ravel(); J = J.ravel()
    faces_v = []
    for axis in range(3):
        for side in (0, n):
            v = np.zeros((len(I), 3), dtype=np.int64)
            a1, a2 = [a for a in range(3) if a != axis]
            v[:, axis] = side
            v[:, a1] = I
            v[:, a2] = J
            faces_v.append(v)
    allv = np.concatenate(faces_v)
    uniq, inv = np.unique(allv, axis=0, return_inverse=True)
    inv = inv.ravel()
    tris = []
    base = 0
    m = n + 1
    for f in range(6):
        idx = inv[base:base + m * m].reshape(m, m)
        a = idx[:-1, :-1].ravel(); b = idx[1:, :-1].ravel()
        c = idx[1:, 1:].ravel(); d = idx[:-1, 1:].ravel()
        tris.append(np.stack([a, b, c], axis=1))
        tris.append(np.stack([a, c, d], axis=1))
        base += m * m
    T = np.concatenate(tris).astype(np.int64)
    P = uniq.astype(np.float64) * (2.0 / n) - 1.0
    u = P / np.linalg.norm(P, axis=1, keepdims=True)
    r = np.full(len(u), float(radius))
    if amp:
        rng = np.random.default_rng(seed)
        c = rng.standard_normal((32, 3))
        c /= np.linalg.norm(c, axis=1, keepdims=True)
        w = rng.uniform(-1.0, 1.0, 32)
        fb = np.zeros(len(u))
        for k in range(32):
            fb += w[k] * np.exp(-((u - c[k]) ** 2).sum(axis=1) / (2 * 0.3 * 0.3))
        fb /= np.abs(fb).max()
        r = r * (1.0 + amp * fb)
    V = u * r[:, None]
    # orient every triangle consistently
    p0, p1, p2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    s = (np.cross(p1 - p0, p2 - p0) * (p0 + p1 + p2)).sum(axis=1)
    flip = (s < 0) if outward else (s > 0)
    T[flip] = T[flip][:, [0, 2, 1]]
    return np.ascontiguousarray(V), np.ascontiguousarray(T.astype(np.int32))


def virus_shell(n_atoms=1_600_000, r_in=230.0, r_out=270.0, n_face=645, seed=7):
    """Virus-scale capsid stand-in: atoms on a jittered FCC lattice in the
    shell r_in + 2 <= rho <= r_out - 2 (radii U[1.2, 2], charges U[-0.8, 0.8],
    zero net charge) inside a two-component closed surface: the outer wall at
    r_out (normals outward) and the inner wall at r_in (normals towards the
    centre, i.e. out of the solute), each a cube sphere of 12 n_face^2
    triangles with a 0.4% bump.  Returns (verts, tris, xyz, radii, q)."""
    xyz, radii, q = fcc_ball_atoms(n_atoms, r_out, 2.85, 0.1, seed=seed, shell=(r_in + 2.0, r_out - 2.0))
    Vo, To = cube_sphere(n_face, r_out, outward=True, amp=0.004, seed=seed + 1)
    Vi, Ti = cube_sphere(n_face, r_in, outward=False, amp=0.004, seed=seed + 2)
    V = np.concatenate([Vo, Vi])
    T = np.concatenate([To, Ti + len(Vo)]).astype(np.int32)
    return V, T, xyz, radii, q
