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
