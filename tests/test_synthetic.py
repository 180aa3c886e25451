"""Seeded input generators (no method arithmetic): the sphere meshes used by
the refinement study, the Born ion and the virus-scale shell are closed,
2-manifold, outward oriented and of the stated sizes."""
import os

import numpy as np
import pytest

import synthetic


def _check_closed_outward(V, F, min_volume):
    # every undirected edge in exactly two faces, with opposite orientations
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    und = np.sort(e, axis=1)
    _, cnt = np.unique(und, axis=0, return_counts=True)
    assert np.all(cnt == 2)
    _, dcnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(dcnt == 1)
    p0, p1, p2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0
    assert vol > min_volume          # positive: normals point outward
    # Euler characteristic of a sphere
    assert len(V) - len(und) // 2 + len(F) == 2


@pytest.mark.parametrize("level", [0, 1, 3, 4])
def test_octasphere(level):
    V, F = synthetic.octasphere(level, 4.0)
    assert len(F) == 8 * 4 ** level and len(V) == 4 * 4 ** level + 2
    assert np.allclose(np.linalg.norm(V, axis=1), 4.0)
    ball = 4.0 / 3.0 * np.pi * 4.0 ** 3
    _check_closed_outward(V, F, 0.95 * ball if level >= 3 else 0.0)


@pytest.mark.parametrize("level", [1, 3])
def test_icosphere(level):
    V, F = synthetic.icosphere(level, 2.0)
    assert len(F) == 20 * 4 ** level and len(V) == 10 * 4 ** level + 2
    _check_closed_outward(V, F, 0.8 * 4.0 / 3.0 * np.pi * 2.0 ** 3)


def test_cube_sphere_counts_and_closure():
    V, F = synthetic.cube_sphere(6, 3.0, outward=True, amp=0.0, seed=1)
    assert len(F) == 12 * 6 * 6
    assert np.allclose(np.linalg.norm(V, axis=1), 3.0)
    _check_closed_outward(V, F, 0.8 * 4.0 / 3.0 * np.pi * 3.0 ** 3)


def test_binding_complex_default_meshes_match_golden():
    """The default (porous) complexes are unchanged: their meshes hash to
    the values recorded with the oracle's binding energies."""
    import hashlib
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "binding_small.json")))
    c = gold["complexes"][0]
    cx = synthetic.binding_complex(c["n_rec"], c["n_lig"], seed=10 + c["n_rec"], spacing=1.0)
    for k in ("cplx", "rec", "lig"):
        V, T = cx["surf"][k]
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(V, np.float64).tobytes())
        h.update(np.ascontiguousarray(T, np.int32).tobytes())
        assert len(T) == c[k]["triangles"]
        assert h.hexdigest()[:16] == c[k]["mesh_sha256_16"], k


@pytest.mark.parametrize("n", [5, 20, 500, 2000])
def test_fcc_fill_radius(n):
    """The dense complexes' balls: a radius at most 0.05 A beyond the n-th
    nearest FCC site, so the ball holds the n atoms with (almost) no empty
    sites."""
    r = synthetic.fcc_fill_radius(n)
    xyz, _, _ = synthetic.fcc_ball_atoms(n, r, 2.85, 0.0, seed=1)
    assert len(xyz) == n
    # brute force: distance of the n-th nearest FCC site (a = 2.85 sqrt 2)
    a = 2.85 * 2 ** 0.5
    g = np.arange(-12, 13)
    base = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * a
    offs = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    rho = np.sort(np.linalg.norm((base[:, None] + offs[None]).reshape(-1, 3), axis=1))
    assert rho[n - 1] < r <= rho[n - 1] + 0.05 + 1e-12
