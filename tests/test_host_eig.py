"""CPU checks of the library's host eigensolver (Householder
tridiagonalisation + implicit symmetric QR with Wilkinson shifts), which the
operator precomputation uses for the factored pseudo-inverses of the check ->
equivalent solves.  Runs on the host only: no GPU needed."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pb():
    import paper_2103_01048_gb300 as pb
    return pb


def surface(p):
    """Boundary points of the p x p x p grid on [-1, 1]^3 (the KIFMM surface)."""
    g = np.linspace(-1.0, 1.0, p)
    pts = [(x, y, z) for x in g for y in g for z in g if max(abs(x), abs(y), abs(z)) == 1.0]
    return np.array(pts)


def kifmm_gram(p, kappa, r=1.0):
    """K^T K of the upward check -> equivalent matrix (check surface at
    2.95 r, equivalent surface at 1.05 r), the matrix the precomputation
    decomposes: condition number up to ~1e20 at p = 10."""
    s = surface(p)
    d = np.linalg.norm(2.95 * r * s[:, None, :] - 1.05 * r * s[None, :, :], axis=2)
    K = np.exp(-kappa * d) / (4 * np.pi * d)
    return K.T @ K


def check(pb, A, tol):
    """Backward-stable decomposition: orthonormal V, A = V diag(w) V^T and
    the LAPACK spectrum, both within tol ||A||_2."""
    w, V = pb._test_sym_eig(A)
    n = len(A)
    ref = np.linalg.eigvalsh(A)
    scale = max(np.abs(ref).max(), 1e-300)
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    assert np.abs(V @ np.diag(w) @ V.T - A).max() < tol * scale
    assert np.abs(np.sort(w) - ref).max() < tol * scale
    return w, V


@pytest.mark.parametrize("n", [1, 2, 3, 17, 160])
def test_random_symmetric(pb, n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    check(pb, B + B.T, 1e-13)


def test_repeated_and_zero_eigenvalues(pb):
    """A diagonal block (already tridiagonal, zero off-diagonals), a
    repeated eigenvalue and an exactly singular matrix."""
    check(pb, np.diag([3.0, 1.0, 1.0, 0.0, -2.0]), 1e-15)
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    w = np.concatenate([np.full(20, 2.0), np.zeros(10), rng.uniform(-1, 1, 10)])
    check(pb, (Q * w) @ Q.T, 1e-13)


@pytest.mark.parametrize("p,kappa", [(4, 0.0), (6, 0.125), (10, 0.125)])
def test_kifmm_gram(pb, p, kappa):
    """The ill-conditioned Gram matrices of the precomputation (n_e = 56,
    152, 488 surface points): reconstruction and spectrum within 1e-13
    ||A||_2 (measured 2e-16 .. 4e-15, LAPACK's own reconstruction 7e-16 ..
    1.2e-15)."""
    A = kifmm_gram(p, kappa)
    assert len(A) == 6 * (p - 1) ** 2 + 2
    check(pb, A, 1e-13)
