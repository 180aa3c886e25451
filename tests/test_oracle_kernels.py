"""Pins of the FP64 direct-sum oracle against closed forms (no GPU).

Sphere identities (radius a, uniform unit density, x at distance r from the
centre): single layer  V_L[1] = a (r < a), a^2/r (r > a);
Yukawa single layer    V_Y[1] = a e^{-ka} sinh(kr)/(kr) (r < a);
double layer (Gauss)   K_L[1] = -1 inside, 0 outside; at the centre
                       K_Y[1] = -e^{-ka}(1 + ka).
Target-normal derivatives are pinned by central finite differences of the
potential along n_x.
"""
import numpy as np
import pytest

from oracle.kernels import LAPLACE, YUKAWA, direct_sum


def sphere_rule(a, nth=48, nph=96):
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    ct, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    u = np.stack([st * np.cos(P), st * np.sin(P), ct], axis=-1).reshape(-1, 3)
    wt = (w[:, None] * np.full(nph, 2 * np.pi / nph)[None, :]).ravel() * a * a
    return u * a, u, wt


@pytest.mark.parametrize("r", [0.0, 0.6, 1.0])
def test_laplace_single_layer_sphere(r):
    a = 1.5
    y, n, w = sphere_rule(a)
    x = np.array([[0.0, 0.0, r]])
    v = direct_sum(LAPLACE, 0.0, y, q=w, tgt=x)[0]
    assert abs(v - a) < 1e-10
    xo = np.array([[0.0, 2.1, 0.9]])
    ro = np.linalg.norm(xo)
    vo = direct_sum(LAPLACE, 0.0, y, q=w, tgt=xo)[0]
    assert abs(vo - a * a / ro) < 1e-10


@pytest.mark.parametrize("r", [0.0, 0.5, 1.0])
def test_yukawa_single_layer_sphere(r):
    a, k = 1.5, 0.7
    y, n, w = sphere_rule(a)
    x = np.array([[r, 0.0, 0.0]])
    v = direct_sum(YUKAWA, k, y, q=w, tgt=x)[0]
    ref = a * np.exp(-k * a) * (np.sinh(k * r) / (k * r) if r > 0 else 1.0)
    assert abs(v - ref) < 1e-10


def test_double_layer_gauss():
    a = 1.2
    y, n, w = sphere_rule(a)
    inside = np.array([[0.1, -0.2, 0.3], [0.0, 0.0, 0.0]])
    outside = np.array([[2.0, 0.5, -1.0]])
    vi = direct_sum(LAPLACE, 0.0, y, dip=w, src_n=n, tgt=inside)
    vo = direct_sum(LAPLACE, 0.0, y, dip=w, src_n=n, tgt=outside)
    assert np.allclose(vi, -1.0, atol=1e-9)
    assert abs(vo[0]) < 1e-9
    k = 0.4
    vc = direct_sum(YUKAWA, k, y, dip=w, src_n=n, tgt=np.zeros((1, 3)))[0]
    assert abs(vc + np.exp(-k * a) * (1 + k * a)) < 1e-10


def test_outside_normal_derivative_closed_form():
    a = 1.0
    y, n, w = sphere_rule(a)
    x = np.array([[0.0, 0.0, 2.5]])
    nx = np.array([[0.0, 0.0, 1.0]])
    _, dn = direct_sum(LAPLACE, 0.0, y, q=w, tgt=x, tgt_n=nx, want_dn=True)
    assert abs(dn[0] + a * a / 2.5 ** 2) < 1e-10


@pytest.mark.parametrize("kernel,kappa", [(LAPLACE, 0.0), (YUKAWA, 0.125), (YUKAWA, 2.0)])
def test_target_derivative_finite_difference(kernel, kappa):
    rng = np.random.default_rng(5)
    src = rng.uniform(-1, 1, (40, 3))
    sn = rng.standard_normal((40, 3)); sn /= np.linalg.norm(sn, axis=1, keepdims=True)
    q = rng.uniform(-1, 1, 40)
    d = rng.uniform(-1, 1, 40)
    tgt = rng.uniform(2, 3, (5, 3))
    tn = rng.standard_normal((5, 3)); tn /= np.linalg.norm(tn, axis=1, keepdims=True)
    h = 1e-5
    for qq, dd in [(q, None), (None, d)]:
        _, dn = direct_sum(kernel, kappa, src, q=qq, dip=dd, src_n=sn, tgt=tgt, tgt_n=tn, want_dn=True)
        fp = direct_sum(kernel, kappa, src, q=qq, dip=dd, src_n=sn, tgt=tgt + h * tn)
        fm = direct_sum(kernel, kappa, src, q=qq, dip=dd, src_n=sn, tgt=tgt - h * tn)
        fd = (fp - fm) / (2 * h)
        assert np.allclose(dn, fd, rtol=1e-6, atol=1e-9)


def test_source_dipole_is_source_normal_derivative():
    """dg/dn_y pinned by finite differences of g in the source position."""
    rng = np.random.default_rng(6)
    src = rng.uniform(-1, 1, (1, 3))
    sn = np.array([[0.6, 0.0, 0.8]])
    tgt = rng.uniform(1.5, 2.5, (7, 3))
    h = 1e-5
    for kernel, kappa in [(LAPLACE, 0.0), (YUKAWA, 0.9)]:
        dl = direct_sum(kernel, kappa, src, dip=np.ones(1), src_n=sn, tgt=tgt)
        gp = direct_sum(kernel, kappa, src + h * sn, q=np.ones(1), tgt=tgt)
        gm = direct_sum(kernel, kappa, src - h * sn, q=np.ones(1), tgt=tgt)
        assert np.allclose(dl, (gp - gm) / (2 * h), rtol=1e-6)


def test_zero_distance_excluded():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    v = direct_sum(LAPLACE, 0.0, x, q=np.array([1.0, 1.0]))
    assert np.allclose(v, 1.0 / (4 * np.pi))
