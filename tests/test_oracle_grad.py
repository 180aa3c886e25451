"""Pins of the oracle's energy gradients (no GPU).

dE/dq = 1/2 (R + R^T) q is checked against central differences of the
dense-LU energy (E is quadratic in q, so the difference is exact up to
rounding), against the Born relation dE/dq = 2E/q for a single charge, and
dE/dr = 0 for the charge at the centre of the sphere (symmetry).
"""
import numpy as np

import synthetic
from oracle import bem

EPS = (4.0, 80.0, 0.125)


def test_grad_q_vs_finite_difference():
    V, F = synthetic.icosphere(2, 3.0)
    mats = bem.assemble_p0(V, F, 3, EPS[2])
    atoms = np.array([[0.5, -0.3, 0.2], [-0.8, 0.4, 0.6], [0.1, 0.9, -0.7]])
    q = np.array([0.6, -0.5, 0.3])
    g = bem.energy_grad_q(V, F, 3, atoms, q, *EPS, mats)
    h = 1e-3
    for k in range(3):
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        ep, *_ = bem.solve_energy(V, F, 3, atoms, qp, *EPS, mats=mats)
        em, *_ = bem.solve_energy(V, F, 3, atoms, qm, *EPS, mats=mats)
        assert abs((ep - em) / (2 * h) - g[k]) < 1e-9 * max(1.0, abs(g[k]))


def test_born_gradient_relations():
    V, F = synthetic.icosphere(2, 2.0)
    mats = bem.assemble_p0(V, F, 3, EPS[2])
    atoms, q = np.zeros((1, 3)), np.array([1.0])
    E, *_ = bem.solve_energy(V, F, 3, atoms, q, *EPS, mats=mats)
    g = bem.energy_grad_q(V, F, 3, atoms, q, *EPS, mats)
    assert abs(g[0] - 2 * E) < 1e-9 * abs(E)
    gx = bem.energy_grad_x_fd(V, F, 3, atoms, q, *EPS, mats, h=1e-3)
    assert all(abs(v) < 1e-6 for v in gx.values())
