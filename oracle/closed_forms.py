"""Closed-form polar solvation energies of a dielectric sphere.

Test infrastructure only.  Used to pin the discrete solver (Sec. "Mesh
refinement study using an analytical solution": a sphere of radius 4 A,
eps 4/80, kappa 0.125 1/A, unit charge at (1,1,1), analytic energy
-12.258363 kcal/mol from Kirkwood's series).

Units: charges in e, lengths in A, energies in kcal/mol through
C = 332.0637 kcal A / (mol e^2) = e^2 / (4 pi eps0 A).  The paper's Eq. energy
works in units where the potential of q in medium eps is q/(4 pi eps r), so
the discrete energy converts as dG[kcal/mol] = 1/2 sum q phi_reac * 4 pi C.
"""
from __future__ import annotations

import numpy as np

KCAL = 332.0637          # kcal A / (mol e^2)


def born_energy(q, a, eps_in, eps_out, kappa):
    """Born ion with Debye screening: (q^2/2a) (1/(eps_out(1+kappa a)) - 1/eps_in) * C."""
    return 0.5 * q * q / a * (1.0 / (eps_out * (1.0 + kappa * a)) - 1.0 / eps_in) * KCAL


def _kn_ratio_terms(x, nmax):
    """x k_n'(x)/k_n(x) for n = 0..nmax, k_n the modified spherical Bessel
    function of the second kind, via the stable forward recurrence of
    R_n = k_{n+1}/k_n:  R_0 = 1 + 1/x,  R_n = 1/R_{n-1} + (2n+1)/x,
    and x k_n'/k_n = n - x R_n."""
    out = np.empty(nmax + 1)
    R = 1.0 + 1.0 / x
    for n in range(nmax + 1):
        if n > 0:
            R = 1.0 / R + (2 * n + 1) / x
        out[n] = n - x * R
    return out


def kirkwood_energy(charges, positions, a, eps_in, eps_out, kappa, nmax=80):
    """Kirkwood (1934) polar solvation energy of point charges inside a sphere.

    Inside: Coulomb + sum_n B_n r^n P_n; outside: C_n k_n(kappa r) P_n.
    Continuity of phi and eps dphi/dr at r = a gives, per order n,
      B_n = q r_k^n / (4 pi eps_in) * ((n+1) eps_in + rho_n) / (a^(2n+1) (n eps_in - rho_n)),
      rho_n = eps_out * x k_n'(x)/k_n(x),  x = kappa a
    (for kappa = 0, rho_n = -(n+1) eps_out).  The energy 1/2 sum q phi_reac is
      1/2 sum_{k,l} q_k q_l / eps_in sum_n (r_k r_l)^n / a^(2n+1)
          ((n+1) eps_in + rho_n)/(n eps_in - rho_n) P_n(cos g_kl)   * C.
    """
    q = np.asarray(charges, dtype=np.float64).ravel()
    p = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    if kappa > 0:
        rho = eps_out * _kn_ratio_terms(kappa * a, nmax)
    else:
        rho = -eps_out * (np.arange(nmax + 1) + 1.0)
    n = np.arange(nmax + 1, dtype=np.float64)
    fac = ((n + 1) * eps_in + rho) / (n * eps_in - rho)
    r = np.linalg.norm(p, axis=1)
    total = 0.0
    for k in range(len(q)):
        for l in range(len(q)):
            rr = r[k] * r[l]
            if rr > 0:
                cg = float(np.dot(p[k], p[l]) / rr)
            else:
                cg = 1.0
            cg = min(1.0, max(-1.0, cg))
            # Legendre P_n(cg) by the three-term recurrence
            P = np.empty(nmax + 1)
            P[0] = 1.0
            if nmax > 0:
                P[1] = cg
            for m in range(1, nmax):
                P[m + 1] = ((2 * m + 1) * cg * P[m] - m * P[m - 1]) / (m + 1)
            terms = (rr ** n) / a ** (2 * n + 1) * fac * P
            total += q[k] * q[l] * terms.sum()
    return 0.5 * total / eps_in * KCAL
