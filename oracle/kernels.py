"""FP64 direct sums: the quantity the FMM approximates (Eq. nbody_sum).

Kernels (Eq. single_double, Eq. adj_hyp), r = |x - y|, x target, y source:
  g_L = 1/(4 pi r),  g_Y = exp(-kappa r)/(4 pi r),
  dg/dn_y = exp(-kappa r)(1 + kappa r)(x - y).n_y / (4 pi r^3)   (double layer),
  dg/dn_x = -exp(-kappa r)(1 + kappa r)(x - y).n_x / (4 pi r^3)  (adjoint double layer),
with kappa = 0 for Laplace.  Pairs at r = 0 are excluded.
Test infrastructure only.
"""
import ctypes

import numpy as np

from ._lib import lib

LAPLACE, YUKAWA = 0, 1


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c3(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)


def _c1(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64).ravel()


def direct_sum(kernel, kappa, src, q=None, dip=None, src_n=None, tgt=None, tgt_n=None,
               want_dn=False):
    """Potential (and, with want_dn, its target-normal derivative) at targets.

    out[i] = sum_j g(x_i, y_j) q_j + dg/dn_y(x_i, y_j) dip_j
    dn[i]  = sum_j dg/dn_x(x_i, y_j) q_j + d2g/dn_x dn_y(x_i, y_j) dip_j
    """
    src = _c3(src)
    tgt = src if tgt is None else _c3(tgt)
    q, dip = _c1(q), _c1(dip)
    src_n, tgt_n = _c3(src_n), _c3(tgt_n)
    if dip is not None and src_n is None:
        raise ValueError("double layer needs source normals")
    if want_dn and tgt_n is None:
        raise ValueError("target normal derivative needs target normals")
    nt = tgt.shape[0]
    out = np.zeros(nt)
    dn = np.zeros(nt) if want_dn else None
    lib().or_direct_sum(int(kernel), float(kappa), src.shape[0], _p(src), _p(q), _p(dip), _p(src_n),
                        nt, _p(tgt), _p(tgt_n), _p(out), _p(dn))
    return (out, dn) if want_dn else out


def rel_l2(a, ref):
    """Relative L2 error ||a - ref|| / ||ref|| (the 'digits' measure)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
