"""The bench's pair accounting for the directly summed adaptive-list boxes.

bench.list_work counts, from the exported tree (box ranges, W and X lists in
CSR), the pairs the leaf kernel sums directly and the far-field work left;
the leaf roofline's FLOP count rests on it.  Checked here on small
hand-built trees against a brute-force count over (target, source box)
entries, with the rules the library applies: a W-list box of at most
n_e // 2 sources, the X list of a leaf of at most n_e targets.
"""
import numpy as np

import bench


def _csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    for i, l in enumerate(lists):
        off[i + 1] = off[i] + len(l)
    ids = np.array([a for l in lists for a in l], np.int32)
    return off, ids


def _tree(rng, nbox=40, ne=56, distinct_targets=False):
    nchild = (rng.random(nbox) < 0.3).astype(np.int32) * 8
    ns = rng.integers(0, 2 * ne, nbox)
    nt = rng.integers(0, 2 * ne, nbox) if distinct_targets else ns
    sb = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int32)
    tb = np.concatenate([[0], np.cumsum(nt)[:-1]]).astype(np.int32)
    W = [list(rng.choice(nbox, rng.integers(0, 6), replace=False)) for _ in range(nbox)]
    X = [list(rng.choice(nbox, rng.integers(0, 4), replace=False)) for _ in range(nbox)]
    ex = {"nchild": nchild, "src_begin": sb, "src_end": (sb + ns).astype(np.int32),
          "tgt_begin": tb if distinct_targets else np.zeros(nbox, np.int32),
          "tgt_end": (tb + nt).astype(np.int32) if distinct_targets else np.zeros(nbox, np.int32),
          "W": _csr(W), "X": _csr(X)}
    return ex, ns, nt, nchild, W, X


def _brute(ns, nt, nchild, W, X, ne, dw, dx):
    w_dir = x_dir = m2p = p2l = 0
    for b in range(len(ns)):
        for a in W[b]:
            if dw and ns[a] <= ne // 2:
                w_dir += nt[b] * ns[a]
            else:
                m2p += nt[b]
        for a in X[b]:
            if dx and nchild[b] == 0 and nt[b] <= ne:
                x_dir += nt[b] * ns[a]
            else:
                p2l += ns[a]
    return w_dir, x_dir, m2p, p2l


def test_list_work_matches_brute_force():
    rng = np.random.default_rng(5)
    for distinct in (False, True):
        ex, ns, nt, nchild, W, X = _tree(rng, distinct_targets=distinct)
        for dw in (False, True):
            for dx in (False, True):
                assert bench.list_work(ex, 56, dw, dx) == _brute(ns, nt, nchild, W, X, 56, dw, dx)


def test_list_work_off_keeps_all_far_work():
    """With both rules off, nothing is direct and the far counts are the
    tree's m2p_targets / p2l_sources totals."""
    rng = np.random.default_rng(6)
    ex, ns, nt, nchild, W, X = _tree(rng)
    w_dir, x_dir, m2p, p2l = bench.list_work(ex, 152, False, False)
    assert w_dir == 0 and x_dir == 0
    assert m2p == sum(nt[b] * len(W[b]) for b in range(len(ns)))
    assert p2l == sum(ns[a] for b in range(len(ns)) for a in X[b])
