"""Pins of the oracle octree and interaction lists (no GPU).

The top-down list construction in oracle/tree.py is checked against the
lists' definitions evaluated by brute force over all box pairs, against the
exactly-once coverage of every (target, source) pair, and the Morton keys
against a per-point bit loop.
"""
import numpy as np
import pytest

import synthetic
from oracle import tree as ot


def brute_keys(pts, c, R):
    lo = c - R
    scale = float(2 ** 21) / (2.0 * R)
    out = []
    for p in np.asarray(pts, dtype=np.float32).astype(np.float64):
        ints = [min(max(int(np.floor((p[a] - lo[a]) * scale)), 0), 2 ** 21 - 1) for a in range(3)]
        k = 0
        for b in range(20, -1, -1):
            for a in range(3):
                k = (k << 1) | ((ints[a] >> b) & 1)
        out.append(k)
    return np.array(out, dtype=np.uint64)


def point_sets():
    rng = np.random.default_rng(11)
    x, _ = synthetic.bumpy_sphere_points(1500, seed=3)
    yield "sphere", x, None, 40
    cl = np.concatenate([rng.normal(0, 0.01, (300, 3)), rng.uniform(-1, 1, (700, 3))]).astype(np.float32)
    yield "clustered", cl, None, 25
    s = rng.uniform(-1, 1, (600, 3)).astype(np.float32)
    t = rng.normal(0.3, 0.2, (500, 3)).astype(np.float32)
    yield "separate", s, t, 30
    dup = np.repeat(rng.uniform(0, 1, (5, 3)).astype(np.float32), 20, axis=0)
    yield "duplicates", dup, None, 8


@pytest.mark.parametrize("name,src,tgt,ncrit", list(point_sets()))
def test_tree_and_lists(name, src, tgt, ncrit):
    res = ot.build_tree(src, ncrit, tgt)
    T = res["tree"]
    c, R = res["c"], res["R"]
    # keys
    ks = brute_keys(src, c, R)
    assert np.array_equal(ks[res["perm_src"]], res["keys_src"])
    assert np.all(np.diff(res["keys_src"].astype(np.float64)) >= 0)
    # every point inside its cube
    pts = np.asarray(src, dtype=np.float64)
    assert np.all(np.abs(pts - c) <= R)
    # leaves partition the points; split rule
    same = tgt is None
    leaves = np.where(T.is_leaf)[0]
    assert sum(T.se[b] - T.sb[b] for b in leaves) == len(src)
    for b in range(T.nbox):
        cnt = (T.se[b] - T.sb[b]) + (0 if same else T.te[b] - T.tb[b])
        if T.is_leaf[b]:
            assert cnt <= ncrit or T.level[b] == ot.MAXLEVEL
        else:
            assert cnt > ncrit
        # the box's points lie in its key range
        sh = np.uint64(3 * (21 - T.level[b]))
        a = T.anchor[b]
        pref = 0
        for bit in range(T.level[b] - 1, -1, -1):
            for ax in range(3):
                pref = (pref << 1) | ((int(a[ax]) >> bit) & 1)
        kk = res["keys_src"][T.sb[b]:T.se[b]] >> sh
        assert np.all(kk == np.uint64(pref))
    L = ot.build_lists(T)
    n = T.nbox
    adj = np.zeros((n, n), dtype=bool)
    for a in range(n):
        for b in range(n):
            adj[a, b] = ot.adjacent(T, a, b)

    def is_desc(a, b):     # a strict descendant of b
        p = T.parent[a]
        while p >= 0:
            if p == b:
                return True
            p = T.parent[p]
        return False

    for b in range(n):
        lvl = T.level[b]
        V = [a for a in range(n) if T.level[a] == lvl and not adj[a, b] and b > 0
             and adj[T.parent[a], T.parent[b]]]
        assert L["V"][b] == V
        if T.is_leaf[b]:
            U = [a for a in range(n) if T.is_leaf[a] and adj[a, b]]
            assert L["U"][b] == U
            W = [a for a in range(n) if T.level[a] > lvl and not adj[a, b] and adj[T.parent[a], b]
                 and any(is_desc(a, cc) for cc in range(n) if T.level[cc] == lvl and adj[cc, b])]
            assert L["W"][b] == W
    # X is the dual of W
    for b in range(n):
        X = [a for a in range(n) if T.is_leaf[a] and b in L["W"][a]]
        assert L["X"][b] == X
    # U and V symmetric
    for b in range(n):
        for a in L["V"][b]:
            assert b in L["V"][a]
        for a in L["U"][b]:
            assert b in L["U"][a]
    # exactly-once coverage of every (target leaf, source box) pair, by points
    ns = len(src)
    src_box = np.empty(ns, dtype=np.int64)   # sorted position -> leaf
    for b in leaves:
        src_box[T.sb[b]:T.se[b]] = b

    def anc_chain(b):
        out = []
        while b >= 0:
            out.append(b)
            b = T.parent[b]
        return out

    def box_pts(a):
        return set(range(T.sb[a], T.se[a]))

    for b in leaves:
        if T.te[b] == T.tb[b] and not same:
            continue
        cover = np.zeros(ns, dtype=np.int64)
        for a in L["U"][b]:
            cover[list(box_pts(a))] += 1
        for a in L["W"][b]:
            cover[list(box_pts(a))] += 1
        for anc in anc_chain(b):
            for a in L["V"][anc] + L["X"][anc]:
                cover[list(box_pts(a))] += 1
        assert np.all(cover == 1), (name, b)


def test_cube_rules():
    pts = np.array([[0, 0, 0], [1, 2, 0.5]], dtype=np.float32)
    c, R = ot.bounding_cube([pts])
    assert np.allclose(c, [0.5, 1.0, 0.25])
    # half the extent is 1, enlarged by 2^-20, rounded up to a power of two
    assert R == 2.0
    c1, R1 = ot.bounding_cube([np.ones((3, 3), dtype=np.float32)])
    assert R1 == 1.0
    # an extent whose enlarged half is already a power of two keeps it, and
    # every cube encloses its points with R a power of two
    _, R2 = ot.bounding_cube([np.array([[0, 0, 0], [2.0 / (1 + 2.0 ** -20), 0, 0]])])
    assert R2 == 1.0
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = rng.uniform(-5, 5, (50, 3)).astype(np.float32) * rng.uniform(0.01, 100)
        c3, R3 = ot.bounding_cube([p])
        m, e = np.frexp(R3)
        assert m == 0.5
        assert np.all(np.abs(p.astype(np.float64) - c3) <= R3)
        assert R3 < 2 * 0.5 * np.ptp(p.astype(np.float64), axis=0).max() * (1 + 2.0 ** -20) + 1e-300
