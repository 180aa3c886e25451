"""Adaptive octree and KIFMM interaction lists, plain recursive definition.

Test infrastructure only.  Follows Sec. "Fast multipole method": a cube that
encloses all sources/targets is subdivided recursively until each leaf holds
no more than ncrit points; the near field N(B) (B and its neighbours) is
summed exactly and the interaction list I(B) (children of the parent's
neighbours that are not adjacent to B) goes through M2L.  The paper describes
a uniform tree; for the adaptive tree the lists are the U/V/W/X lists of
the kernel-independent FMM it cites (Ying, Biros, Zorin 2004).

Readings (the paper is silent on these):
  * cube: centre = midpoint of the coordinate min/max (FP32 values promoted
    to FP64); half-width R = the smallest power of two >= (0.5 * max
    extent) * (1 + 2^-20), so that trees of similar size share their boxes'
    sizes (and translation operators); R = 1 if all points coincide.
  * Morton integer per axis: floor((x - lo) * (2^21 / (2R))), clamped to
    [0, 2^21 - 1], every step a correctly rounded FP64 operation.
  * keys interleave x, y, z bits from the most significant bit (63 bits);
    points are sorted stably by key.
  * a box splits while its point count (sources plus targets when the two
    sets differ) exceeds ncrit and its level is below 21; empty children are
    dropped; boxes are numbered level by level in Morton order.
  * adjacency = the closed cubes intersect.
"""
from __future__ import annotations

import math

import numpy as np

MAXLEVEL = 21


def bounding_cube(points_list):
    """Centre (3,) and half-width R of the enclosing cube, FP64."""
    pts = np.concatenate([np.asarray(p, dtype=np.float32).reshape(-1, 3) for p in points_list])
    lo = pts.min(axis=0).astype(np.float64)
    hi = pts.max(axis=0).astype(np.float64)
    c = (lo + hi) * 0.5
    ext = float((hi - lo).max())
    R = (0.5 * ext) * (1.0 + 2.0 ** -20)
    if R == 0.0:
        return c, 1.0
    m, e = math.frexp(R)            # R = m 2^e, 0.5 <= m < 1 (exact)
    return c, (R if m == 0.5 else math.ldexp(1.0, e))


def morton_keys(points, c, R):
    """63-bit Morton keys (uint64) of FP32 points in the cube (c, R)."""
    p = np.asarray(points, dtype=np.float32).reshape(-1, 3).astype(np.float64)
    lo = c - R
    scale = float(2 ** MAXLEVEL) / (2.0 * R)
    q = np.floor((p - lo) * scale)
    q = np.clip(q, 0, 2 ** MAXLEVEL - 1).astype(np.uint64)
    key = np.zeros(p.shape[0], dtype=np.uint64)
    for b in range(MAXLEVEL - 1, -1, -1):
        for axis in range(3):
            bit = (q[:, axis] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + 2 - axis)
    return key


class Tree:
    """Boxes in level order.  Per box: level, parent, first_child, nchild,
    anchor (integer corner at its level), src range, tgt range."""

    def __init__(self):
        self.level, self.parent, self.first_child, self.nchild = [], [], [], []
        self.anchor = []
        self.sb, self.se, self.tb, self.te = [], [], [], []

    def add(self, level, parent, anchor, sb, se, tb, te):
        self.level.append(level); self.parent.append(parent)
        self.first_child.append(-1); self.nchild.append(0)
        self.anchor.append(anchor)
        self.sb.append(sb); self.se.append(se); self.tb.append(tb); self.te.append(te)
        return len(self.level) - 1

    def finalize(self):
        for k in ("level", "parent", "first_child", "nchild", "sb", "se", "tb", "te"):
            setattr(self, k, np.asarray(getattr(self, k), dtype=np.int64))
        self.anchor = np.asarray(self.anchor, dtype=np.int64).reshape(-1, 3)
        self.nbox = len(self.level)
        self.is_leaf = self.nchild == 0
        return self


def build_tree(src, ncrit, tgt=None):
    """Adaptive octree over sources (and targets, if a distinct set is given).

    Returns dict with: c, R, perm_src, keys_src (sorted), perm_tgt, keys_tgt,
    tree (Tree).  With tgt None the target set is the source set.
    """
    same = tgt is None
    c, R = bounding_cube([src] if same else [src, tgt])
    ks = morton_keys(src, c, R)
    ps = np.argsort(ks, kind="stable")
    ks = ks[ps]
    if same:
        kt, pt = ks, ps
    else:
        kt = morton_keys(tgt, c, R)
        pt = np.argsort(kt, kind="stable")
        kt = kt[pt]
    T = Tree()
    T.add(0, -1, (0, 0, 0), 0, len(ks), 0, len(kt))
    frontier = [0]
    level = 0
    while frontier and level < MAXLEVEL:
        nxt = []
        shift = np.uint64(3 * (MAXLEVEL - 1 - level))
        for b in frontier:
            sb, se, tb, te = T.sb[b], T.se[b], T.tb[b], T.te[b]
            count = (se - sb) if same else (se - sb) + (te - tb)
            if count <= ncrit:
                continue
            ds = ((ks[sb:se] >> shift) & np.uint64(7)).astype(np.int64)
            dt = ds if same else ((kt[tb:te] >> shift) & np.uint64(7)).astype(np.int64)
            first = None
            ax, ay, az = T.anchor[b]
            for dgt in range(8):
                s0 = sb + int(np.searchsorted(ds, dgt, "left"))
                s1 = sb + int(np.searchsorted(ds, dgt, "right"))
                t0 = tb + int(np.searchsorted(dt, dgt, "left"))
                t1 = tb + int(np.searchsorted(dt, dgt, "right"))
                if s1 == s0 and t1 == t0:
                    continue
                anc = (2 * ax + (dgt >> 2 & 1), 2 * ay + (dgt >> 1 & 1), 2 * az + (dgt & 1))
                ch = T.add(level + 1, b, anc, s0, s1, t0, t1)
                if first is None:
                    first = ch
                T.nchild[b] += 1
                nxt.append(ch)
            T.first_child[b] = first
        frontier = nxt
        level += 1
    T.finalize()
    return dict(c=c, R=R, perm_src=ps, keys_src=ks, perm_tgt=pt, keys_tgt=kt, tree=T, same=same)


def adjacent(T, a, b):
    """True iff the closed cubes of boxes a and b intersect."""
    la, lb = T.level[a], T.level[b]
    L = max(la, lb)
    sa, sb_ = 1 << (L - la), 1 << (L - lb)
    A0, B0 = T.anchor[a] * sa, T.anchor[b] * sb_
    A1, B1 = A0 + sa, B0 + sb_
    return bool(np.all(A0 <= B1) and np.all(B0 <= A1))


def children(T, b):
    if T.nchild[b] == 0:
        return []
    return list(range(T.first_child[b], T.first_child[b] + T.nchild[b]))


def build_lists(T):
    """U, V, W, X lists (sorted box ids) of every box, plus colleagues.

    Coll(B): same-level boxes adjacent to B (B included).
    V(B)   : children of Coll(parent) not adjacent to B        (M2L).
    X(B)   : coarser leaves adjacent to parent(B), not to B      (P2L).
    U(B)   : for a leaf, every leaf adjacent to B (B included)  (P2P).
    W(B)   : for a leaf, descendants D of B's colleagues with parent(D)
             adjacent to B and D not adjacent to B               (M2P).
    """
    n = T.nbox
    coll = [[] for _ in range(n)]
    cn = [[] for _ in range(n)]     # coarser leaves adjacent to the box
    V = [[] for _ in range(n)]
    X = [[] for _ in range(n)]
    U = [[] for _ in range(n)]
    W = [[] for _ in range(n)]
    coll[0] = [0]
    for b in range(1, n):           # level order: parents come first
        P = T.parent[b]
        for C in coll[P]:
            if T.is_leaf[C]:
                (cn[b] if adjacent(T, C, b) else X[b]).append(C)
            else:
                for D in children(T, C):
                    (coll[b] if adjacent(T, D, b) else V[b]).append(D)
        for A in cn[P]:
            (cn[b] if adjacent(T, A, b) else X[b]).append(A)
    for b in range(n):
        if not T.is_leaf[b]:
            continue
        u = set(cn[b])
        for C in coll[b]:
            if T.is_leaf[C]:
                u.add(C)
                continue
            stack = children(T, C)
            while stack:
                D = stack.pop()
                if adjacent(T, D, b):
                    if T.is_leaf[D]:
                        u.add(D)
                    else:
                        stack.extend(children(T, D))
                else:
                    W[b].append(D)
        U[b] = sorted(u)
        W[b] = sorted(W[b])
    for b in range(n):
        coll[b] = sorted(coll[b]); V[b] = sorted(V[b]); X[b] = sorted(X[b])
    return dict(U=U, V=V, W=W, X=X, coll=coll)


def to_csr(lists):
    off = np.zeros(len(lists) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    ids = np.fromiter((i for l in lists for i in l), dtype=np.int64, count=int(off[-1]))
    return off, ids
