"""O4: Morton codes, stable sort, adaptive quadtree and interaction lists.

TEST INFRASTRUCTURE ONLY.  Written independently of the CUDA tree builder so
that the two can be compared bit for bit.

Paper Section 2.2: the square D containing the points is partitioned into
2^{l+1} x 2^{l+1} blocks at levels l = 1..L, children obtained by bisecting
edges.  Here the hierarchy is the adaptive generalisation of that partition:

* Domain D = (x0, y0, S).  Default: the exact bounding square of the points
  (lower-left corner at the coordinate minima, side = larger extent, S = 1 when
  the extent is zero).
* Quantisation, FP64 with every operation rounded as written (no fused
  multiply-add): q = floor(((x - x0) / S) * 65536), clamped to [0, 65535].  A
  point on an interior block edge therefore belongs to the upper/right block.
* Morton code: bit b of qx goes to bit 2b, bit b of qy to bit 2b+1 (uint32).
* Stable sort by code; equal codes keep their input order.
* Box = (level, prefix): the sorted points whose code has the 2*level-bit
  prefix.  A box is split into its non-empty quadrants iff it holds more than
  `leaf` points and level < 16.  Boxes are numbered in (level, prefix) order.
  The paper's level l is depth l+1 here (its first level is already 4x4).
* Lists (Carrier-Greengard-Rokhlin adaptive definitions; the paper's S_p is
  the V list and NS_p the U list on a uniform tree):
    colleagues(B): same-level boxes adjacent to B, B included;
    V(B): children of colleagues(parent(B)) not adjacent to B;
    U(B), leaf B: all leaves adjacent to B (any level, B included);
    W(B), leaf B: descendants of B's colleagues that are not adjacent to B
           but whose parent is;
    X(B): boxes A with B in W(A).
  "Adjacent" means the closed squares intersect (shared edge or corner).
  Each list is sorted by box number.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAX_LEVEL = 16
QMAX = (1 << 16) - 1


def default_domain(points) -> tuple:
    pts = np.asarray(points, dtype=np.float64)
    if pts.shape[0] == 0:
        return (0.0, 0.0, 1.0)
    x0 = float(pts[:, 0].min())
    y0 = float(pts[:, 1].min())
    ex = float(pts[:, 0].max()) - x0
    ey = float(pts[:, 1].max()) - y0
    s = max(ex, ey)
    if s == 0.0:
        s = 1.0
    return (x0, y0, s)


def quantise(points, domain) -> tuple:
    """Integer cell (qx, qy) of each point, FP64 exactly as written above."""
    pts = np.asarray(points, dtype=np.float64)
    x0, y0, s = domain
    tx = ((pts[:, 0] - x0) / s) * 65536.0
    ty = ((pts[:, 1] - y0) / s) * 65536.0
    qx = np.clip(np.floor(tx), 0, QMAX).astype(np.uint32)
    qy = np.clip(np.floor(ty), 0, QMAX).astype(np.uint32)
    return qx, qy


def interleave(qx, qy) -> np.ndarray:
    qx = np.asarray(qx, dtype=np.uint32)
    qy = np.asarray(qy, dtype=np.uint32)
    code = np.zeros(qx.shape, dtype=np.uint32)
    for b in range(16):
        code |= ((qx >> np.uint32(b)) & np.uint32(1)) << np.uint32(2 * b)
        code |= ((qy >> np.uint32(b)) & np.uint32(1)) << np.uint32(2 * b + 1)
    return code


def deinterleave(code, nbits: int = 16) -> tuple:
    code = np.asarray(code, dtype=np.uint32)
    qx = np.zeros(code.shape, dtype=np.uint32)
    qy = np.zeros(code.shape, dtype=np.uint32)
    for b in range(nbits):
        qx |= ((code >> np.uint32(2 * b)) & np.uint32(1)) << np.uint32(b)
        qy |= ((code >> np.uint32(2 * b + 1)) & np.uint32(1)) << np.uint32(b)
    return qx, qy


def morton_codes(points, domain) -> np.ndarray:
    qx, qy = quantise(points, domain)
    return interleave(qx, qy)


@dataclass
class Tree:
    domain: tuple
    leaf_size: int
    codes: np.ndarray          # unsorted Morton codes, per input point
    perm: np.ndarray           # sorted position -> input index
    sorted_codes: np.ndarray
    level: np.ndarray
    prefix: np.ndarray
    begin: np.ndarray
    end: np.ndarray
    parent: np.ndarray
    child: np.ndarray          # [nbox, 4], -1 where absent (quadrant q = 2*ybit + xbit)
    is_leaf: np.ndarray
    ix: np.ndarray
    iy: np.ndarray
    colleagues: list = field(default_factory=list)
    U: list = field(default_factory=list)
    V: list = field(default_factory=list)
    W: list = field(default_factory=list)
    X: list = field(default_factory=list)

    @property
    def nbox(self) -> int:
        return int(self.level.shape[0])

    def centre(self, b: int) -> tuple:
        x0, y0, s = self.domain
        h = s / float(1 << int(self.level[b]))
        return (x0 + (float(self.ix[b]) + 0.5) * h, y0 + (float(self.iy[b]) + 0.5) * h)

    def centres(self) -> np.ndarray:
        x0, y0, s = self.domain
        h = s / np.exp2(self.level.astype(np.float64))
        return np.stack([x0 + (self.ix + 0.5) * h, y0 + (self.iy + 0.5) * h], axis=1)

    def size(self, b: int) -> float:
        return self.domain[2] / float(1 << int(self.level[b]))

    def children(self, b: int) -> list:
        return [int(q) for q in self.child[b] if q >= 0]

    def csr(self, name: str) -> tuple:
        lists = getattr(self, name)
        offs = np.zeros(self.nbox + 1, dtype=np.int32)
        offs[1:] = np.cumsum([len(l) for l in lists])
        items = np.array([q for l in lists for q in l], dtype=np.int32)
        return offs, items


def adjacent(t: Tree, a: int, b: int) -> bool:
    """Closed squares of boxes a and b intersect (integer test at the finer level)."""
    la, lb = int(t.level[a]), int(t.level[b])
    L = max(la, lb)
    sa, sb = L - la, L - lb
    ax0, ax1 = int(t.ix[a]) << sa, (int(t.ix[a]) + 1) << sa
    ay0, ay1 = int(t.iy[a]) << sa, (int(t.iy[a]) + 1) << sa
    bx0, bx1 = int(t.ix[b]) << sb, (int(t.ix[b]) + 1) << sb
    by0, by1 = int(t.iy[b]) << sb, (int(t.iy[b]) + 1) << sb
    return ax0 <= bx1 and bx0 <= ax1 and ay0 <= by1 and by0 <= ay1


def build_tree(points, leaf: int, domain=None, lists: bool = True) -> Tree:
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    if domain is None:
        domain = default_domain(pts)
    domain = tuple(float(v) for v in domain)
    codes = morton_codes(pts, domain)
    perm = np.argsort(codes, kind="stable").astype(np.int64)
    sc = codes[perm]

    level = [0]
    prefix = [0]
    begin = [0]
    end = [n]
    parent = [-1]
    child = [[-1, -1, -1, -1]]
    cur = [0]
    for lev in range(MAX_LEVEL):
        shifted = (sc >> np.uint32(32 - 2 * (lev + 1))).astype(np.int64)
        nxt = []
        for b in cur:
            if end[b] - begin[b] <= leaf:
                continue
            seg = shifted[begin[b]:end[b]]
            for q in range(4):
                cp = 4 * prefix[b] + q
                lo = begin[b] + int(np.searchsorted(seg, cp, side="left"))
                hi = begin[b] + int(np.searchsorted(seg, cp, side="right"))
                if hi > lo:
                    idx = len(level)
                    level.append(lev + 1)
                    prefix.append(cp)
                    begin.append(lo)
                    end.append(hi)
                    parent.append(b)
                    child.append([-1, -1, -1, -1])
                    child[b][q] = idx
                    nxt.append(idx)
        if not nxt:
            break
        cur = nxt

    level = np.array(level, dtype=np.int32)
    prefix = np.array(prefix, dtype=np.uint32)
    ix, iy = deinterleave(prefix)
    child = np.array(child, dtype=np.int32)
    t = Tree(domain=domain, leaf_size=int(leaf), codes=codes, perm=perm, sorted_codes=sc,
             level=level, prefix=prefix, begin=np.array(begin, dtype=np.int64),
             end=np.array(end, dtype=np.int64), parent=np.array(parent, dtype=np.int32),
             child=child, is_leaf=np.all(child < 0, axis=1), ix=ix.astype(np.int64),
             iy=iy.astype(np.int64))
    if lists:
        build_lists(t)
    return t


def build_lists(t: Tree) -> None:
    nb = t.nbox
    col = [None] * nb
    V = [[] for _ in range(nb)]
    col[0] = [0]
    for b in range(1, nb):
        pb = int(t.parent[b])
        cands = [d for q in col[pb] for d in t.children(q)]
        col[b] = sorted(d for d in cands if adjacent(t, d, b))
        V[b] = sorted(d for d in cands if not adjacent(t, d, b))
    U = [[] for _ in range(nb)]
    W = [[] for _ in range(nb)]
    X = [[] for _ in range(nb)]
    for b in range(nb):
        if not t.is_leaf[b]:
            continue
        u = []
        a = int(t.parent[b])
        while a >= 0:
            for q in col[a]:
                if t.is_leaf[q] and adjacent(t, q, b):
                    u.append(q)
            a = int(t.parent[a])
        stack = list(col[b])
        while stack:
            q = stack.pop()
            if t.is_leaf[q]:
                u.append(q)
            else:
                for d in t.children(q):
                    if adjacent(t, d, b):
                        stack.append(d)
        U[b] = sorted(u)
        w = []
        stack = [q for q in col[b] if q != b and not t.is_leaf[q]]
        while stack:
            q = stack.pop()
            for d in t.children(q):
                if adjacent(t, d, b):
                    if not t.is_leaf[d]:
                        stack.append(d)
                else:
                    w.append(d)
        W[b] = sorted(w)
        for d in W[b]:
            X[d].append(b)
    for b in range(nb):
        X[b].sort()
    t.colleagues, t.U, t.V, t.W, t.X = col, U, V, W, X


def coverage(t: Tree) -> np.ndarray:
    """Count, for every (target, source) pair in sorted order, how many list
    entries cover it; an exact partition gives the all-ones matrix."""
    n = int(t.end[0])
    cnt = np.zeros((n, n), dtype=np.int64)
    for b in range(t.nbox):
        tb = slice(int(t.begin[b]), int(t.end[b]))
        for name in ("U", "V", "W", "X"):
            for s in getattr(t, name)[b]:
                cnt[tb, int(t.begin[s]):int(t.end[s])] += 1
    return cnt


def brute_force_lists(t: Tree) -> dict:
    """U/V/W/X recomputed from their set definitions by enumerating all box
    pairs (tiny trees only)."""
    nb = t.nbox
    anc = []
    for b in range(nb):
        a, chain = b, []
        while a >= 0:
            chain.append(a)
            a = int(t.parent[a])
        anc.append(chain)   # b, parent(b), ..., root
    adj = np.array([[adjacent(t, a, b) for b in range(nb)] for a in range(nb)])
    leaves = [b for b in range(nb) if t.is_leaf[b]]
    U, V, W, X = ([[] for _ in range(nb)] for _ in range(4))
    for b in range(nb):
        if b > 0:
            pb = int(t.parent[b])
            for d in range(nb):
                if t.level[d] == t.level[b] and t.parent[d] >= 0:
                    pd = int(t.parent[d])
                    if t.level[pd] == t.level[pb] and adj[pd, pb] and not adj[d, b]:
                        V[b].append(d)
        if t.is_leaf[b]:
            U[b] = [a for a in leaves if adj[a, b]]
            for d in range(nb):
                if d == 0 or t.level[d] <= t.level[b]:
                    continue
                pd = int(t.parent[d])
                # d descends from a colleague of b: its ancestor at b's level is adjacent to b
                a_at = anc[d][int(t.level[d]) - int(t.level[b])]
                if a_at != b and adj[a_at, b] and adj[pd, b] and not adj[d, b]:
                    W[b].append(d)
    for b in range(nb):
        for d in W[b]:
            X[d].append(b)
    return {"U": U, "V": V, "W": W, "X": [sorted(x) for x in X]}
