"""Oracle: Morton order, octree, directional (HF) and KI-FMM (LF) lists.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package;
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.

Plain numpy, integer arithmetic for every geometric predicate so that results
are exact and comparable bit for bit with the CUDA plan.

Paper passages followed (Benson, Poulson, Tran, Engquist, Ying,
arXiv:1311.4257):
  * Sec. 2.2: a box is high-frequency (HF) if w >= 1, low-frequency (LF) if
    w < 1; the octree splits every non-empty HF box and an LF box only if it
    holds more than a fixed number of points.
  * Sec. 2.2: near field N^B, far field, interaction list I^B = N^P \\ N^B.
    The printed near-field radius is garbled (sqrt(3) w / 2 in the
    definition, 3 w^2 / 4 in the proof of Prop. 1); the reading used here is
    "A is near B iff the closed box A has a point within rho * w^2 of the
    centre of B", rho = 1, which for w = 1 gives exactly the 27 colleagues.
  * Sec. 2.2, Fig. 2: hierarchical wedges; boxes on a wedge boundary go to
    the first wedge in a lexicographic order. Reading: the directions of a
    width-w box are the cells of a w x w grid on each of the 6 cube faces.
  * Sec. 2.3, Alg. 1: M2L partner direction l' is the direction in which B
    lies as seen from A.
  * LF lists (deferred by the paper to Engquist-Ying 2007): the standard
    adaptive kernel-independent FMM lists U, V, W, X with "adjacent" meaning
    the closed boxes touch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LEVEL_BITS = 21          # Morton quantisation bits per axis
MAX_DEPTH = LEVEL_BITS   # deepest level of the octree


# ---------------------------------------------------------------- Morton ---

def root_width(K: float) -> float:
    """Root box width W = 2^ceil(log2 K): box widths stay powers of two, so the
    HF/LF threshold w = 1 falls exactly on a level."""
    if not K > 0:
        raise ValueError("K must be positive")
    return float(2.0 ** max(0, math.ceil(math.log2(K))))


def quantize(points: np.ndarray, W: float) -> np.ndarray:
    """q_d = floor((x_d + W/2) * 2^21 / W), clamped to [0, 2^21 - 1].

    One rounding only (the FP64 addition); the scaling is by a power of two.
    A point on an internal face belongs to the upper box; a point on the
    root's upper face is clamped into the last box.
    """
    scale = float(2 ** LEVEL_BITS) / W
    t = (points + 0.5 * W) * scale
    q = np.floor(t)
    q = np.clip(q, 0, 2 ** LEVEL_BITS - 1)
    return q.astype(np.int64)


def interleave(q: np.ndarray) -> np.ndarray:
    """63-bit Morton key: bit b of x, y, z goes to key bits 3b+2, 3b+1, 3b."""
    q = q.astype(np.uint64)
    key = np.zeros(q.shape[0], dtype=np.uint64)
    for b in range(LEVEL_BITS):
        for d, sh in ((0, 2), (1, 1), (2, 0)):
            bit = (q[:, d] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + sh)
    return key


def deinterleave(key: np.ndarray, nbits: int) -> np.ndarray:
    """Inverse of interleave for a key of nbits bits per axis -> (n, 3) int64."""
    key = np.asarray(key, dtype=np.uint64)
    out = np.zeros((key.shape[0], 3), dtype=np.int64)
    for b in range(nbits):
        for d, sh in ((0, 2), (1, 1), (2, 0)):
            bit = (key >> np.uint64(3 * b + sh)) & np.uint64(1)
            out[:, d] |= (bit.astype(np.int64) << b)
    return out


def morton_sort(points: np.ndarray, K: float):
    """Keys and the stable permutation sorting points by (key, index)."""
    W = root_width(K)
    keys = interleave(quantize(points, W))
    perm = np.argsort(keys, kind="stable")
    return keys[perm], perm


# ------------------------------------------------------------------ tree ---

@dataclass
class Level:
    l: int
    w: float
    prefix: np.ndarray      # uint64 Morton prefixes of the boxes, ascending
    coords: np.ndarray      # (n, 3) int64 integer box coordinates
    first: np.ndarray       # first sorted point index
    count: np.ndarray       # number of points
    parent: np.ndarray      # index into level l-1 (-1 at the root)
    leaf: np.ndarray        # bool
    child_first: np.ndarray = field(default=None)   # index into level l+1
    nchild: np.ndarray = field(default=None)

    @property
    def n(self) -> int:
        return int(self.prefix.shape[0])

    @property
    def hf(self) -> bool:
        return self.w >= 1.0

    def centers(self, W: float) -> np.ndarray:
        return -0.5 * W + (self.coords + 0.5) * self.w

    def lookup(self, coords: np.ndarray) -> np.ndarray:
        """Box index for integer coordinates, -1 where no such box exists."""
        n = 1 << self.l
        inside = np.all((coords >= 0) & (coords < n), axis=-1)
        c = np.where(inside[..., None], coords, 0)
        key = interleave(c.reshape(-1, 3)).reshape(c.shape[:-1])
        pos = np.searchsorted(self.prefix, key)
        pos = np.minimum(pos, self.n - 1)
        hit = inside & (self.prefix[pos] == key)
        return np.where(hit, pos, -1)


@dataclass
class Tree:
    K: float
    W: float
    N: int
    leaf_max: int
    keys: np.ndarray
    perm: np.ndarray
    levels: list

    def level_of_width(self, w: float) -> int:
        return int(round(math.log2(self.W / w)))

    @property
    def hf_levels(self):
        return [L for L in self.levels if L.hf]

    @property
    def lf_levels(self):
        return [L for L in self.levels if not L.hf]


def build_tree(points: np.ndarray, K: float, leaf_max: int = 64) -> Tree:
    """Sec. 2.2: split every non-empty HF box; split an LF box iff it holds more
    than leaf_max points; stop at depth 21 (duplicates only beyond that)."""
    W = root_width(K)
    keys, perm = morton_sort(points, K)
    N = points.shape[0]
    levels = []
    # level 0: the root
    prefix = np.array([0], dtype=np.uint64)
    first = np.array([0], dtype=np.int64)
    count = np.array([N], dtype=np.int64)
    parent = np.array([-1], dtype=np.int64)
    l = 0
    while True:
        w = W / (1 << l)
        coords = deinterleave(prefix, l) if l > 0 else np.zeros((1, 3), np.int64)
        if w >= 1.0:
            split = count > 0
        else:
            split = count > leaf_max
        if l == MAX_DEPTH:
            split[:] = False
        L = Level(l=l, w=w, prefix=prefix, coords=coords, first=first, count=count,
                  parent=parent, leaf=~split)
        levels.append(L)
        if not split.any():
            L.child_first = np.zeros(L.n, np.int64)
            L.nchild = np.zeros(L.n, np.int64)
            break
        # children: unique level-(l+1) prefixes inside each split box
        shift = np.uint64(3 * (LEVEL_BITS - (l + 1)))
        cp, cf, cc, cpar = [], [], [], []
        child_first = np.zeros(L.n, np.int64)
        nchild = np.zeros(L.n, np.int64)
        nxt = 0
        for b in np.nonzero(split)[0]:
            s, c = int(first[b]), int(count[b])
            pk = keys[s:s + c] >> shift
            u, idx, cnt = np.unique(pk, return_index=True, return_counts=True)
            child_first[b] = nxt
            nchild[b] = u.shape[0]
            nxt += u.shape[0]
            cp.append(u)
            cf.append(idx + s)
            cc.append(cnt)
            cpar.append(np.full(u.shape[0], b, np.int64))
        L.child_first = child_first
        L.nchild = nchild
        prefix = np.concatenate(cp).astype(np.uint64)
        first = np.concatenate(cf).astype(np.int64)
        count = np.concatenate(cc).astype(np.int64)
        parent = np.concatenate(cpar)
        l += 1
    return Tree(K=K, W=W, N=N, leaf_max=leaf_max, keys=keys, perm=perm, levels=levels)


# ------------------------------------------------------------ directions ---

def n_cells(w: float) -> int:
    """Cells per face side for width-w boxes (reading of Sec. 2.2/4.1)."""
    return int(round(w))


def n_directions(w: float) -> int:
    return 6 * n_cells(w) ** 2


def _ceil_div(p, q):
    return -((-p) // q)


def direction(m: np.ndarray, n: int) -> np.ndarray:
    """Direction index of a nonzero integer offset m (..., 3) on the n x n face
    grids, cells closed, ties to the lexicographically first (face, i, j) with
    faces ordered +x, -x, +y, -y, +z, -z.  Index = (face * n + i) * n + j."""
    m = np.asarray(m, dtype=np.int64)
    am = np.abs(m)
    M = am.max(axis=-1)
    if np.any(M == 0):
        raise ValueError("zero offset has no direction")
    a = np.argmax(am == M[..., None], axis=-1)            # first axis at max
    ma = np.take_along_axis(m, a[..., None], axis=-1)[..., 0]
    face = 2 * a + (ma < 0)
    ob = np.where(a == 0, 1, 0)
    oc = np.where(a == 2, 1, 2)
    mb = np.take_along_axis(m, ob[..., None], axis=-1)[..., 0]
    mc = np.take_along_axis(m, oc[..., None], axis=-1)[..., 0]
    i = np.maximum(0, _ceil_div(n * (mb + M), 2 * M) - 1)
    j = np.maximum(0, _ceil_div(n * (mc + M), 2 * M) - 1)
    return (face * n + i) * n + j


def in_closed_cell(m: np.ndarray, cell: int, n: int) -> np.ndarray:
    """Whether offset m lies in the closed cone of face cell `cell` (n x n)."""
    m = np.asarray(m, dtype=np.int64)
    face, rem = divmod(cell, n * n)
    i, j = divmod(rem, n)
    a, neg = divmod(face, 2)
    M = np.abs(m).max(axis=-1)
    ma = m[..., a]
    ok = (np.abs(ma) == M) & (M > 0) & ((ma < 0) == bool(neg))
    others = [d for d in range(3) if d != a]
    for d, k in zip(others, (i, j)):
        t = n * (m[..., d] + M)          # cell k covers 2M k <= t <= 2M (k+1)
        ok &= (t >= 2 * M * k) & (t <= 2 * M * (k + 1))
    return ok


def parent_direction(dir_parent: np.ndarray, n_parent: int) -> np.ndarray:
    """Fig. 2 hierarchy: cell (f, i, j) of the 2w grid lies inside cell
    (f, i//2, j//2) of the w grid.  Maps a parent-width direction to the
    child-width direction whose wedge contains it."""
    d = np.asarray(dir_parent, dtype=np.int64)
    f, rem = np.divmod(d, n_parent * n_parent)
    i, j = np.divmod(rem, n_parent)
    nc = n_parent // 2
    return (f * nc + i // 2) * nc + j // 2


# -------------------------------------------------------- near-field tests ---

def hf_near(m: np.ndarray, w: float, rho: float = 1.0) -> np.ndarray:
    """A (offset m in units of w) is in N^B iff its closed box has a point within
    rho w^2 of B's centre:  sum_d max(0, 2|m_d| - 1)^2 <= 4 rho^2 w^2."""
    m = np.asarray(m, dtype=np.int64)
    t = np.maximum(0, 2 * np.abs(m) - 1)
    lim = int(round(4 * rho * rho * w * w))
    return (t * t).sum(axis=-1) <= lim


def hf_near_template(w: float) -> np.ndarray:
    """All offsets m with hf_near(m, w)."""
    R = int(math.ceil(w)) + 1
    r = np.arange(-R, R + 1)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return g[hf_near(g, w)]


# --------------------------------------------------------------- HF lists ---

@dataclass
class HFPairs:
    """M2L pairs at one HF level: target B, source A, offset m = (c_A - c_B)/w,
    B's incoming direction dir(m), A's outgoing direction dir(-m)."""
    l: int
    w: float
    tgt: np.ndarray
    src: np.ndarray
    m: np.ndarray
    dir_in: np.ndarray
    dir_out: np.ndarray


def hf_lists(tree: Tree) -> list:
    out = []
    for L in tree.hf_levels:
        if L.l == 0:
            continue
        P = tree.levels[L.l - 1]
        w = L.w
        tmpl = hf_near_template(2 * w)
        # near pairs of parents (P, P')
        nb = P.lookup(P.coords[:, None, :] + tmpl[None, :, :])     # (nP, T)
        pi, ti = np.nonzero(nb >= 0)
        pj = nb[pi, ti]
        tg, sr = [], []
        for a in range(8):
            for b in range(8):
                ok = (a < P.nchild[pi]) & (b < P.nchild[pj])
                tg.append((P.child_first[pi] + a)[ok])
                sr.append((P.child_first[pj] + b)[ok])
        tgt = np.concatenate(tg)
        src = np.concatenate(sr)
        m = L.coords[src] - L.coords[tgt]
        far = ~hf_near(m, w)
        tgt, src, m = tgt[far], src[far], m[far]
        order = np.lexsort((src, tgt))
        tgt, src, m = tgt[order], src[order], m[order]
        n = n_cells(w)
        out.append(HFPairs(l=L.l, w=w, tgt=tgt, src=src, m=m,
                           dir_in=direction(m, n), dir_out=direction(-m, n)))
    return out


def active_directions(tree: Tree, hf: list):
    """Per HF level, sorted unique (box, dir) pairs needing an outgoing and an
    incoming representation: those M2L uses, closed downward under the wedge
    hierarchy (a parent's direction L needs the child direction containing it).
    Returns {level: (out_keys, in_keys)} with key = box * ndir + dir."""
    by_level = {p.l: p for p in hf}
    act = {}
    parent_sets = None
    for L in tree.hf_levels:
        if L.l == 0:
            continue
        nd = n_directions(L.w)
        p = by_level.get(L.l)
        o = [] if p is None else [p.src * nd + p.dir_out]
        i = [] if p is None else [p.tgt * nd + p.dir_in]
        if parent_sets is not None:
            Pl = tree.levels[L.l - 1]
            ndp = n_directions(Pl.w)
            for lst, keys in ((o, parent_sets[0]), (i, parent_sets[1])):
                if keys.size == 0:
                    continue
                pb, pd = np.divmod(keys, ndp)
                cd = parent_direction(pd, n_cells(Pl.w))
                for c in range(8):
                    ok = c < Pl.nchild[pb]
                    lst.append((Pl.child_first[pb] + c)[ok] * nd + cd[ok])
        o = np.unique(np.concatenate(o)) if o else np.zeros(0, np.int64)
        i = np.unique(np.concatenate(i)) if i else np.zeros(0, np.int64)
        act[L.l] = (o.astype(np.int64), i.astype(np.int64))
        parent_sets = act[L.l]
    return act


# --------------------------------------------------------------- LF lists ---

def _touch(ca, la, cb, lb):
    """Closed boxes (integer coords at levels la, lb) touch or overlap."""
    L = max(la, lb)
    sa, sb = 1 << (L - la), 1 << (L - lb)
    alo, ahi = ca * sa, (ca + 1) * sa
    blo, bhi = cb * sb, (cb + 1) * sb
    return np.all((alo <= bhi) & (blo <= ahi), axis=-1)


COLLEAGUE_OFFSETS = np.stack(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij"),
                             axis=-1).reshape(-1, 3)


@dataclass
class LFLists:
    """Per LF level l, arrays of (target box, source (level, box)).
    U: leaf targets, sources leaves; V: same-level pairs; W: leaf targets,
    sources finer boxes; X: inverse of W."""
    U: list
    V: dict
    W: list
    X: list


def lf_lists(tree: Tree) -> LFLists:
    U, W = [], []
    V = {}
    levels = tree.levels
    for L in tree.lf_levels:
        P = levels[L.l - 1]
        # V list: children of the parent's colleagues that do not touch B
        nb = P.lookup(P.coords[L.parent][:, None, :] + COLLEAGUE_OFFSETS[None])
        bi, ci = np.nonzero(nb >= 0)
        pc = nb[bi, ci]
        tg, sr = [], []
        for c in range(8):
            ok = c < P.nchild[pc]
            tg.append(bi[ok])
            sr.append((P.child_first[pc] + c)[ok])
        tgt = np.concatenate(tg)
        src = np.concatenate(sr)
        m = L.coords[src] - L.coords[tgt]
        far = np.abs(m).max(axis=1) >= 2
        tgt, src = tgt[far], src[far]
        order = np.lexsort((src, tgt))
        V[L.l] = (tgt[order], src[order], m[far][order])

    # U and W for leaves.  Same-level colleagues and coarser touching leaves
    # are found with vectorised lookups; descents into finer colleagues (only
    # present where the LF tree is adaptive) run as a plain loop.
    for L in tree.lf_levels:
        leaves = np.nonzero(L.leaf)[0]
        if leaves.size == 0:
            continue
        cb = L.coords[leaves]
        # coarser leaves touching b: colleagues of b's LF ancestors that are leaves
        anc = leaves.copy()
        for la in range(L.l - 1, -1, -1):
            anc = levels[la + 1].parent[anc]
            A = levels[la]
            if A.hf:
                break
            nbr = A.lookup(A.coords[anc][:, None, :] + COLLEAGUE_OFFSETS[None])
            bi, ci = np.nonzero(nbr >= 0)
            a = nbr[bi, ci]
            ok = A.leaf[a] & _touch(A.coords[a], la, cb[bi], L.l)
            for b_, a_ in zip(leaves[bi[ok]], a[ok]):
                U.append((L.l, int(b_), la, int(a_)))
        nbr = L.lookup(cb[:, None, :] + COLLEAGUE_OFFSETS[None])
        bi, ci = np.nonzero(nbr >= 0)
        c = nbr[bi, ci]
        lf = L.leaf[c]
        U.extend(np.stack([np.full(lf.sum(), L.l), leaves[bi[lf]],
                           np.full(lf.sum(), L.l), c[lf]], axis=1).tolist())
        for b_, c_ in zip(leaves[bi[~lf]], c[~lf]):
            cbb = L.coords[b_]
            stack = [(L.l, int(c_))]
            while stack:
                lc, bc = stack.pop()
                Lc = levels[lc]
                La = levels[lc + 1]
                for k in range(int(Lc.nchild[bc])):
                    a = int(Lc.child_first[bc] + k)
                    if _touch(La.coords[a], lc + 1, cbb, L.l):
                        if La.leaf[a]:
                            U.append((L.l, int(b_), lc + 1, a))
                        else:
                            stack.append((lc + 1, a))
                    else:
                        W.append((L.l, int(b_), lc + 1, a))
    X = [(la, a, lb, b) for (lb, b, la, a) in W]
    U = np.array(U, dtype=np.int64).reshape(-1, 4)
    W = np.array(W, dtype=np.int64).reshape(-1, 4)
    X = np.array(X, dtype=np.int64).reshape(-1, 4)
    return LFLists(U=U, V=V, W=W, X=X)
