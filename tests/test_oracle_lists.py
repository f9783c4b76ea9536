"""Pins of the oracle's Morton order, octree, directions and lists (Sec. 2.2)
to hand-computed keys, brute force and the paper's invariants (Prop. 1,
hierarchical wedges of Fig. 2, exact coverage of all pairs by Alg. 1, the
per-level counts behind the complexity bounds of Sec. 3.4-3.5)."""
import math

import numpy as np
import pytest

import workloads
from oracle import octree as ot


# ------------------------------------------------------------ Morton ---

def test_morton_hand_computed_keys():
    W = 8.0
    h = W / 2 ** 21
    q = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 5, 6]])
    pts = -W / 2 + (q + 0.5) * h
    keys = ot.interleave(ot.quantize(pts, W))
    # (3,5,6): bit0 x1 y1 z0 -> 6; bit1 x1 y0 z1 -> 5; bit2 x0 y1 z1 -> 3
    assert keys.tolist() == [0, 4, 2, 1, 6 + (5 << 3) + (3 << 6)]
    assert np.array_equal(ot.deinterleave(keys, 21), q)


def test_quantize_faces_and_clamp():
    W = 8.0
    pts = np.array([[0.0, 0.0, 0.0], [4.0, 4.0, 4.0], [-4.0, -4.0, -4.0]])
    q = ot.quantize(pts, W)
    assert q[0].tolist() == [2 ** 20] * 3          # internal face -> upper box
    assert q[1].tolist() == [2 ** 21 - 1] * 3      # root's upper face clamped
    assert q[2].tolist() == [0, 0, 0]


def test_root_width_power_of_two():
    assert ot.root_width(8) == 8 and ot.root_width(5) == 8 and ot.root_width(64) == 64
    assert ot.root_width(0.7) == 1


def test_tree_splits_and_partitions():
    p = workloads.clustered(8.0, 1, 3000)
    T = ot.build_tree(p, 8.0, leaf_max=16)
    seen = np.zeros(p.shape[0], int)
    for L in T.levels:
        assert np.all(np.diff(L.prefix.astype(np.int64)) > 0)
        if L.hf:
            assert not L.leaf.any()                      # every non-empty HF box splits
        else:
            assert np.array_equal(L.leaf, L.count <= 16) or L.l == ot.MAX_DEPTH
        for b in np.nonzero(L.leaf)[0]:
            seen[L.first[b]:L.first[b] + L.count[b]] += 1
        if L.l > 0:
            P = T.levels[L.l - 1]
            assert np.all(P.child_first[L.parent] <= np.arange(L.n))
    assert np.all(seen == 1)
    assert any(not L.hf and L.leaf.any() and L.l > T.level_of_width(0.5) for L in T.levels)


# -------------------------------------------------------- directions ---

@pytest.mark.parametrize("n", [1, 2, 4])
def test_direction_is_first_closed_cell(n):
    r = np.arange(-6, 7)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.abs(m).max(1) > 0]
    d = ot.direction(m, n)
    nd = 6 * n * n
    member = np.stack([ot.in_closed_cell(m, c, n) for c in range(nd)], axis=1)
    assert member.any(axis=1).all()
    first = np.argmax(member, axis=1)                   # lexicographic (face, i, j)
    assert np.array_equal(d, first)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_hierarchical_wedges(n):
    # Fig. 2: the wedge of a parent cell (2n grid) lies in the child cell it maps to
    r = np.arange(-9, 10)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.abs(m).max(1) > 0]
    for L in range(6 * (2 * n) ** 2):
        inside = ot.in_closed_cell(m, L, 2 * n)
        c = int(ot.parent_direction(np.array([L]), 2 * n)[0])
        assert ot.in_closed_cell(m[inside], c, n).all()


def test_near_field_at_w1_is_the_colleagues_and_has_no_ties():
    t = ot.hf_near_template(1.0)
    assert len(t) == 27 and np.abs(t).max() == 1
    for w in (1, 2, 4, 8, 16):
        R = w + 2
        r = np.arange(-R, R + 1)
        m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
        s = (np.maximum(0, 2 * np.abs(m) - 1) ** 2).sum(1)
        assert not np.any(s == 4 * w * w)


def _box_closest_dist(cB, cA, w):
    g = np.maximum(0.0, np.abs(cA - cB) - w / 2)
    return np.sqrt((g * g).sum(-1))


# ------------------------------------------------------------ HF lists ---

def test_hf_lists_match_brute_force_and_separation():
    p = workloads.sphere(8.0, 0, n=3000)
    T = ot.build_tree(p, 8.0)
    hf = {h.l: h for h in ot.hf_lists(T)}
    for L in T.hf_levels:
        if L.l == 0:
            continue
        P = T.levels[L.l - 1]
        B, A = np.meshgrid(np.arange(L.n), np.arange(L.n), indexing="ij")
        B, A = B.ravel(), A.ravel()
        m = L.coords[A] - L.coords[B]
        pm = P.coords[L.parent[A]] - P.coords[L.parent[B]]
        keep = ot.hf_near(pm, P.w) & ~ot.hf_near(m, L.w)
        want = set(zip(B[keep].tolist(), A[keep].tolist()))
        h = hf[L.l]
        got = set(zip(h.tgt.tolist(), h.src.tolist()))
        assert got == want
        if h.tgt.size:
            C = L.centers(T.W)
            # separation: A has no point within w^2 of c_B (near-field reading)
            assert np.all(_box_closest_dist(C[h.tgt], C[h.src], L.w) > L.w ** 2)
            n = ot.n_cells(L.w)
            for k in range(0, h.tgt.size, max(1, h.tgt.size // 200)):
                assert ot.in_closed_cell(h.m[k], h.dir_in[k], n)
                assert ot.in_closed_cell(-h.m[k], h.dir_out[k], n)


@pytest.mark.parametrize("K", [4.0, 8.0, 16.0])
def test_prop1_no_interactions_at_top(K):
    p = workloads.sphere(K, 2, n=4000)
    T = ot.build_tree(p, K)
    for h in ot.hf_lists(T):
        if h.w >= 2 * math.sqrt(K):
            assert h.tgt.size == 0


# ----------------------------------------------------------- coverage ---

def test_every_pair_covered_exactly_once():
    """Alg. 1 + near field: each ordered pair (i, j) is covered by exactly one
    of P2P (U), LF-M2L (V), M2P (W), P2L (X) or an HF-M2L pair."""
    p = workloads.clustered(8.0, 3, 1500, n_clusters=3, spread=0.08)
    T = ot.build_tree(p, 8.0, leaf_max=8)
    hf = ot.hf_lists(T)
    lf = ot.lf_lists(T)
    assert lf.W.shape[0] > 0 and lf.X.shape[0] > 0
    N = p.shape[0]
    cover = np.zeros((N, N), np.int32)
    lv = T.levels

    def pts(l, b):
        return np.arange(lv[l].first[b], lv[l].first[b] + lv[l].count[b])

    for (lb, b, la, a) in lf.U:
        cover[np.ix_(pts(lb, b), pts(la, a))] += 1
    for (lb, b, la, a) in lf.W:
        cover[np.ix_(pts(lb, b), pts(la, a))] += 1
    for (lb, b, la, a) in lf.X:
        cover[np.ix_(pts(lb, b), pts(la, a))] += 1
    for l, (tg, sr, _) in lf.V.items():
        for b, a in zip(tg, sr):
            cover[np.ix_(pts(l, b), pts(l, a))] += 1
    for h in hf:
        for b, a in zip(h.tgt, h.src):
            cover[np.ix_(pts(h.l, b), pts(h.l, a))] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_v_pairs_do_not_touch():
    p = workloads.sphere(8.0, 0, n=3000)
    T = ot.build_tree(p, 8.0)
    lf = ot.lf_lists(T)
    for l, (tg, sr, m) in lf.V.items():
        assert np.all(np.abs(m).max(1) >= 2)
        assert np.array_equal(m, T.levels[l].coords[sr] - T.levels[l].coords[tg])


def test_active_directions_closed_under_hierarchy():
    p = workloads.sphere(8.0, 0, n=4000)
    T = ot.build_tree(p, 8.0)
    hf = [h for h in ot.hf_lists(T) if h.tgt.size]
    act = ot.active_directions(T, hf)
    for h in hf:
        nd = ot.n_directions(h.w)
        assert np.isin(h.src * nd + h.dir_out, act[h.l][0]).all()
        assert np.isin(h.tgt * nd + h.dir_in, act[h.l][1]).all()
    # both sides: outgoing (HF-M2M reads the children's direction containing
    # the parent's) and incoming (HF-L2L writes it)
    checked = 0
    for side in (0, 1):
        for l in act:
            if l + 1 in act and act[l][side].size:
                P, L = T.levels[l], T.levels[l + 1]
                ndp, nd = ot.n_directions(P.w), ot.n_directions(L.w)
                pb, pdir = np.divmod(act[l][side], ndp)
                cd = ot.parent_direction(pdir, ot.n_cells(P.w))
                for k in range(8):
                    ok = k < P.nchild[pb]
                    need = (P.child_first[pb[ok]] + k) * nd + cd[ok]
                    assert np.isin(need, act[l + 1][side]).all()
                    checked += need.size
    assert checked > 0
    # nothing beyond the closure: every active key is used by an M2L pair or
    # needed by an active key of the parent level
    for side in (0, 1):
        for l in act:
            L = T.levels[l]
            nd = ot.n_directions(L.w)
            used = set()
            h = next((q for q in hf if q.l == l), None)
            if h is not None:
                used |= set((h.src * nd + h.dir_out if side == 0 else h.tgt * nd + h.dir_in).tolist())
            if l - 1 in act:
                P = T.levels[l - 1]
                ndp = ot.n_directions(P.w)
                pb, pdir = np.divmod(act[l - 1][side], ndp)
                cd = ot.parent_direction(pdir, ot.n_cells(P.w))
                for k in range(8):
                    ok = k < P.nchild[pb]
                    used |= set(((P.child_first[pb[ok]] + k) * nd + cd[ok]).tolist())
            assert set(act[l][side].tolist()) == used


def test_hf_work_per_level_scales_as_a_surface():
    """The counting behind the complexity bounds of Sec. 3.4-3.5 (Prop. 2 and 4),
    for points sampled from a surface with N = O(K^2): a level of width w has
    O(K^2 / w^2) non-empty boxes, each target (box, direction) O(1) interaction
    partners, so each HF level O(K^2) M2L pairs.  On spheres of diameter 16 and
    32 (same sampling density): boxes x w^2 / K^2 stays between 3 and 6, the
    w = 1 pair count grows with K^2, and the mean number of pairs per target
    state stays put as K doubles."""
    stats = {}
    for K in (16.0, 32.0):
        T = ot.build_tree(workloads.sphere(K, 1), K, 64)
        for q in ot.hf_lists(T):
            if q.tgt.size == 0:
                continue
            nd = ot.n_directions(q.w)
            states = np.unique(q.tgt * nd + q.dir_in).size
            stats[(K, q.w)] = (T.levels[q.l].n, q.tgt.size, q.tgt.size / states)
    for (K, w), (boxes, pairs, per_state) in stats.items():
        if w <= 2:
            assert 3.0 <= boxes * w * w / (K * K) <= 6.0, (K, w, boxes)
            assert per_state <= 40.0, (K, w, per_state)
    ratio = stats[(32.0, 1.0)][1] / stats[(16.0, 1.0)][1]
    assert 3.5 <= ratio <= 4.5, ratio                       # O(K^2) pairs at a level
    a, b = stats[(16.0, 1.0)][2], stats[(32.0, 1.0)][2]
    assert abs(a - b) <= 0.2 * max(a, b), (a, b)            # O(1) per target state
