"""Oracle: the sequential directional FMM of Alg. 1 in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Passes, in the order of Alg. 1 (Sec. 2.3):
  1. LF upward (postorder over w < 1): P2M at leaves, LF-M2M into parents.
  2. HF upward (w = 1 .. w_top): for each active direction l of B, HF-M2M
     from the children's direction l' whose wedge contains l (at w = 1 the
     children are LF boxes with non-directional representations).
  3. HF downward (w_top .. 1): HF-M2L from every A in I^B in direction l,
     using A's outgoing direction l' (the direction of B seen from A), then
     HF-L2L into the children (at w = 1 into the LF incoming states).
  4. LF downward (w < 1): LF-M2L over the V list, P2L over the X list,
     LF-L2L into children; at leaves L2P and M2P over the W list.
  5. Near field (not written in Alg. 1, implied by Eq. 1): P2P over U lists.

Representations and operators are those of oracle.skeleton: by default the
least-squares form of Eq. 2 (form="ls"), or with form="plain" the paper's own
form, equivalent charges D u on the r check points with D = G(a, b)^{-1}.
Every operator is grouped by its key (direction, octant or offset) and
applied with numpy matmul to the stacked states of its boxes.  With fp32=True
the operators and the states are rounded to complex64 and the translations
run in complex64, to estimate the effect of single precision.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import octree as ot
from . import skeleton as sk
from .kernel import G, TWO_PI


@dataclass
class FMMParams:
    eps: float
    leaf_max: int = 64
    eps_op_factor: float = 0.3     # eps_op = eps * factor
    S_Y: int = 1024
    S_X: int = 4096
    sketch: int = 400

    def skel(self) -> sk.SkelParams:
        return sk.SkelParams(eps_op=self.eps * self.eps_op_factor, S_Y=self.S_Y,
                             S_X=self.S_X, sketch=self.sketch)


def octant_offset(o: int, w_child: float) -> np.ndarray:
    """c_child - c_parent for child octant o = 4x + 2y + z bits."""
    ob = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1], np.float64)
    return (ob - 0.5) * w_child


class Plan:
    """Tree, lists and representations for one geometry."""

    def __init__(self, points: np.ndarray, K: float, prm: FMMParams):
        self.prm = prm
        self.points = np.asarray(points, dtype=np.float64)
        self.K = K
        self.tree = ot.build_tree(self.points, K, prm.leaf_max)
        self.hf = [p for p in ot.hf_lists(self.tree) if p.tgt.size > 0]
        self.lf = ot.lf_lists(self.tree)
        self.act = ot.active_directions(self.tree, self.hf)
        self.hf_levels = sorted({p.l for p in self.hf})
        # HF levels that carry states: from the finest HF level (w = 1) up to
        # the coarsest level with a non-empty interaction list.
        T = self.tree
        self.w_top = T.levels[min(self.hf_levels)].w if self.hf_levels else 1.0
        self.reps = sk.RepSet(prm.skel(), self.w_top)
        self.ys = self.points[T.perm]
        l1 = T.level_of_width(1.0)
        self.l_top = min(self.hf_levels) if self.hf_levels else l1
        self.l1 = l1
        self.centers = [L.centers(T.W) for L in T.levels]
        self.point_leaf = np.zeros(T.N, np.int64)
        self.point_level = np.zeros(T.N, np.int64)
        for L in T.lf_levels:
            for b in np.nonzero(L.leaf)[0]:
                s, c = L.first[b], L.count[b]
                self.point_leaf[s:s + c] = b
                self.point_level[s:s + c] = L.l

    def hf_rank(self, l: int, cell: int) -> int:
        return self.reps.hf(self.tree.levels[l].w, cell).r


# Translation operators (Alg. 1), each from the relative position of the two
# boxes alone (translation invariance, Sec. 2.2); every one maps the source
# box's state to the target box's state.

def m2m_operator(rep_parent, rep_child, delta: np.ndarray) -> np.ndarray:
    """Child outgoing state -> parent outgoing state; delta = c_child - c_parent.
    The child's field at the parent's check points (parent frame a2, i.e.
    a2 - delta in the child frame), projected by the parent."""
    return rep_parent.p_out() @ rep_child.phi(rep_parent.a2 - delta)


def m2l_operator(rep_tgt, rep_src, delta: np.ndarray) -> np.ndarray:
    """Source outgoing state -> target incoming state; delta = c_src - c_tgt.
    The source's field at the target's box check points."""
    return rep_tgt.p_in() @ rep_src.phi(rep_tgt.b2 - delta)


def l2l_operator(rep_child, rep_parent, delta: np.ndarray) -> np.ndarray:
    """Parent incoming state -> child incoming state; delta = c_child - c_parent.
    The parent's incoming field at the child's box check points."""
    return rep_child.p_in() @ rep_parent.psi(rep_child.b2 + delta)


def _mm(op, x, fp32):
    """op (r_t, r_s) applied to x (n, nrhs, r_s) -> (n, nrhs, r_t)."""
    if fp32:
        return np.einsum("ts,nks->nkt", op.astype(np.complex64), x.astype(np.complex64))
    return np.einsum("ts,nks->nkt", op, x)


def _rnd(x, fp32):
    return x.astype(np.complex64).astype(np.complex128) if fp32 else x


class _PlainForm:
    """The plan's representations in the paper's form of Eq. 2."""

    def __init__(self, reps: sk.RepSet):
        self.reps = reps

    def hf(self, w: float, cell: int):
        return self.reps.hf(w, cell).plain()

    def lf(self, w: float):
        return self.reps.lf(w).plain()


def fmm(plan: Plan, f: np.ndarray, fp32: bool = False, form: str = "ls") -> np.ndarray:
    """Potentials (nrhs, N) in the caller's point order for densities f (nrhs, N).
    form: "ls" (least-squares form of Eq. 2) or "plain" (D = G(a, b)^{-1})."""
    T = plan.tree
    f = np.atleast_2d(np.asarray(f, dtype=np.complex128))
    nrhs = f.shape[0]
    fs = f[:, T.perm].T.copy()                   # (N, nrhs), Morton order
    ys = plan.ys
    levels = T.levels
    if form not in ("ls", "plain"):
        raise ValueError("form must be 'ls' or 'plain'")
    reps = plan.reps if form == "ls" else _PlainForm(plan.reps)
    C = plan.centers

    # ---------------------------------------------------- 1. LF upward ---
    S_lf, T_lf = {}, {}
    for L in reversed(T.lf_levels):
        rep = reps.lf(L.w)
        S = np.zeros((L.n, nrhs, rep.r), np.complex128)
        leaves = np.nonzero(L.leaf)[0]
        Pout = rep.p_out()
        for b in leaves:                                        # P2M
            s, c = L.first[b], L.count[b]
            U = G(C[L.l][b] + rep.a2, ys[s:s + c]) @ fs[s:s + c]     # (2r, nrhs)
            S[b] = (Pout @ U).T
        if L.l + 1 < len(levels) and not L.leaf.all():          # LF-M2M
            Lc = levels[L.l + 1]
            rc = reps.lf(Lc.w)
            for o in range(8):
                op = m2m_operator(rep, rc, octant_offset(o, Lc.w))
                par = Lc.parent
                oc = _octant_of(Lc.coords)
                sel = np.nonzero(oc == o)[0]
                if sel.size:
                    np.add.at(S, par[sel], _mm(op, S_lf[Lc.l][sel], fp32))
        S_lf[L.l] = _rnd(S, fp32)

    # ---------------------------------------------------- 2. HF upward ---
    S_hf = {}
    for l in range(plan.l1, plan.l_top - 1, -1):
        L = levels[l]
        nd = ot.n_directions(L.w)
        keys = plan.act[l][0]
        box, dirs = np.divmod(keys, nd)
        rmax = max([reps.hf(L.w, d).r for d in np.unique(dirs)], default=0)
        S = np.zeros((keys.size, nrhs, rmax), np.complex128)
        Lc = levels[l + 1]
        oc = _octant_of(Lc.coords)
        for d in np.unique(dirs):
            rep = reps.hf(L.w, d)
            slots = np.nonzero(dirs == d)[0]
            pb = box[slots]
            for k in range(8):
                has = k < L.nchild[pb]
                ch = L.child_first[pb[has]] + k
                sl = slots[has]
                if ch.size == 0:
                    continue
                for o in np.unique(oc[ch]):
                    so = oc[ch] == o
                    if l == plan.l1:
                        rc = reps.lf(Lc.w)
                        src = S_lf[Lc.l][ch[so]]
                    else:
                        ndc = ot.n_directions(Lc.w)
                        cd = int(ot.parent_direction(np.array([d]), ot.n_cells(L.w))[0])
                        rc = reps.hf(Lc.w, cd)
                        ckeys = ch[so] * ndc + cd
                        pos = np.searchsorted(plan.act[l + 1][0], ckeys)
                        src = S_hf[l + 1][pos][:, :, :rc.r]
                    op = m2m_operator(rep, rc, octant_offset(int(o), Lc.w))
                    S[sl[so], :, :rep.r] += _mm(op, src, fp32)
        S_hf[l] = _rnd(S, fp32)

    # -------------------------------------------------- 3. HF downward ---
    T_hf = {}
    for l in range(plan.l_top, plan.l1 + 1):
        L = levels[l]
        nd = ot.n_directions(L.w)
        keys = plan.act[l][1]
        box, dirs = np.divmod(keys, nd)
        rmax = max([reps.hf(L.w, d).r for d in np.unique(dirs)], default=0)
        Tin = np.zeros((keys.size, nrhs, rmax), np.complex128)
        # HF-L2L from the parent level
        if l > plan.l_top:
            Lp = levels[l - 1]
            ndp = ot.n_directions(Lp.w)
            pkeys = plan.act[l - 1][1]
            pbox, pdirs = np.divmod(pkeys, ndp)
            oc = _octant_of(L.coords)
            for d in np.unique(pdirs):
                rp = reps.hf(Lp.w, d)
                cd = int(ot.parent_direction(np.array([d]), ot.n_cells(Lp.w))[0])
                rc = reps.hf(L.w, cd)
                slots = np.nonzero(pdirs == d)[0]
                pb = pbox[slots]
                for k in range(8):
                    has = k < Lp.nchild[pb]
                    ch = Lp.child_first[pb[has]] + k
                    sl = slots[has]
                    for o in np.unique(oc[ch]):
                        so = oc[ch] == o
                        op = l2l_operator(rc, rp, octant_offset(int(o), L.w))
                        pos = np.searchsorted(keys, ch[so] * nd + cd)
                        np.add.at(Tin, (pos, slice(None), slice(0, rc.r)),
                                  _mm(op, T_hf[l - 1][sl[so]][:, :, :rp.r], fp32))
        # HF-M2L over the interaction lists
        p = next((q for q in plan.hf if q.l == l), None)
        if p is not None:
            okeys = plan.act[l][0]
            mk = p.m[:, 0] * 1_000_003 + p.m[:, 1] * 1009 + p.m[:, 2]
            uniq, inv = np.unique(mk, return_inverse=True)
            order = np.argsort(inv, kind="stable")
            bounds = np.searchsorted(inv[order], np.arange(uniq.size + 1))
            for g in range(uniq.size):
                idx = order[bounds[g]:bounds[g + 1]]
                m = p.m[idx[0]]
                din, dout = int(p.dir_in[idx[0]]), int(p.dir_out[idx[0]])
                rb = reps.hf(L.w, din)
                ra = reps.hf(L.w, dout)
                op = m2l_operator(rb, ra, L.w * m)
                spos = np.searchsorted(okeys, p.src[idx] * nd + dout)
                tpos = np.searchsorted(keys, p.tgt[idx] * nd + din)
                np.add.at(Tin, (tpos, slice(None), slice(0, rb.r)),
                          _mm(op, S_hf[l][spos][:, :, :ra.r], fp32))
        T_hf[l] = _rnd(Tin, fp32)

    # -------------------------------------------------- 4. LF downward ---
    u = np.zeros((T.N, nrhs), np.complex128)
    for L in T.lf_levels:
        rep = reps.lf(L.w)
        Tin = np.zeros((L.n, nrhs, rep.r), np.complex128)
        oc = _octant_of(L.coords)
        Lp = levels[L.l - 1]
        if Lp.hf:
            # HF-L2L at w = 1 into the LF incoming states, summed over directions
            ndp = ot.n_directions(Lp.w)
            pkeys = plan.act[L.l - 1][1] if (L.l - 1) in plan.act else np.zeros(0, np.int64)
            pbox, pdirs = np.divmod(pkeys, ndp)
            for d in np.unique(pdirs):
                rp = reps.hf(Lp.w, d)
                slots = np.nonzero(pdirs == d)[0]
                pb = pbox[slots]
                for k in range(8):
                    has = k < Lp.nchild[pb]
                    ch = Lp.child_first[pb[has]] + k
                    sl = slots[has]
                    for o in np.unique(oc[ch]):
                        so = oc[ch] == o
                        op = l2l_operator(rep, rp, octant_offset(int(o), L.w))
                        np.add.at(Tin, ch[so], _mm(op, T_hf[L.l - 1][sl[so]][:, :, :rp.r], fp32))
        else:
            # LF-L2L from the LF parent
            rp = reps.lf(Lp.w)
            for o in range(8):
                sel = np.nonzero(oc == o)[0]
                if sel.size:
                    op = l2l_operator(rep, rp, octant_offset(o, L.w))
                    Tin[sel] += _mm(op, T_lf[Lp.l][L.parent[sel]], fp32)
        # LF-M2L over the V list
        tgt, src, m = plan.lf.V.get(L.l, (np.zeros(0, np.int64),) * 2 + (np.zeros((0, 3), np.int64),))
        if tgt.size:
            mk = (m[:, 0] + 3) * 49 + (m[:, 1] + 3) * 7 + (m[:, 2] + 3)
            for key in np.unique(mk):
                sel = np.nonzero(mk == key)[0]
                op = m2l_operator(rep, rep, L.w * m[sel[0]])
                np.add.at(Tin, tgt[sel], _mm(op, S_lf[L.l][src[sel]], fp32))
        # P2L over the X list (targets at this level)
        X = plan.lf.X
        for (lb, b, la, a) in X[X[:, 0] == L.l]:
            A = levels[la]
            s, c = A.first[a], A.count[a]
            V = G(C[L.l][b] + rep.b2, ys[s:s + c]) @ fs[s:s + c]
            Tin[b] += (rep.p_in() @ V).T
        Tin = _rnd(Tin, fp32)
        T_lf[L.l] = Tin
        # L2P at the leaves of this level
        for b in np.nonzero(L.leaf)[0]:
            s, c = L.first[b], L.count[b]
            u[s:s + c] += rep.psi(ys[s:s + c] - C[L.l][b]) @ Tin[b].T
    # M2P over the W list
    W = plan.lf.W
    for (lb, b, la, a) in W:
        Lb, La = levels[lb], levels[la]
        s, c = Lb.first[b], Lb.count[b]
        ra = reps.lf(La.w)
        u[s:s + c] += ra.phi(ys[s:s + c] - C[la][a]) @ S_lf[la][a].T

    # ------------------------------------------------------ 5. P2P (U) ---
    U = plan.lf.U
    for (lb, b, la, a) in U:
        Lb, La = levels[lb], levels[la]
        s, c = Lb.first[b], Lb.count[b]
        s2, c2 = La.first[a], La.count[a]
        d = np.sqrt(((ys[s:s + c, None, :] - ys[None, s2:s2 + c2, :]) ** 2).sum(-1))
        same = d == 0.0
        g = np.where(same, 0.0, np.exp(1j * TWO_PI * np.where(same, 1.0, d)) / np.where(same, 1.0, d))
        u[s:s + c] += g @ fs[s2:s2 + c2]

    out = np.empty((nrhs, T.N), np.complex128)
    out[:, T.perm] = u.T
    return out


def _octant_of(coords: np.ndarray) -> np.ndarray:
    """Child octant (4x + 2y + z) from integer box coordinates."""
    return ((coords[:, 0] & 1) << 2) | ((coords[:, 1] & 1) << 1) | (coords[:, 2] & 1)
