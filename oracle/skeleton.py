"""Oracle: directional and non-directional low-rank skeletons (Eq. 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. 2 (Sec. 2.1): for sources y in a box Y and targets x in a far region X,
    G(x, y) ~= G(x, b) D G(a, y),   D = G(a, b)^{-1},
with r equivalent points b in the box and r check points a in the far region.
The paper obtains {a}, {b} by random sampling and pivoted QR (Sec. 2.1, citing
Engquist-Ying 2010, which is not available).  The reading implemented here:

  1. Draw S_Y points in the box (half on its surface, half inside) and S_X
     points in the far region where this representation is ever evaluated
     (region_hf / region_lf).
  2. Column-pivoted Householder QR of a random +-1 row sketch of the
     row-weighted G(X_s, Y_s) (weight |x|, so every target counts relative
     to its own potential) orders the box samples; the rank r is the number
     of pivots with |R_kk| > eps_op |R_00|.  The first r pivots are the
     equivalent points b, the first 2r the box check points b2.
  3. Two rounds of column-pivoted QR on the transpose of the weighted
     G(X_s, b) pick 2r far check points a2; the first r are the incoming
     equivalent points (reciprocity, G(x, y) = G(y, x)).
  4. D of Eq. 2 is applied in least-squares form over the 2r check points
     (PlainRep below is the paper's own form, D = G(a, b)^{-1}, on the same
     skeleton; the FMM runs on either),
     and the equivalent charges are carried in the basis that is orthonormal
     on the weighted check points:  with  W G(a2, b) = Q_o R_o,
         outgoing state  s = Q_o^H W u(a2)        (u = check potentials),
         its field       phi(x) s,   phi(x) = G(x, b) R_o^{-1};
     and with  G(b2, a_in) W = Q_i R_i,
         incoming state  t = Q_i^H v(b2)          (v = check potentials),
         its field       psi(y) t,   psi(y) = G(y, a_in) W R_i^{-1}.
     Every translation operator is then a product of bounded factors
     (an orthonormal projection and a basis evaluated inside its region),
     formed in FP64, which keeps single-precision application stable.

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014) used as a
counter-based generator: the k-th draw of stream s is mix(s + (k+1) * gamma).
Only +, *, floor and integer operations turn draws into sample points, so the
samples are reproducible bit for bit.

Rotational invariance (Sec. 2.2: operators depend only on size and accuracy):
G(Qx, Qy) = G(x, y) for the 48 signed permutations Q of the cube, which map
face cells to face cells.  Skeletons are computed for one cell per orbit and
mapped to the others.  Sample regions are built from closed cells and
sign-symmetric tests so that the region of Q(cell) is Q(region of cell).
"""
from __future__ import annotations

import functools
import itertools
import math
from dataclasses import dataclass

import numpy as np

from . import octree as ot
from .kernel import G

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(x: int) -> int:
    """SplitMix64 output function applied to the 64-bit state x."""
    z = x & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class Stream:
    """Counter-based uniform doubles in [0, 1): (mix(seed + (k+1) gamma) >> 11) * 2^-53."""

    def __init__(self, seed: int):
        self.seed = seed & MASK64
        self.k = 0

    def next(self) -> float:
        self.k += 1
        z = splitmix64(self.seed + self.k * GAMMA)
        return (z >> 11) * (1.0 / 9007199254740992.0)

    def below(self, n: int) -> int:
        """Integer in [0, n)."""
        return min(int(math.floor(self.next() * n)), n - 1)


def stream_seed(kind: int, w: float, cell: int, w_top: float, tol_code: int) -> int:
    """64-bit seed of the sample stream of one skeleton."""
    h = 0x243F6A8885A308D3
    for v in (kind, int(round(w * 1024)), cell, int(round(w_top * 1024)), tol_code):
        h = splitmix64(h ^ (v & MASK64))
    return h


# -------------------------------------------------------- cube symmetry ---

SYMMETRIES = [(perm, signs) for perm in itertools.permutations(range(3))
              for signs in itertools.product((1, -1), repeat=3)]


def apply_sym(sym, x: np.ndarray) -> np.ndarray:
    """(Qx)_k = s_k x_{perm[k]}."""
    perm, signs = sym
    return x[..., list(perm)] * np.array(signs, dtype=x.dtype)


def cell_center_dir(cell: int, n: int) -> np.ndarray:
    face, rem = divmod(cell, n * n)
    i, j = divmod(rem, n)
    a, neg = divmod(face, 2)
    v = np.zeros(3)
    v[a] = -1.0 if neg else 1.0
    others = [d for d in range(3) if d != a]
    v[others[0]] = 2 * (i + 0.5) / n - 1
    v[others[1]] = 2 * (j + 0.5) / n - 1
    return v


def cell_of_dir(v: np.ndarray, n: int) -> int:
    a = int(np.argmax(np.abs(v)))
    M = abs(v[a])
    face = 2 * a + (1 if v[a] < 0 else 0)
    others = [d for d in range(3) if d != a]
    i = min(n - 1, int(math.floor(n * (v[others[0]] / M + 1) / 2)))
    j = min(n - 1, int(math.floor(n * (v[others[1]] / M + 1) / 2)))
    return (face * n + i) * n + j


def canonical_cells(n: int):
    """For every cell: (canonical cell, index of the symmetry Q with
    Q(canonical) = cell).  Canonical = smallest cell index of the orbit."""
    nd = 6 * n * n
    img = np.zeros((len(SYMMETRIES), nd), np.int64)
    for s, sym in enumerate(SYMMETRIES):
        for c in range(nd):
            img[s, c] = cell_of_dir(apply_sym(sym, cell_center_dir(c, n)), n)
    canon = np.zeros(nd, np.int64)
    which = np.zeros(nd, np.int64)
    for c in range(nd):
        # orbit of c = {img[s, c]}; canonical = min over orbit
        k = int(img[:, c].min())
        canon[c] = k
        # symmetry mapping k -> c
        which[c] = int(np.nonzero(img[:, k] == c)[0][0])
    return canon, which


# ----------------------------------------------------------- sample regions ---

def box_samples(st: Stream, w: float, S: int) -> np.ndarray:
    y = np.empty((S, 3))
    for q in range(S):
        for d in range(3):
            y[q, d] = (st.next() - 0.5) * w
    return y


def _closed_cell_range(M: int, k: int, n: int):
    """Integer m_b with 2Mk <= n (m_b + M) <= 2M(k+1)."""
    lo = -((-(2 * M * k)) // n) - M
    hi = (2 * M * (k + 1)) // n - M
    return lo, hi


def _hf_box_point(st: Stream, cw: float, cell: int) -> np.ndarray:
    """A point of a width-cw box that can be in the interaction list of a
    width-cw box at the origin, with offset in the closed cell `cell`."""
    n = ot.n_cells(cw)
    face, rem = divmod(cell, n * n)
    i, j = divmod(rem, n)
    a, neg = divmod(face, 2)
    others = [d for d in range(3) if d != a]
    Mmax = 4 * int(round(cw)) + 2
    for _ in range(100000):
        oB = st.below(8)
        M = 1 + st.below(Mmax)
        m = np.zeros(3, np.int64)
        m[a] = -M if neg else M
        for d, k in zip(others, (i, j)):
            lo, hi = _closed_cell_range(M, k, n)
            m[d] = lo + st.below(hi - lo + 1)
        ob = np.array([(oB >> 2) & 1, (oB >> 1) & 1, oB & 1], np.int64)
        if ot.hf_near(m, cw):
            continue
        if not ot.hf_near((ob + m) // 2, 2 * cw):
            continue
        x = np.empty(3)
        for d in range(3):
            x[d] = cw * m[d] + (st.next() - 0.5) * cw
        return x
    raise RuntimeError("rejection sampling did not terminate")


def _hf_point(st: Stream, w: float, cell: int, w_top: float) -> np.ndarray:
    kmax = int(round(math.log2(w_top / w)))
    u = st.next()
    k = 0 if (kmax == 0 or u < 0.6) else min(kmax, 1 + int(math.floor((u - 0.6) * 2.5 * kmax)))
    shift = np.zeros(3)
    cw = w
    n = ot.n_cells(cw)
    for _ in range(k):
        o = st.below(8)
        ob = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1], np.float64)
        shift = shift - (ob - 0.5) * cw
        face, rem = divmod(cell, n * n)
        i, j = divmod(rem, n)
        di, dj = st.below(2), st.below(2)
        n2 = 2 * n
        cell = (face * n2 + 2 * i + di) * n2 + 2 * j + dj
        cw *= 2
        n = n2
    return shift + _hf_box_point(st, cw, cell)


def region_hf(st: Stream, w: float, cell: int, w_top: float, S: int) -> np.ndarray:
    """S samples of the region where the width-w, direction-`cell` outgoing
    representation is evaluated (relative to the box centre): boxes of the
    interaction list in that closed wedge, and (recursively, up to width
    w_top) the parent's region seen from the child."""
    return np.array([_hf_point(st, w, cell, w_top) for _ in range(S)])


def _lf_point(st: Stream, w: float, w_top: float) -> np.ndarray:
    u = st.next()
    if u < 0.4:
        # a box of the V list (child of the parent's colleague, not touching)
        while True:
            oB = st.below(8)
            ob = np.array([(oB >> 2) & 1, (oB >> 1) & 1, oB & 1], np.int64)
            m = np.array([st.below(7) - 3 for _ in range(3)], np.int64)
            if np.abs(m).max() < 2:
                continue
            if np.abs((ob + m) // 2).max() > 1:
                continue
            return np.array([w * m[d] + (st.next() - 0.5) * w for d in range(3)])
    if u < 0.6:
        # the exterior shell 1.5 w <= |x|_inf <= 6 w (W and X lists)
        R = 1.5 * w + st.next() * 4.5 * w
        face = st.below(6)
        a, neg = divmod(face, 2)
        x = np.empty(3)
        for d in range(3):
            x[d] = (2 * st.next() - 1) * R
        x[a] = -R if neg else R
        return x
    # the parent's region, seen from this child
    o = st.below(8)
    ob = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1], np.float64)
    shift = -(ob - 0.5) * w
    if 2 * w < 1.0:
        return shift + _lf_point(st, 2 * w, w_top)
    return shift + _hf_point(st, 2 * w, st.below(6), w_top)


def region_lf(st: Stream, w: float, w_top: float, S: int) -> np.ndarray:
    """S samples of the far region of an LF box of width w: V-list boxes, the
    exterior shell around the colleague block, and the parent's region."""
    return np.array([_lf_point(st, w, w_top) for _ in range(S)])


# ---------------------------------------------------------- pivoted QR ---

def pivoted_qr_pivots(A: np.ndarray, tol: float, rmax: int | None = None):
    """Column-pivoted Householder QR, plain loop, column norms recomputed at
    every step.  Returns (pivot columns in order, |R_kk|), stopping when the
    largest remaining column norm is <= tol * |R_00| or after rmax steps."""
    A = np.array(A, dtype=np.complex128, copy=True)
    m, n = A.shape
    cols = np.arange(n)
    piv, diag = [], []
    kmax = min(m, n) if rmax is None else min(m, n, rmax)
    r00 = None
    for k in range(kmax):
        norms = np.sqrt((A[k:, k:].real ** 2 + A[k:, k:].imag ** 2).sum(axis=0))
        j = int(np.argmax(norms))
        nk = float(norms[j])
        if r00 is None:
            r00 = nk
        if nk <= tol * r00 or nk == 0.0:
            break
        A[:, [k, k + j]] = A[:, [k + j, k]]
        cols[[k, k + j]] = cols[[k + j, k]]
        piv.append(int(cols[k]))
        diag.append(nk)
        x = A[k:, k]
        alpha = x[0]
        phase = alpha / abs(alpha) if abs(alpha) > 0 else 1.0
        v = x.copy()
        v[0] += phase * nk
        vn = float(np.vdot(v, v).real)
        A[k:, k:] -= np.outer(v, (2.0 / vn) * (v.conj() @ A[k:, k:]))
    return piv, diag


def rademacher(seed: int, rows: int, cols: int) -> np.ndarray:
    """+-1 matrix from SplitMix64 draws (vectorised; entry k in row-major
    order is the k-th draw: +1 if its top bit is clear)."""
    k = np.arange(1, rows * cols + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return np.where((z >> np.uint64(63)) == 0, 1.0, -1.0).reshape(rows, cols)


# --------------------------------------------------------------- skeleton ---

@dataclass(frozen=True)
class SkelParams:
    eps_op: float
    S_Y: int = 1024
    S_X: int = 4096
    sketch: int = 400


@dataclass
class Rep:
    """One representation type: box width w and face cell (-1 = LF), in the
    box's local frame."""
    w: float
    cell: int
    r: int
    b2: np.ndarray       # (2r, 3) box check points; b = b2[:r] equivalent points
    a2: np.ndarray       # (2r, 3) far check points; a_in = a2[:r]
    Wa2: np.ndarray      # (2r,) weights |a2|
    Qo: np.ndarray       # (2r, r)
    Ro_inv: np.ndarray   # (r, r)
    Qi: np.ndarray       # (2r, r)
    Ri_inv: np.ndarray   # (r, r)

    @property
    def b(self):
        return self.b2[:self.r]

    @property
    def a_in(self):
        return self.a2[:self.r]

    def phi(self, x: np.ndarray) -> np.ndarray:
        """Outgoing basis at points x (local frame): (m, r)."""
        return G(x, self.b) @ self.Ro_inv

    def psi(self, y: np.ndarray) -> np.ndarray:
        """Incoming basis at points y (local frame): (m, r)."""
        return (G(y, self.a_in) * self.Wa2[None, :self.r]) @ self.Ri_inv

    def p_out(self) -> np.ndarray:
        """Check potentials at a2 -> outgoing state: (r, 2r)."""
        return self.Qo.conj().T * self.Wa2[None, :]

    def p_in(self) -> np.ndarray:
        """Check potentials at b2 -> incoming state: (r, 2r)."""
        return self.Qi.conj().T

    def mapped(self, sym, cell: int) -> "Rep":
        return Rep(self.w, cell, self.r, apply_sym(sym, self.b2), apply_sym(sym, self.a2),
                   self.Wa2, self.Qo, self.Ro_inv, self.Qi, self.Ri_inv)

    def plain(self) -> "PlainRep":
        """The same skeleton in the paper's own form of Eq. 2 (cached)."""
        if getattr(self, "_plain", None) is None:
            self._plain = PlainRep(self)
        return self._plain


class PlainRep:
    """Eq. 2 exactly as Sec. 2.1 states it, on the skeleton of a Rep:
    r equivalent points b = b2[:r] in the box and r check points a = a2[:r]
    in the far region, with the translation matrix D = G(a, b)^{-1}.

    Outgoing: the check potentials u(a) = sum_i G(a, y_i) f_i of the box's
    sources give the equivalent charges f_b = D u(a), whose field at a far x
    is G(x, b) f_b.  Incoming (the mirror image, reciprocity G(x, y) = G(y, x)):
    far equivalent points a with charges g = D_in v(b), D_in = G(b, a)^{-1},
    from the check potentials v(b) of the far sources; their field at y in the
    box is G(y, a) g.

    Same interface as Rep (p_out, phi, p_in, psi; the check-point matrices
    take all 2r check points and use the first r), so the FMM passes run
    unchanged on either form."""

    def __init__(self, rep: Rep):
        self.w, self.cell, self.r = rep.w, rep.cell, rep.r
        self.b2, self.a2 = rep.b2, rep.a2
        r = rep.r
        self.b = rep.b2[:r]
        self.a = rep.a2[:r]
        self.D_out = np.linalg.inv(G(self.a, self.b))
        self.D_in = np.linalg.inv(G(self.b, self.a))

    def p_out(self) -> np.ndarray:
        """Check potentials at a2 -> equivalent charges D u(a): (r, 2r)."""
        return np.hstack([self.D_out, np.zeros((self.r, self.r), np.complex128)])

    def phi(self, x: np.ndarray) -> np.ndarray:
        """Field at x of unit equivalent charges at b: (m, r)."""
        return G(x, self.b)

    def p_in(self) -> np.ndarray:
        """Check potentials at b2 -> incoming equivalent charges D_in v(b): (r, 2r)."""
        return np.hstack([self.D_in, np.zeros((self.r, self.r), np.complex128)])

    def psi(self, y: np.ndarray) -> np.ndarray:
        """Field at y (in the box) of unit equivalent charges at a: (m, r)."""
        return G(y, self.a)


def box_samples_mixed(st: Stream, w: float, S: int) -> np.ndarray:
    """S box samples: the first S/2 uniform on the box surface, the rest
    uniform inside."""
    h = 0.5 * w
    ns = S // 2
    y = np.empty((S, 3))
    for q in range(ns):
        face = st.below(6)
        a, neg = divmod(face, 2)
        for d in range(3):
            y[q, d] = (2.0 * st.next() - 1.0) * h
        y[q, a] = -h if neg else h
    y[ns:] = box_samples(st, w, S - ns)
    return y


def build_rep(Y: np.ndarray, X: np.ndarray, prm: SkelParams, sketch_seed: int,
              w: float, cell: int) -> Rep:
    Wx = np.linalg.norm(X, axis=1)
    A = Wx[:, None] * G(X, Y)
    Z = rademacher(sketch_seed, prm.sketch, X.shape[0]) @ A
    piv, diag = pivoted_qr_pivots(Z, 0.0, rmax=prm.sketch)
    diag = np.asarray(diag)
    r = int((diag > prm.eps_op * diag[0]).sum())
    if 2 * r > len(piv):
        raise RuntimeError(f"rank {r} too large for sketch {prm.sketch}")
    b2 = Y[piv[:2 * r]]
    b = b2[:r]
    A2 = (Wx[:, None] * G(X, b)).T
    p1, _ = pivoted_qr_pivots(A2, 0.0, rmax=r)
    rest = np.setdiff1d(np.arange(X.shape[0]), np.asarray(p1))
    p2, _ = pivoted_qr_pivots(A2[:, rest], 0.0, rmax=r)
    a2 = X[np.concatenate([np.asarray(p1), rest[np.asarray(p2)]])]
    Wa2 = np.linalg.norm(a2, axis=1)
    Qo, Ro = _qr_pos(Wa2[:, None] * G(a2, b))
    Qi, Ri = _qr_pos(G(b2, a2[:r]) * Wa2[None, :r])
    return Rep(w, cell, r, b2, a2, Wa2, Qo, np.linalg.inv(Ro), Qi, np.linalg.inv(Ri))


def _qr_pos(M: np.ndarray):
    """Thin QR with the diagonal of R made real positive (unique factors)."""
    Q, R = np.linalg.qr(M)
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return Q * ph[None, :], R * ph.conj()[:, None]


def _tol_code(eps_op: float) -> int:
    return int(round(-math.log10(eps_op) * 100))


@functools.lru_cache(maxsize=512)
def hf_rep(w: float, cell: int, w_top: float, prm: SkelParams) -> Rep:
    seed = stream_seed(1, w, cell, w_top, _tol_code(prm.eps_op))
    st = Stream(seed)
    Y = box_samples_mixed(st, w, prm.S_Y)
    X = region_hf(st, w, cell, w_top, prm.S_X)
    return build_rep(Y, X, prm, splitmix64(seed ^ 0x5DEECE66D), w, cell)


@functools.lru_cache(maxsize=64)
def lf_rep(w: float, w_top: float, prm: SkelParams) -> Rep:
    seed = stream_seed(2, w, 0, w_top, _tol_code(prm.eps_op))
    st = Stream(seed)
    Y = box_samples_mixed(st, w, prm.S_Y)
    X = region_lf(st, w, w_top, prm.S_X)
    return build_rep(Y, X, prm, splitmix64(seed ^ 0x5DEECE66D), w, -1)


class RepSet:
    """All representation types one FMM needs: HF per (width, cell), built
    for one canonical cell per symmetry orbit and mapped; LF per width."""

    def __init__(self, prm: SkelParams, w_top: float):
        self.prm = prm
        self.w_top = w_top
        self._canon = {}
        self._hf = {}
        self._lf = {}

    def canon(self, w: float):
        n = ot.n_cells(w)
        if n not in self._canon:
            self._canon[n] = canonical_cells(n)
        return self._canon[n]

    def hf(self, w: float, cell: int) -> Rep:
        key = (w, int(cell))
        if key not in self._hf:
            canon, which = self.canon(w)
            c0 = int(canon[cell])
            if (w, c0) not in self._hf:
                self._hf[(w, c0)] = hf_rep(w, c0, self.w_top, self.prm)
            base = self._hf[(w, c0)]
            self._hf[key] = base.mapped(SYMMETRIES[int(which[cell])], int(cell))
        return self._hf[key]

    def lf(self, w: float) -> Rep:
        if w not in self._lf:
            self._lf[w] = lf_rep(w, self.w_top, self.prm)
        return self._lf[w]
