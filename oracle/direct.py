"""Oracle: the direct O(N^2) sum of Eq. 1 in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

u_i = sum_j G(p_i, p_j) f_j with G(x, y) = exp(2 pi i |x - y|) / |x - y|.
Reading of the self term (G(p, p) is infinite): every source j whose point is
bitwise equal to p_i is skipped, j = i included.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def direct(points: np.ndarray, f: np.ndarray, targets: np.ndarray | None = None,
           chunk: int = 256) -> np.ndarray:
    """Potentials at points[targets] (all points if targets is None).

    f: (nrhs, N) complex.  Returns (nrhs, len(targets)) complex128.
    """
    f = np.atleast_2d(np.asarray(f, dtype=np.complex128))
    N = points.shape[0]
    tix = np.arange(N) if targets is None else np.asarray(targets)
    out = np.zeros((f.shape[0], tix.shape[0]), dtype=np.complex128)
    for s in range(0, tix.shape[0], chunk):
        t = tix[s:s + chunk]
        d = np.sqrt(((points[t][:, None, :] - points[None, :, :]) ** 2).sum(axis=-1))
        same = d == 0.0
        d = np.where(same, 1.0, d)
        g = np.where(same, 0.0, np.exp(1j * TWO_PI * d) / d)
        out[:, s:s + chunk] = f @ g.T
    return out


def direct_loop(points: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Pure-Python double loop (tiny inputs only), for pinning direct()."""
    N = points.shape[0]
    f = np.atleast_2d(f)
    u = np.zeros((f.shape[0], N), dtype=np.complex128)
    for i in range(N):
        for j in range(N):
            dx = points[i, 0] - points[j, 0]
            dy = points[i, 1] - points[j, 1]
            dz = points[i, 2] - points[j, 2]
            d = (dx * dx + dy * dy + dz * dz) ** 0.5
            if d == 0.0:
                continue
            g = complex(np.cos(TWO_PI * d), np.sin(TWO_PI * d)) / d
            for k in range(f.shape[0]):
                u[k, i] += g * f[k, j]
    return u


def rel_err(u: np.ndarray, ref: np.ndarray) -> float:
    """Relative 2-norm error over all entries (the error measure of the tests)."""
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
