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


_WORKER = {}


def _worker_init(points, f):
    _WORKER["points"] = points
    _WORKER["f"] = f


def _worker_run(targets):
    return direct(_WORKER["points"], _WORKER["f"], targets, chunk=8)


class DirectPool:
    """direct() on a sample of targets spread over `workers` processes (one per
    host core): the same sums, split by target (equal up to the summation order
    of the BLAS product).  The processes are started with
    `spawn` (safe after CUDA has been initialised in the parent) and keep the
    points and densities; each runs single-threaded numpy."""

    def __init__(self, points: np.ndarray, f: np.ndarray, workers: int):
        import multiprocessing as mp
        import os
        self.workers = max(1, int(workers))
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        old = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(
                self.workers, initializer=_worker_init,
                initargs=(np.ascontiguousarray(points), np.atleast_2d(np.asarray(f, dtype=np.complex128))))
            self.pool.map(_worker_run, [np.zeros(0, dtype=np.int64)] * self.workers)   # started
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, targets: np.ndarray) -> np.ndarray:
        parts = [p for p in np.array_split(np.asarray(targets), self.workers) if p.size]
        return np.concatenate(self.pool.map(_worker_run, parts), axis=1)

    def close(self):
        self.pool.close()
        self.pool.join()


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
