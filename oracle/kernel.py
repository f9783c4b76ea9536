"""Oracle: the Helmholtz kernel of Eq. 1 in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

G(x, y) = exp(2 pi i |x - y|) / |x - y|  (wavelength 1, Sec. 1).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def G(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Kernel matrix G(X_i, Y_j) for X (m, 3), Y (n, 3); complex128 (m, n)."""
    d = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=-1))
    return np.exp(1j * TWO_PI * d) / d


def G_pairs(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Kernel for matched rows: G(X_i, Y_i)."""
    d = np.sqrt(((X - Y) ** 2).sum(axis=-1))
    return np.exp(1j * TWO_PI * d) / d
