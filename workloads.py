"""Seeded synthetic workloads: surface point clouds and densities.

This module is shared by the tests, the benchmark and the CPU oracle. It holds
no arithmetic of the fast multipole method, only the input recipes:

* The paper samples triangulated scattering surfaces at about 10 points per
  wavelength and draws densities from a standard normal distribution (Sec. 4.2).
  The meshes (sphere, F16, submarine) are not available, so analytic surfaces
  stand in for them, sampled at 100 points per square wavelength (the 2-D
  density that 10 points per wavelength implies).
* Points satisfy |p|_inf <= K/2 so that they fit the root box of the octree
  (Eq. 1 states |p| <= K/2 in the Euclidean norm; every generator here meets it
  for the sphere, ellipsoid and torus).
* Densities: independent real and imaginary parts, each N(0, 1).

Every generator takes a numpy seed and is deterministic.
"""
from __future__ import annotations

import math

import numpy as np

POINTS_PER_SQ_WAVELENGTH = 100.0


def _unit_sphere(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def sphere_count(K: float) -> int:
    """Points on a sphere of diameter K at 100 points per square wavelength."""
    return int(POINTS_PER_SQ_WAVELENGTH * math.pi * K * K)


def sphere(K: float, seed: int, n: int | None = None) -> np.ndarray:
    """Uniform random points on the sphere of diameter K centred at the origin."""
    rng = np.random.default_rng(seed)
    n = sphere_count(K) if n is None else n
    return _unit_sphere(rng, n) * (0.5 * K)


def ellipsoid_area(a: float, b: float, c: float, nq: int = 2000) -> float:
    """Surface area of the ellipsoid with semi-axes a, b, c (midpoint quadrature
    over the unit sphere in (cos theta, phi))."""
    t = (np.arange(nq) + 0.5) / nq * 2.0 - 1.0          # cos(theta) in (-1, 1)
    p = (np.arange(2 * nq) + 0.5) / (2 * nq) * 2 * math.pi
    ct, ph = np.meshgrid(t, p, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    u1, u2, u3 = st * np.cos(ph), st * np.sin(ph), ct
    g = np.sqrt((b * c * u1) ** 2 + (a * c * u2) ** 2 + (a * b * u3) ** 2)
    return float(g.mean() * 4 * math.pi)


def ellipsoid_count(a: float, b: float, c: float) -> int:
    return int(round(POINTS_PER_SQ_WAVELENGTH * ellipsoid_area(a, b, c)))


def ellipsoid(a: float, b: float, c: float, seed: int, n: int | None = None) -> np.ndarray:
    """Area-uniform random points on the ellipsoid (a >= b >= c) by rejection:
    a uniform unit-sphere point u maps to (a u1, b u2, c u3) and is kept with
    probability sqrt((bc u1)^2 + (ac u2)^2 + (ab u3)^2) / (ab), the ratio of
    the surface elements."""
    assert a >= b >= c > 0
    rng = np.random.default_rng(seed)
    n = ellipsoid_count(a, b, c) if n is None else n
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = max(1024, int(1.5 * (n - out.shape[0])))
        u = _unit_sphere(rng, m)
        acc = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2) / (a * b)
        keep = rng.random(m) < acc
        out = np.concatenate([out, u[keep] * np.array([a, b, c])])
    return out[:n]


def torus_count(R: float) -> int:
    r = R / 4.0
    return int(POINTS_PER_SQ_WAVELENGTH * 4 * math.pi ** 2 * R * r)


def torus(R: float, seed: int, n: int | None = None) -> np.ndarray:
    """Area-uniform points on the torus with major radius R, minor R/4: theta
    is kept with probability (R + r cos theta) / (R + r), phi uniform."""
    r = R / 4.0
    rng = np.random.default_rng(seed)
    n = torus_count(R) if n is None else n
    th = np.empty(0)
    while th.shape[0] < n:
        m = max(1024, int(2.0 * (n - th.shape[0])))
        t = rng.random(m) * 2 * math.pi
        keep = rng.random(m) < (R + r * np.cos(t)) / (R + r)
        th = np.concatenate([th, t[keep]])
    th = th[:n]
    ph = rng.random(n) * 2 * math.pi
    rr = R + r * np.cos(th)
    return np.stack([rr * np.cos(ph), rr * np.sin(ph), r * np.sin(th)], axis=1)


def cube_surface(edge: float, seed: int, n: int | None = None) -> np.ndarray:
    """Uniform points on the surface of the axis-aligned cube of the given edge
    centred at the origin (face chosen uniformly, point uniform on the face)."""
    rng = np.random.default_rng(seed)
    n = int(POINTS_PER_SQ_WAVELENGTH * 6 * edge * edge) if n is None else n
    face = rng.integers(0, 6, n)
    uv = (rng.random((n, 2)) - 0.5) * edge
    p = np.empty((n, 3))
    ax = face // 2
    sgn = np.where(face % 2 == 0, 0.5, -0.5) * edge
    for a in range(3):
        sel = ax == a
        others = [d for d in range(3) if d != a]
        p[sel, a] = sgn[sel]
        p[sel, others[0]] = uv[sel, 0]
        p[sel, others[1]] = uv[sel, 1]
    return p


def densities(N: int, nrhs: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """nrhs x N complex densities, real and imaginary parts i.i.d. N(0,1)."""
    rng = np.random.default_rng(seed + 7919)
    f = rng.standard_normal((nrhs, N)) + 1j * rng.standard_normal((nrhs, N))
    return f.astype(dtype)


def clustered(K: float, seed: int, n: int, n_clusters: int = 4, spread: float = 0.05) -> np.ndarray:
    """A sphere of diameter K with extra tight clusters of points, so that the
    low-frequency octree is adaptive (leaves at several levels)."""
    rng = np.random.default_rng(seed)
    base = _unit_sphere(rng, n) * (0.5 * K)
    centres = _unit_sphere(rng, n_clusters) * (0.5 * K * 0.9)
    k = n // 3
    idx = rng.integers(0, n_clusters, k)
    base[:k] = centres[idx] + rng.standard_normal((k, 3)) * spread
    return np.clip(base, -0.5 * K, 0.5 * K)


# The workloads the benchmark and the parity tests use, by name.
WORKLOADS = {
    "sphere_K8": dict(kind="sphere", K=8.0, seed=0),
    "sphere_K64": dict(kind="sphere", K=64.0, seed=1),
    "ellipsoid_64_32_16": dict(kind="ellipsoid", K=128.0, axes=(64.0, 32.0, 16.0), seed=2),
}


def make(name: str) -> tuple[np.ndarray, float]:
    w = WORKLOADS[name]
    if w["kind"] == "sphere":
        return sphere(w["K"], w["seed"]), w["K"]
    if w["kind"] == "ellipsoid":
        return ellipsoid(*w["axes"], seed=w["seed"]), w["K"]
    raise KeyError(name)


def batch_geometries() -> list[tuple[str, np.ndarray, float, int]]:
    """Twelve geometries of uneven size for the batched form, seeds 10-21 in
    this order: spheres K = 8/16/24/32/48; ellipsoids with semi-axes
    (K/2, K/4, K/8) for K = 16/32/64; tori (R, R/4) for R = 8/16/24/32 with
    K = 2.5 R.  Right-hand sides are assigned round-robin from (1, 4, 16, 32).
    Returns (name, points, K, nrhs) tuples."""
    out = []
    seed = 10
    for K in (8.0, 16.0, 24.0, 32.0, 48.0):
        out.append((f"sphere_K{K:g}", sphere(K, seed), K))
        seed += 1
    for K in (16.0, 32.0, 64.0):
        out.append((f"ellipsoid_K{K:g}", ellipsoid(K / 2, K / 4, K / 8, seed), K))
        seed += 1
    for R in (8.0, 16.0, 24.0, 32.0):
        out.append((f"torus_R{R:g}", torus(R, seed), 2.5 * R))
        seed += 1
    rhs = (1, 4, 16, 32)
    return [(name, p, K, rhs[k % 4]) for k, (name, p, K) in enumerate(out)]


def served_geometries(scale: float = 1.0) -> list[tuple[str, np.ndarray, float]]:
    """The eight resident plans of the served form (seeds 40-47): spheres
    K = 16/32/64, ellipsoids (K/2, K/4, K/8) for K = 32/128, tori (R, R/4) for
    R = 16/32 (K = 2.5 R) and a cube surface of edge 48.  `scale` < 1 shrinks
    every size in wavelengths (for quick tests)."""
    out = []
    seed = 40
    for K in (16.0, 32.0, 64.0):
        out.append((f"sphere_K{K * scale:g}", sphere(K * scale, seed), K * scale))
        seed += 1
    for K in (32.0, 128.0):
        k = K * scale
        out.append((f"ellipsoid_K{k:g}", ellipsoid(k / 2, k / 4, k / 8, seed), k))
        seed += 1
    for R in (16.0, 32.0):
        r = R * scale
        out.append((f"torus_R{r:g}", torus(r, seed), 2.5 * r))
        seed += 1
    e = 48.0 * scale
    out.append((f"cube_E{e:g}", cube_surface(e, seed), e))
    return out


def poisson_arrivals(n: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))
