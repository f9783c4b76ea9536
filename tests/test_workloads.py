"""The seeded synthetic inputs (workloads.py): their sizes follow the stated
density of 100 points per square wavelength, every point lies on its surface
and inside the root box, and the area quadrature behind the ellipsoid count
agrees with closed forms."""
import math

import numpy as np

import workloads


def test_sphere_counts_and_radius():
    assert workloads.sphere_count(8.0) == 20106          # 100 pi K^2
    assert workloads.sphere_count(64.0) == 1286796
    p = workloads.sphere(8.0, 0)
    assert p.shape == (20106, 3)
    assert np.allclose(np.linalg.norm(p, axis=1), 4.0, atol=1e-12)
    assert np.abs(p).max() <= 4.0                         # inside the root box |x|_inf <= K/2


def test_ellipsoid_area_against_closed_forms():
    # a sphere: 4 pi a^2
    assert abs(workloads.ellipsoid_area(3.0, 3.0, 3.0) - 4 * math.pi * 9.0) < 1e-6 * 4 * math.pi * 9.0
    # a prolate spheroid (a > b = c): 2 pi b^2 (1 + a / (b e) asin e), e^2 = 1 - b^2 / a^2
    a, b = 4.0, 1.0
    e = math.sqrt(1 - b * b / (a * a))
    exact = 2 * math.pi * b * b * (1 + a / (b * e) * math.asin(e))
    assert abs(workloads.ellipsoid_area(a, b, b) - exact) < 1e-5 * exact


def test_ellipsoid_points_on_the_surface():
    assert workloads.ellipsoid_count(64.0, 32.0, 16.0) == 1625002
    p = workloads.ellipsoid(8.0, 4.0, 2.0, 3)
    assert p.shape[0] == workloads.ellipsoid_count(8.0, 4.0, 2.0)
    q = (p[:, 0] / 8.0) ** 2 + (p[:, 1] / 4.0) ** 2 + (p[:, 2] / 2.0) ** 2
    assert np.allclose(q, 1.0, atol=1e-12)


def test_ellipsoid_sampling_is_area_uniform():
    # the share of points with |z| > c / 2 against the share of the area there
    a, b, c = 6.0, 3.0, 1.5
    p = workloads.ellipsoid(a, b, c, 5, n=200000)
    nq = 800
    t = (np.arange(nq) + 0.5) / nq * 2.0 - 1.0
    ph = (np.arange(2 * nq) + 0.5) / (2 * nq) * 2 * math.pi
    ct, pp = np.meshgrid(t, ph, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    g = np.sqrt((b * c * st * np.cos(pp)) ** 2 + (a * c * st * np.sin(pp)) ** 2 + (a * b * ct) ** 2)
    share = g[np.abs(ct) > 0.5].sum() / g.sum()
    assert abs(np.mean(np.abs(p[:, 2]) > c / 2) - share) < 0.005


def test_torus_points_on_the_surface():
    R = 8.0
    r = R / 4
    assert workloads.torus_count(R) == int(100 * 4 * math.pi ** 2 * R * r)
    p = workloads.torus(R, 4)
    rho = np.hypot(p[:, 0], p[:, 1])
    assert np.allclose((rho - R) ** 2 + p[:, 2] ** 2, r * r, atol=1e-9)
    assert np.abs(p).max() <= 2.5 * R / 2             # K = 2.5 R


def test_cube_surface_points_on_faces():
    p = workloads.cube_surface(4.0, 6)
    assert p.shape[0] == 100 * 6 * 16
    m = np.abs(p).max(axis=1)
    assert np.allclose(m, 2.0)


def test_densities_are_standard_complex_normal():
    f = workloads.densities(200000, 1, 3)
    assert abs(f.real.std() - 1) < 0.01 and abs(f.imag.std() - 1) < 0.01
    assert abs(f.real.mean()) < 0.01 and abs(f.imag.mean()) < 0.01


def test_poisson_arrivals():
    t = workloads.poisson_arrivals(20000, 200.0, 30)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.03 / 200.0
