"""Pins of the oracle's direct sum (Eq. 1) to closed forms, brute force and
the symmetry of the kernel."""
import math

import numpy as np

from oracle.direct import direct, direct_loop, rel_err


def test_direct_matches_python_loop():
    rng = np.random.default_rng(3)
    p = rng.uniform(-2, 2, (40, 3))
    f = rng.standard_normal((2, 40)) + 1j * rng.standard_normal((2, 40))
    assert rel_err(direct(p, f, chunk=7), direct_loop(p, f)) < 1e-13


def test_single_source_closed_form():
    # one source at distance d: u_0 = exp(2 pi i d) / d * f_1 (wavelength 1)
    for d in (0.1, 0.75, 3.3, 41.25):
        p = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
        f = np.array([[0.0, 2.0 - 1.0j]])
        u = direct(p, f)
        want = complex(math.cos(2 * math.pi * d), math.sin(2 * math.pi * d)) / d * (2.0 - 1.0j)
        assert abs(u[0, 0] - want) < 1e-14 * abs(want)
        assert u[0, 1] == 0.0


def test_reciprocity_without_conjugation():
    # G(x, y) = G(y, x): g^T (G f) = f^T (G g)
    rng = np.random.default_rng(4)
    p = rng.uniform(-3, 3, (300, 3))
    f = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    g = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    a = g @ direct(p, f[None])[0]
    b = f @ direct(p, g[None])[0]
    assert abs(a - b) < 1e-12 * abs(a)


def test_duplicate_points_are_skipped():
    p = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    f = np.array([[1.0, 10.0, 1.0]], dtype=complex)
    u = direct(p, f)
    g = complex(math.cos(3 * math.pi), math.sin(3 * math.pi)) / 1.5
    assert abs(u[0, 0] - g) < 1e-15 and abs(u[0, 1] - g) < 1e-15
    assert abs(u[0, 2] - 11 * g) < 1e-14


def test_targets_subset_equals_full():
    rng = np.random.default_rng(5)
    p = rng.uniform(-2, 2, (500, 3))
    f = rng.standard_normal((1, 500)) + 0j
    t = np.array([0, 17, 499, 250])
    assert np.allclose(direct(p, f, t), direct(p, f)[:, t], rtol=1e-14, atol=0)


def test_process_pool_equals_single_process():
    """The CPU baseline splits the targets over spawned processes: the same sums,
    up to the summation order of the BLAS product (other chunk shapes, one thread)."""
    from oracle.direct import DirectPool
    rng = np.random.default_rng(7)
    p = rng.standard_normal((400, 3))
    f = rng.standard_normal((2, 400)) + 1j * rng.standard_normal((2, 400))
    t = rng.choice(400, 37, replace=False)
    pool = DirectPool(p, f, 3)
    try:
        got = pool.run(t)
    finally:
        pool.close()
    assert got.shape == (2, 37)
    assert rel_err(got, direct(p, f, t, chunk=8)) < 1e-13
