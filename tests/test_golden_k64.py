"""The stored oracle values of the benchmarked workload (sphere diameter 64,
N = 1,286,796): tests/golden/sphere_k64_oracle.txt, written by
tests/golden/make_sphere_k64_oracle.py from the oracle alone.  They are pinned
here to Eq. 1: the oracle FMM's values lie within eps of the direct sum at the
stored targets, and the stored direct sums equal a fresh evaluation."""
import os

import numpy as np

import workloads
from oracle import direct as OD

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere_k64_oracle.txt")


def _load():
    a = np.loadtxt(GOLDEN)
    return a[:, 0].astype(np.int64), a[:, 1] + 1j * a[:, 2], a[:, 3] + 1j * a[:, 4]


def test_stored_targets_are_the_documented_draw():
    t, _, _ = _load()
    N = workloads.sphere_count(64.0)
    assert N == 1286796
    assert np.array_equal(t, np.sort(np.random.default_rng(6464).choice(N, 1000, replace=False)))


def test_oracle_fmm_within_eps_of_direct_sum():
    """Eq. 1 at eps = 1e-5: the error bound the FMM is built to (Sec. 2.1)."""
    _, u_fmm, u_dir = _load()
    e = OD.rel_err(u_fmm, u_dir)
    assert 1e-8 < e <= 1e-5, e     # an approximation, not a copy of the direct sum


def test_stored_direct_sums_match_a_fresh_evaluation():
    t, _, u_dir = _load()
    p = workloads.sphere(64.0, 1)
    f = workloads.densities(p.shape[0], 1, 64)
    k = np.arange(0, t.size, 125)          # 8 of the 1000 targets
    fresh = OD.direct(p, f, t[k], chunk=8)[0]
    assert np.allclose(fresh, u_dir[k], rtol=1e-12, atol=0.0)
