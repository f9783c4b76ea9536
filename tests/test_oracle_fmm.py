"""Pins of the oracle's representations (Eq. 2) and FMM (Alg. 1) to the direct
sum, to linearity, to Table 1's separation ranks, and to the symmetry the
precomputation relies on."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from oracle import fmm as F
from oracle import skeleton as S
from oracle.direct import direct, rel_err
from oracle.kernel import G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ls_error(rep, X, Y):
    """Relative error (weighted by |x|) of the outgoing representation applied
    to fresh sources Y and evaluated at fresh targets X."""
    wt = np.linalg.norm(X, axis=1)[:, None]
    exact = G(X, Y)
    approx = rep.phi(X) @ (rep.p_out() @ G(rep.a2, Y))
    return np.linalg.norm(wt * (exact - approx)) / np.linalg.norm(wt * exact)


def _ls_error_in(rep, X, Y):
    """Incoming representation: far sources X, targets in the box Y."""
    exact = G(Y, X)
    approx = rep.psi(Y) @ (rep.p_in() @ G(rep.b2, X))
    wt = np.linalg.norm(X, axis=1)[None, :]
    return np.linalg.norm(wt * (exact - approx)) / np.linalg.norm(wt * exact)


@pytest.mark.parametrize("kind", ["hf", "lf"])
def test_representation_accuracy_on_fresh_samples(kind):
    prm = S.SkelParams(eps_op=1e-5)
    st = S.Stream(2024)
    if kind == "hf":
        rep = S.hf_rep(2.0, 0, 4.0, prm)
        X = S.region_hf(st, 2.0, 0, 4.0, 600)
        Y = S.box_samples(st, 2.0, 300)
    else:
        rep = S.lf_rep(0.5, 2.0, prm)
        X = S.region_lf(st, 0.5, 2.0, 600)
        Y = S.box_samples(st, 0.5, 300)
    assert _ls_error(rep, X, Y) < 20 * prm.eps_op
    assert _ls_error_in(rep, X, Y) < 20 * prm.eps_op
    # orthonormal bases on the check points, R with real positive diagonal
    assert np.allclose(rep.Qo.conj().T @ rep.Qo, np.eye(rep.r), atol=1e-10)
    assert np.allclose(rep.Qi.conj().T @ rep.Qi, np.eye(rep.r), atol=1e-10)
    Ro = np.linalg.inv(rep.Ro_inv)
    assert np.all(np.abs(np.diag(Ro).imag) < 1e-9 * np.abs(np.diag(Ro)))
    assert np.all(np.diag(Ro).real > 0)


def test_symmetry_mapped_representation_is_accurate():
    # rotational invariance (Sec. 2.2): a representation mapped by a cube
    # symmetry is as accurate on the mapped cell's own region
    prm = S.SkelParams(eps_op=1e-5)
    rs = S.RepSet(prm, w_top=4.0)
    canon, which = rs.canon(2.0)
    cell = 17
    assert canon[cell] != cell
    rep = rs.hf(2.0, cell)
    st = S.Stream(77)
    X = S.region_hf(st, 2.0, cell, 4.0, 500)
    Y = S.box_samples(st, 2.0, 200)
    assert _ls_error(rep, X, Y) < 20 * prm.eps_op


def test_separation_ranks_near_table1():
    gold = json.load(open(os.path.join(GOLD, "table1_separation_rank.json")))
    for eps_key in ("1e-4", "1e-6"):
        eps = float(eps_key)
        for k, w in enumerate((1.0, 2.0)):
            r = S.hf_rep(w, 0, 4.0, S.SkelParams(eps_op=eps)).r
            ref = gold["rank"][eps_key][k]
            assert 0.5 * ref <= r <= 2.0 * ref, (eps, w, r, ref)


def test_single_precision_translations_stay_within_tolerance():
    # the least-squares form keeps single-precision translations stable: the
    # FMM with complex64 operators and states stays within the tolerance
    p = workloads.sphere(4.0, 5)
    f = workloads.densities(p.shape[0], 1, 5)
    plan = F.Plan(p, 4.0, F.FMMParams(eps=1e-4))
    t = np.arange(0, p.shape[0], 7)
    ref = direct(p, f, t)
    e64 = rel_err(F.fmm(plan, f)[:, t], ref)
    e32 = rel_err(F.fmm(plan, f, fp32=True)[:, t], ref)
    assert e64 < 1e-4 and e32 < 1e-4 and e32 < 3 * e64 + 1e-6


def test_error_falls_with_eps():
    p = workloads.sphere(4.0, 6)
    f = workloads.densities(p.shape[0], 1, 6)
    t = np.arange(0, p.shape[0], 5)
    ref = direct(p, f, t)
    errs = []
    for eps in (1e-3, 1e-4, 1e-5):
        plan = F.Plan(p, 4.0, F.FMMParams(eps=eps))
        errs.append(rel_err(F.fmm(plan, f)[:, t], ref))
        assert errs[-1] <= eps
    assert errs[0] > errs[1] > errs[2]


def test_linearity_over_rhs():
    p = workloads.sphere(4.0, 7, n=3000)
    plan = F.Plan(p, 4.0, F.FMMParams(eps=1e-4))
    f = workloads.densities(p.shape[0], 2, 7)
    u = F.fmm(plan, f)
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    v = F.fmm(plan, (a * f[0] + b * f[1])[None])[0]
    assert np.linalg.norm(v - (a * u[0] + b * u[1])) < 1e-12 * np.linalg.norm(v)


def test_adaptive_tree_with_w_and_x_lists():
    p = workloads.clustered(8.0, 3, 6000, n_clusters=3, spread=0.08)
    plan = F.Plan(p, 8.0, F.FMMParams(eps=1e-5, leaf_max=16))
    assert plan.lf.W.shape[0] > 0 and plan.lf.X.shape[0] > 0
    f = workloads.densities(p.shape[0], 1, 8)
    t = np.arange(0, p.shape[0], 11)
    assert rel_err(F.fmm(plan, f)[:, t], direct(p, f, t)) <= 1e-5


@pytest.mark.slow
def test_sphere_k8_against_direct_sum():
    """Sphere of diameter 8, N = 20,106 (seed 0): FMM within eps of Eq. 1."""
    p = workloads.sphere(8.0, 0)
    assert p.shape[0] == 20106
    f = workloads.densities(p.shape[0], 1, 0)
    plan = F.Plan(p, 8.0, F.FMMParams(eps=1e-5))
    t = np.random.default_rng(1000).choice(p.shape[0], 1000, replace=False)
    e = rel_err(F.fmm(plan, f)[:, t], direct(p, f, t))
    assert e <= 1e-5
