"""GMRES around the resident matvec (dfmm_solve) against dense FP64 solves.

The system is single-layer-like: (1/2) x + (a / 4 pi) G x = b with a the surface
area per point (1/100 square wavelength at 100 points per square wavelength),
well conditioned.  The dense reference is the oracle's FP64 kernel matrix
(self term excluded, Eq. 1) solved by LU, on inputs small enough for it.
"""
import numpy as np
import pytest

import workloads
from oracle import direct as OD
from oracle import kernel as OK

pytestmark = pytest.mark.gpu

ALPHA = 0.5
BETA = (1.0 / workloads.POINTS_PER_SQ_WAVELENGTH) / (4.0 * np.pi)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()


def _dense(p):
    with np.errstate(divide="ignore", invalid="ignore"):   # the self term, dropped below
        G = OK.G(p, p)
    np.fill_diagonal(G, 0.0)
    return ALPHA * np.eye(p.shape[0]) + BETA * G


@pytest.mark.parametrize("eps", [1e-6, 1e-5])
def test_gmres_matches_dense_solve(eps):
    import torch
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(2.0, 7)
    b = workloads.densities(p.shape[0], 1, 8)[0]
    plan = Plan(p, 2.0, eps)
    x, it, rr = plan.solve(torch.as_tensor(b.astype(np.complex64), device="cuda"), ALPHA, BETA, tol=eps)
    x = x.cpu().numpy().astype(np.complex128)
    assert rr <= 3 * eps and 0 < it < 300
    x_ref = np.linalg.solve(_dense(p), b)
    assert OD.rel_err(x, x_ref) < 10 * eps


def test_gmres_residual_against_direct_sum_k8():
    """Sphere K = 8 (N = 20,106, tensor-core form): the returned x satisfies the
    system to about eps when the residual rows are formed by the direct sum of
    Eq. 1 on sampled targets."""
    import torch
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(8.0, 0)
    b = workloads.densities(p.shape[0], 1, 9)[0]
    plan = Plan(p, 8.0, 1e-5)
    x, it, rr = plan.solve(torch.as_tensor(b.astype(np.complex64), device="cuda"), ALPHA, BETA, tol=1e-5,
                           restart=40)
    assert rr <= 3e-5
    x = x.cpu().numpy().astype(np.complex128)
    t = np.random.default_rng(3).choice(p.shape[0], 400, replace=False)
    Gx = OD.direct(p, x[None, :], t)[0]
    r = b[t] - (ALPHA * x[t] + BETA * Gx)
    assert np.linalg.norm(r) / np.linalg.norm(b[t]) < 5e-5


def test_gmres_zero_rhs_gives_zero():
    import torch
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(2.0, 7)
    plan = Plan(p, 2.0, 1e-5)
    x, it, rr = plan.solve(torch.zeros(p.shape[0], dtype=torch.complex64, device="cuda"), ALPHA, BETA)
    assert it == 0 and torch.count_nonzero(x).item() == 0
