"""Failure detection on the device, without faulting or hanging the GPU.

Every wait of the tensor-core translation kernel is bounded (0.2 s).  The plan
option wait_test makes the first CTA of each tensor-core launch wait on a
barrier that nothing arrives at: the wait gives up, the CTA and the rest of
the apply's tensor-core launches stop early, and the status word that
dfmm_sync_status reads reports DFMM_ERR_TIMEOUT.  The context stays usable:
the next apply of an ordinary plan on the same stream is correct.
"""
import numpy as np
import pytest

import workloads
from oracle import direct as OD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()
    from paper_1311_4257_gb300 import dfmm
    return torch, dfmm


def test_wait_that_runs_out_reports_timeout_and_context_survives(env):
    torch, dfmm = env
    p = workloads.sphere(4.0, 31)
    f = workloads.densities(p.shape[0], 1, 31)
    fd = torch.as_tensor(f.astype(np.complex64), device="cuda")
    stream = torch.cuda.Stream()
    stalled = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2, wait_test=1)
    with torch.cuda.stream(stream):
        stalled.apply(fd)
    assert stalled.sync_status(stream) == dfmm.ERR_TIMEOUT
    assert b"wait" in dfmm.lib().dfmm_last_error()
    # the same stream and device afterwards: an ordinary plan gives correct potentials
    plan = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2)
    with torch.cuda.stream(stream):
        u = plan.apply(fd)
    assert plan.sync_status(stream) == dfmm.OK
    u = u.cpu().numpy().astype(np.complex128)
    assert OD.rel_err(u, OD.direct(p, f)) < 1e-5
    # the stalled plan keeps reporting the timeout on every apply
    with torch.cuda.stream(stream):
        stalled.apply(fd)
    assert stalled.sync_status(stream) == dfmm.ERR_TIMEOUT


def test_wait_that_runs_out_in_the_real_block_form(env):
    """The same failure path in the real-block tensor-core kernel (tc_layout 1)."""
    torch, dfmm = env
    p = workloads.sphere(4.0, 33)
    f = workloads.densities(p.shape[0], 1, 33)
    fd = torch.as_tensor(f.astype(np.complex64), device="cuda")
    stalled = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2, tc_layout=1, wait_test=1)
    stalled.apply(fd)
    assert stalled.sync_status() == dfmm.ERR_TIMEOUT
    plan = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2, tc_layout=1)
    u = plan.apply(fd)
    assert plan.sync_status() == dfmm.OK
    assert OD.rel_err(u.cpu().numpy().astype(np.complex128), OD.direct(p, f)) < 1e-5


def test_status_is_ok_after_ordinary_applies(env):
    torch, dfmm = env
    p = workloads.sphere(4.0, 32)
    fd = torch.as_tensor(workloads.densities(p.shape[0], 2, 32).astype(np.complex64), device="cuda")
    for mode in (1, 2):
        plan = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=mode)
        plan.apply(fd)
        assert plan.sync_status() == dfmm.OK


@pytest.mark.parametrize("eps,kw", [(1e-5, {}), (1e-6, {}), (1e-8, {}), (1e-5, {"tc_layout": 1})])
def test_validate_finds_every_table_in_range(env, eps, kw):
    """dfmm_validate: device-side bounds check of every index table of the plan
    (and of the work tiles of the workspaces laid out by an apply) passes on
    plans of the tensor-core, FP32, FP64 and real-block forms, on an adaptive
    tree with W and X lists."""
    torch, dfmm = env
    p = workloads.clustered(8.0, 3, 6000, n_clusters=3, spread=0.08)
    g = dfmm.Plan(p, 8.0, eps, leaf_max=16, **kw)
    f = torch.as_tensor(workloads.densities(p.shape[0], 2, 3), device="cuda").to(g.dtype)
    g.apply(f)
    torch.cuda.synchronize()
    g.validate()


def test_validate_reports_an_entry_out_of_range(env):
    """The planted check (a scratch copy of one pair table with one source row
    at its bound; the plan is not touched) makes dfmm_validate fail with
    DFMM_ERR_DEVICE and name the table; the plan still validates and applies."""
    torch, dfmm = env
    p = workloads.sphere(4.0, 33)
    g = dfmm.Plan(p, 4.0, 1e-5)
    with pytest.raises(dfmm.DfmmError) as e:
        g.validate(plant=True)
    assert e.value.code == dfmm.ERR_DEVICE
    assert "planted" in str(e.value) and "entry 0" in str(e.value)
    g.validate()
    f = workloads.densities(p.shape[0], 1, 33)
    u = g.apply(torch.as_tensor(f.astype(np.complex64), device="cuda")).cpu().numpy()
    t = np.arange(0, p.shape[0], 50)
    assert OD.rel_err(u[:, t].astype(np.complex128), OD.direct(p, f, t)) <= 1e-5
