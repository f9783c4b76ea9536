"""Failure paths of the request server, all made on the host (no device fault,
no hang): a handle that is not a live plan, destroying a plan that queued
requests hold, a cancelled request, a wait that times out, and a group whose
queueing fails on the host (dfmm_server_fail_next) while the plan stays
resident and the server keeps serving."""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import direct as OD

pytestmark = pytest.mark.gpu

ERR_INVALID, ERR_CUDA, ERR_TIMEOUT, ERR_CANCELLED = -1, -4, -6, -8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def plan():
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(4.0, 2)
    return Plan(p, 4.0, 1e-5)


def _buffers(plan, n, seed):
    fs = [workloads.densities(plan.N, 1, seed + k).astype(np.complex64) for k in range(n)]
    us = [np.full((1, plan.N), np.nan, np.complex64) for _ in range(n)]
    return fs, us


def _submit(srv, plan_h, f, u):
    from paper_1311_4257_gb300 import lib
    t = ctypes.c_int64(0)
    rc = lib().dfmm_server_submit(srv._h, plan_h, f.ctypes.data, u.ctypes.data, 1, ctypes.byref(t))
    return rc, t.value


def test_handles_that_are_not_live_plans_are_refused(plan):
    from paper_1311_4257_gb300 import Plan, Server
    srv = Server(streams=1, budget_bytes=1 << 30, max_rhs=1)
    f, u = _buffers(plan, 1, 0)
    rc, _ = _submit(srv, ctypes.c_void_p(f[0].ctypes.data), f[0], u[0])   # an address that is no plan
    assert rc == ERR_INVALID
    g = Plan(workloads.sphere(4.0, 3, n=2000), 4.0, 1e-4)
    h = g._h
    g.close()
    rc, _ = _submit(srv, h, f[0], u[0])                                   # a destroyed plan
    assert rc == ERR_INVALID
    assert np.isnan(u[0]).all()
    srv.close()


def test_destroy_refused_while_requests_hold_the_plan():
    from paper_1311_4257_gb300 import DfmmError, Plan, Server
    g = Plan(workloads.sphere(4.0, 4), 4.0, 1e-5)
    srv = Server(streams=1, budget_bytes=1 << 30, max_rhs=1)
    f, u = _buffers(g, 200, 10)
    tickets = [srv.submit(g, f[k].ctypes.data, u[k].ctypes.data, 1) for k in range(200)]
    with pytest.raises(DfmmError) as e:
        g.close()                      # 200 requests queued or running on it
    assert e.value.code == ERR_INVALID
    for t in tickets:
        srv.wait(t)
    g.close()                          # released by every finished request
    srv.close()


def test_cancel_a_queued_request(plan):
    import torch
    from paper_1311_4257_gb300 import DfmmError, Server
    srv = Server(streams=1, budget_bytes=1 << 30, max_rhs=1)
    n = 100
    f, u = _buffers(plan, n, 20)
    tickets = [srv.submit(plan, f[k].ctypes.data, u[k].ctypes.data, 1) for k in range(n)]
    srv.cancel(tickets[-1])            # 99 single-RHS applies ahead of it on one stream
    for t in tickets[:-1]:
        srv.wait(t)
    with pytest.raises(DfmmError) as e:
        srv.wait(tickets[-1])
    assert e.value.code == ERR_CANCELLED
    assert np.isnan(u[-1]).all()       # never written
    with pytest.raises(DfmmError) as e:
        srv.cancel(tickets[0])         # finished and collected
    assert e.value.code == ERR_INVALID
    ref = plan.apply(torch.as_tensor(f[0], device="cuda")).cpu().numpy()
    assert OD.rel_err(u[0].astype(np.complex128), ref.astype(np.complex128)) < 1e-6
    assert srv.stats()["requests_failed"] == 1
    srv.close()


def test_wait_times_out_and_the_ticket_stays_valid(plan):
    from paper_1311_4257_gb300 import DfmmError, Server
    srv = Server(streams=1, budget_bytes=1 << 30, max_rhs=1)
    f, u = _buffers(plan, 50, 30)
    tickets = [srv.submit(plan, f[k].ctypes.data, u[k].ctypes.data, 1) for k in range(50)]
    with pytest.raises(DfmmError) as e:
        srv.wait(tickets[-1], timeout=0.0)
    assert e.value.code == ERR_TIMEOUT
    for t in tickets:
        srv.wait(t)
    assert not np.isnan(u[-1]).any()
    srv.close()


def test_injected_failure_fails_one_group_and_serving_goes_on(plan):
    import torch
    from paper_1311_4257_gb300 import DfmmError, Server
    srv = Server(streams=2, budget_bytes=1 << 30, max_rhs=4)
    f, u = _buffers(plan, 3, 40)
    srv.fail_next(ERR_CUDA)
    t0 = srv.submit(plan, f[0].ctypes.data, u[0].ctypes.data, 1)
    with pytest.raises(DfmmError) as e:
        srv.wait(t0)
    assert e.value.code == ERR_CUDA
    assert np.isnan(u[0]).all()        # nothing was queued for the failed group
    t1 = srv.submit(plan, f[1].ctypes.data, u[1].ctypes.data, 1)
    t2 = srv.submit(plan, f[2].ctypes.data, u[2].ctypes.data, 1)
    srv.wait(t1)
    srv.wait(t2)
    for k in (1, 2):
        ref = plan.apply(torch.as_tensor(f[k], device="cuda")).cpu().numpy()
        assert OD.rel_err(u[k].astype(np.complex128), ref.astype(np.complex128)) < 1e-6
    st = srv.stats()
    assert st["requests_failed"] == 1 and st["requests_done"] == 2
    srv.close()
