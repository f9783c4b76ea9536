"""Batched and served forms through the C ABI.

* dfmm_apply_batched runs several geometries of uneven size (and uneven
  right-hand-side counts) in one call: each result equals that plan's own
  apply.
* The request server batches requests of a Poisson stream across plans and
  right-hand sides: each result is the same alone and in the mix, requests are
  grouped (fewer applies than requests), the memory budget bounds how many
  groups run at once, and a request that can never fit fails cleanly.
Results of separate applies may differ in the last bits: the scatter-adds of
the translation stages run in a data-dependent order.  The tolerance is 1e-6
relative.
"""
import time

import numpy as np
import pytest

import workloads
from oracle import direct as OD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plans():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()
    from paper_1311_4257_gb300 import Plan
    geo = [(workloads.sphere(4.0, 3), 4.0), (workloads.ellipsoid(4.0, 2.0, 1.0, 4), 8.0),
           (workloads.torus(3.0, 5), 7.5), (workloads.cube_surface(4.0, 6), 4.0)]
    return [(Plan(p, K, 1e-5), p) for p, K in geo]


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_apply_batched_equals_single_applies(plans):
    import torch
    from paper_1311_4257_gb300 import apply_batched
    nrhs = [1, 3, 2, 4]
    fs = [torch.as_tensor(workloads.densities(p.N, r, 50 + k).astype(np.complex64), device="cuda")
          for k, ((p, _), r) in enumerate(zip(plans, nrhs))]
    us = apply_batched([p for p, _ in plans], fs)
    torch.cuda.synchronize()
    for (p, pts), f, u in zip(plans, fs, us):
        ref = p.apply(f)
        torch.cuda.synchronize()
        assert _rel(u.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    # and the batch is accurate: torus against the direct sum of Eq. 1
    p, pts = plans[2]
    t = np.arange(0, p.N, 11)
    ud = OD.direct(pts, fs[2].cpu().numpy().astype(np.complex128), t)
    assert _rel(us[2].cpu().numpy()[:, t], ud) < 1e-5


def test_merged_batch_equals_single_applies(plans):
    """The batched form with one merged launch per translation stage across the
    plans (dfmm_batch_*), autotuned and captured as a graph: each geometry's
    result equals its single apply, after set-up and on replays with new
    densities; fewer launches than the plans' applies together."""
    import torch
    from paper_1311_4257_gb300 import Batch
    nrhs = [1, 4, 2, 3]
    fs = [torch.as_tensor(workloads.densities(p.N, r, 70 + k).astype(np.complex64), device="cuda")
          for k, ((p, _), r) in enumerate(zip(plans, nrhs))]
    b = Batch([p for p, _ in plans], fs, graph=True, tune=True)
    torch.cuda.synchronize()
    st = b.stats()
    assert st["graph"] == 1 and st["merged_launches"] > 0 and st["merged_stages"] > st["merged_launches"]
    assert sum(st["order_chosen"]) == st["merged_launches"]
    assert st["launches"] < sum(p.launches(r) for (p, _), r in zip(plans, nrhs))
    for rnd in range(3):
        if rnd:
            for k, f in enumerate(fs):   # new densities in the same buffers, then one replay
                f.copy_(torch.as_tensor(workloads.densities(f.shape[1], f.shape[0], 80 + 10 * rnd + k)
                                        .astype(np.complex64), device="cuda"))
            b.launch()
            torch.cuda.synchronize()
        for (p, _), f, u in zip(plans, fs, b.us):
            ref = p.apply(f)
            torch.cuda.synchronize()
            assert _rel(u.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    b.close()


def test_apply_batched_rejects_bad_arguments(plans):
    import torch
    from paper_1311_4257_gb300 import DfmmError, apply_batched
    p, _ = plans[0]
    f = torch.zeros((1, p.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(DfmmError) as e:
        apply_batched([p], [f], [f])   # f and u alias
    assert e.value.code == -1


def _pinned(a):
    import torch
    return torch.as_tensor(a).pin_memory()


def test_server_results_same_alone_and_in_mix(plans):
    import torch
    from paper_1311_4257_gb300 import Server
    rng = np.random.default_rng(30)
    n = 48
    which = rng.integers(0, len(plans), n)
    nrhs = rng.integers(1, 7, n)
    arrive = workloads.poisson_arrivals(n, 2000.0, 31)
    fs = [_pinned(workloads.densities(plans[w][0].N, int(r), 100 + k).astype(np.complex64))
          for k, (w, r) in enumerate(zip(which, nrhs))]
    us = [_pinned(np.zeros_like(f.numpy())) for f in fs]
    srv = Server(streams=3, budget_bytes=4 << 30, max_rhs=16)
    t0 = time.perf_counter()
    tickets = []
    for k in range(n):
        dt = arrive[k] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(plans[which[k]][0], fs[k].data_ptr(), us[k].data_ptr(), int(nrhs[k])))
    lat = [srv.wait(t, timeout=120.0) for t in tickets]
    st = srv.stats()
    srv.close()
    for k in range(n):
        p = plans[which[k]][0]
        ref = p.apply(fs[k].cuda())
        torch.cuda.synchronize()
        assert _rel(us[k].numpy(), ref.cpu().numpy()) < 1e-6, k
    assert st["requests_done"] == n and st["requests_failed"] == 0
    assert st["rhs_done"] == int(nrhs.sum())
    assert st["applies"] < n            # requests on the same plan were grouped
    assert st["max_concurrent_applies"] >= 1
    assert 0 < st["latency_p50_ms"] <= st["latency_p99_ms"]
    assert min(lat) > 0


def test_server_memory_budget_bounds_concurrency(plans):
    from paper_1311_4257_gb300 import DfmmError, Server
    p, _ = plans[1]
    need = 2 * p.N * 4 * 8 + p.workspace_bytes(4) + 4096
    srv = Server(streams=4, budget_bytes=int(1.5 * need), max_rhs=4)
    fs = [_pinned(workloads.densities(p.N, 4, 200 + k).astype(np.complex64)) for k in range(6)]
    us = [_pinned(np.zeros_like(f.numpy())) for f in fs]
    tickets = [srv.submit(p, f.data_ptr(), u.data_ptr(), 4) for f, u in zip(fs, us)]
    for t in tickets:
        srv.wait(t, timeout=120.0)
    st = srv.stats()
    srv.close()
    assert st["requests_done"] == 6 and st["max_concurrent_applies"] == 1
    ref = p.apply(fs[5].cuda()).cpu().numpy()
    assert _rel(us[5].numpy(), ref) < 1e-6
    # a request that can never fit the budget fails alone
    tiny = Server(streams=1, budget_bytes=1 << 20, max_rhs=4)
    t = tiny.submit(p, fs[0].data_ptr(), us[0].data_ptr(), 4)
    with pytest.raises(DfmmError) as e:
        tiny.wait(t, timeout=60.0)
    assert e.value.code == -3
    tiny.close()


def test_graph_replay_equals_apply(plans):
    """dfmm_graph_*: the captured apply recomputes u from the current f."""
    import torch
    p, _ = plans[2]
    f = torch.as_tensor(workloads.densities(p.N, 2, 300).astype(np.complex64), device="cuda")
    u = torch.empty_like(f)
    g = p.graph(f, u)
    for seed in (301, 302):
        f.copy_(torch.as_tensor(workloads.densities(p.N, 2, seed).astype(np.complex64)))
        g.launch()
        ref = p.apply(f)
        torch.cuda.synchronize()
        assert _rel(u.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    g.close()
