"""dfmm_apply_noalloc, the allocation-free matvec, called through the C ABI.

Some callers may not let a library allocate device memory: services whose
request path forbids allocation after start-up (the allocator is someone
else's, or its latency and failures are not allowed there) and hosts whose
device memory is budgeted in advance.  This entry point must give the same
potentials as dfmm_apply, call after call, although every call reuses the one
static scratch array left over from the previous call; it must not change
the device's free memory; it must accept exactly the applies whose workspace
fits its array; and its device status must reach dfmm_sync_status.
This file is collected last so that a failure here does not hide the others.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()
    from paper_1311_4257_gb300 import dfmm
    L = dfmm.lib()
    L.dfmm_apply_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]
    L.dfmm_apply_noalloc.restype = ctypes.c_int
    L.dfmm_noalloc_capacity.restype = ctypes.c_int64
    return torch, dfmm, L


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_apply_on_two_calls_in_a_row(env):
    torch, dfmm, L = env
    p = workloads.sphere(4.0, 21)
    plan = dfmm.Plan(p, 4.0, 1e-5)
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (1, 2):
        f = torch.as_tensor(workloads.densities(p.shape[0], 2, seed).astype(np.complex64), device="cuda")
        u_ref = plan.apply(f)
        u = torch.full_like(f, complex(np.nan, np.nan))
        rc = L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), 2, stream)
        assert rc == 0, L.dfmm_last_error()
        assert plan.sync_status() == dfmm.OK       # the status word of the allocation-free apply
        assert torch.isfinite(torch.view_as_real(u)).all()
        assert _rel(u, u_ref) < 1e-6


def test_noalloc_leaves_free_device_memory_unchanged(env):
    torch, dfmm, L = env
    p = workloads.sphere(4.0, 22)
    plan = dfmm.Plan(p, 4.0, 1e-5)
    f = torch.as_tensor(workloads.densities(p.shape[0], 1, 3).astype(np.complex64), device="cuda")
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream().cuda_stream
    assert L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), 1, stream) == 0   # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), 1, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_accepts_exactly_the_applies_that_fit(env):
    """The K = 8 sphere (N = 20,106): an apply is accepted exactly when its
    workspace (dfmm_apply_workspace_bytes) fits the array; larger ones are
    rejected with DFMM_ERR_UNSUPPORTED and a message naming the scratch."""
    torch, dfmm, L = env
    cap = L.dfmm_noalloc_capacity()
    assert cap == 64 << 20
    p = workloads.sphere(8.0, 0)
    plan = dfmm.Plan(p, 8.0, 1e-5)
    stream = torch.cuda.current_stream().cuda_stream
    seen = {True: False, False: False}
    for nrhs in (1, 2, 4, 8, 16, 32, 64):
        fits = plan.workspace_bytes(nrhs) <= cap
        f = torch.as_tensor(workloads.densities(p.shape[0], nrhs, 7).astype(np.complex64), device="cuda")
        u = torch.empty_like(f)
        rc = L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), nrhs, stream)
        if fits:
            assert rc == 0, (nrhs, L.dfmm_last_error())
            assert _rel(u, plan.apply(f)) < 1e-6
        else:
            assert rc == dfmm.ERR_UNSUPPORTED, nrhs
            assert b"scratch" in L.dfmm_last_error()
        seen[fits] = True
    assert seen[True] and seen[False]


def test_noalloc_timeout_reaches_sync_status(env):
    """A bounded device wait that gives up inside an allocation-free apply is
    reported by dfmm_sync_status on that stream; the next ordinary
    allocation-free apply clears it."""
    torch, dfmm, L = env
    p = workloads.sphere(4.0, 23)
    f = torch.as_tensor(workloads.densities(p.shape[0], 1, 4).astype(np.complex64), device="cuda")
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream().cuda_stream
    stalled = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2, wait_test=1)
    assert L.dfmm_apply_noalloc(stalled._h, f.data_ptr(), u.data_ptr(), 1, stream) == 0
    assert stalled.sync_status() == dfmm.ERR_TIMEOUT
    plan = dfmm.Plan(p, 4.0, 1e-5, m2l_mode=2)
    assert L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), 1, stream) == 0
    assert plan.sync_status() == dfmm.OK
    assert _rel(u, plan.apply(f)) < 1e-6
