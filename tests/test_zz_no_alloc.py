"""dfmm_apply_noalloc, the allocation-free matvec, called through the C ABI.

Callers that may not let a library allocate device memory (graph capture,
allocation-free request paths, fixed memory budgets) use this entry point; it
must give the same potentials as dfmm_apply, call after call, although every
call reuses the one static scratch array left over from the previous call.
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
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(u)).all()
        assert _rel(u, u_ref) < 1e-6


def test_noalloc_rejects_applies_beyond_its_capacity(env):
    torch, dfmm, L = env
    assert L.dfmm_noalloc_capacity() == 64 << 20
    p = workloads.sphere(8.0, 0)
    plan = dfmm.Plan(p, 8.0, 1e-5)
    f = torch.zeros((64, p.shape[0]), dtype=torch.complex64, device="cuda")
    u = torch.empty_like(f)
    rc = L.dfmm_apply_noalloc(plan._h, f.data_ptr(), u.data_ptr(), 64, torch.cuda.current_stream().cuda_stream)
    assert rc == dfmm.ERR_UNSUPPORTED
    assert b"scratch" in L.dfmm_last_error()
