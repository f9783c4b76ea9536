"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/dfmm.h declares, and its host-side representation builder selects
exactly the oracle's skeleton points (same reading of Sec. 2.1, written
independently)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dfmm.h")).read()
    decl = r"^\s*(?:int|int64_t|const char\s*\*)\s*\**\s*(dfmm_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    from paper_1311_4257_gb300 import build
    build.build()
    from paper_1311_4257_gb300 import dfmm
    return dfmm.lib()


def test_library_exports_every_declared_symbol(L):
    names = _declared()
    assert "dfmm_plan" in names and "dfmm_apply" in names
    for n in names:
        assert hasattr(L, n), n


def test_invalid_arguments_are_rejected_without_a_device(L):
    import ctypes
    from paper_1311_4257_gb300 import dfmm
    h = ctypes.c_void_p()
    pts = np.zeros((4, 3))
    assert L.dfmm_plan(pts.ctypes.data, 0, 8.0, 1e-5, None, ctypes.byref(h)) == dfmm.ERR_INVALID
    assert L.dfmm_plan(pts.ctypes.data, 4, 8.0, 1.0, None, ctypes.byref(h)) == dfmm.ERR_UNSUPPORTED
    assert L.dfmm_plan(pts.ctypes.data, 4, -1.0, 1e-5, None, ctypes.byref(h)) == dfmm.ERR_UNSUPPORTED
    # options are checked before any device call
    o = dfmm.Options(0, 0, 0, 0, 0.0, 3, 0, None, 0)
    assert L.dfmm_plan(pts.ctypes.data, 4, 8.0, 1e-5, ctypes.byref(o), ctypes.byref(h)) == dfmm.ERR_INVALID
    o = dfmm.Options(0, 0, 0, 0, 0.0, 2, 0, None, 32)
    assert L.dfmm_plan(pts.ctypes.data, 4, 8.0, 1e-5, ctypes.byref(o), ctypes.byref(h)) == dfmm.ERR_INVALID
    assert b"tc_stages" in L.dfmm_last_error()
    assert L.dfmm_apply(None, None, None, 1, None) == dfmm.ERR_INVALID
    assert b"null" in L.dfmm_last_error()
    # batched apply: an empty batch is a no-op; missing arrays are rejected
    assert L.dfmm_apply_batched(None, None, None, None, 0, None) == dfmm.OK
    assert L.dfmm_apply_batched(None, None, None, None, 2, None) == dfmm.ERR_INVALID
    assert L.dfmm_apply_batched(None, None, None, None, -1, None) == dfmm.ERR_INVALID
    assert L.dfmm_plan_bytes(None) == -1
    assert L.dfmm_apply_workspace_bytes(None, 1) == -1
    # request server: argument checks come before any device call
    assert L.dfmm_server_create(0, 1 << 20, 16, ctypes.byref(h)) == dfmm.ERR_INVALID
    assert L.dfmm_server_create(4, 0, 16, ctypes.byref(h)) == dfmm.ERR_INVALID
    assert L.dfmm_server_create(4, 1 << 20, 0, ctypes.byref(h)) == dfmm.ERR_INVALID
    t = ctypes.c_int64(0)
    assert L.dfmm_server_submit(None, None, None, None, 1, ctypes.byref(t)) == dfmm.ERR_INVALID
    assert L.dfmm_server_wait(None, 1, 0.0, None) == dfmm.ERR_INVALID
    assert L.dfmm_server_stats(None, None) == dfmm.ERR_INVALID
    assert L.dfmm_server_destroy(None) == dfmm.OK
    assert L.dfmm_graph_create(None, None, None, 1, None, ctypes.byref(h)) == dfmm.ERR_INVALID
    assert L.dfmm_graph_launch(None, None) == dfmm.ERR_INVALID
    assert L.dfmm_graph_destroy(None) == dfmm.OK
    # GMRES: argument checks come before any device call
    it, rr = ctypes.c_int(0), ctypes.c_double(0)
    assert L.dfmm_solve(None, 1.0, 0.0, 1.0, 0.0, None, None, 30, 100, 1e-5, None,
                        ctypes.byref(it), ctypes.byref(rr)) == dfmm.ERR_INVALID


@pytest.mark.parametrize("w,cell", [(1.0, 0), (0.5, -1)])
def test_host_skeleton_matches_oracle_exactly(L, w, cell):
    from paper_1311_4257_gb300 import dfmm
    from oracle import skeleton as S
    prm = S.SkelParams(eps_op=3e-6)
    ref = S.lf_rep(w, 2.0, prm) if cell < 0 else S.hf_rep(w, cell, 2.0, prm)
    r, b2, a2 = dfmm.representation(w, cell, 2.0, 3e-6)
    assert r == ref.r
    assert np.array_equal(b2, ref.b2) and np.array_equal(a2, ref.a2)
