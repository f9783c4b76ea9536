"""GPU parity of the FP64 form (options.arith 64, automatic below eps 1e-6).

Table 1 of the paper goes down to eps = 1e-8, where complex64 densities and
FP32 arithmetic cannot reach the tolerance (their rounding alone is ~6e-8).
The FP64 form keeps operators, rows, states, densities and potentials in
complex128 and evaluates Eq. 1 in FP64 throughout.

* Sphere of diameter 4 (N = 5,026), eps = 1e-8: within eps of the direct sum
  of Eq. 1 on every target, and equal to the oracle FMM (same 800-row sketch
  and eps_op = 0.1 eps, the library's defaults below eps 1e-7, so the same
  skeletons) up to FP64 summation order.
* Sphere of diameter 8 (N = 20,106), eps = 1e-8: within eps of the direct sum
  on every target.
* The host-buffer, allocation-free and batched entry points take complex128
  for such plans and give the same potentials; dfmm_solve refuses them.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import direct as OD
from oracle import fmm as OF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()


def _apply(plan, f):
    import torch
    fd = torch.as_tensor(np.asarray(f, dtype=np.complex128), device="cuda")
    u = plan.apply(fd)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.fixture(scope="module")
def sphere4():
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(4.0, 0)
    # host pivot selection: its skeletons are the oracle's, so the FMM-vs-FMM
    # comparison below sees only rounding.  At eps_op = 1e-9 the GPU selection
    # may pick other, equally valid, near-tied pivots (reading A15);
    # test_sphere_k8_eps1e8_all_targets runs the default GPU selection.
    g = Plan(p, 4.0, 1e-8, skeleton_host=1)
    return p, g


def test_fp64_form_is_automatic_below_1e6(sphere4):
    import torch
    p, g = sphere4
    st = g.stats()
    assert st["arith"] == 64 and g.dtype == torch.complex128
    assert max(st["rank"]) > 128   # ranks grow with the accuracy level
    with pytest.raises(TypeError):
        g.apply(torch.zeros(p.shape[0], dtype=torch.complex64, device="cuda"))


def test_sphere_k4_eps1e8_against_direct_and_oracle(sphere4):
    p, g = sphere4
    assert p.shape[0] == 5026
    f = workloads.densities(p.shape[0], 2, 0)
    u = _apply(g, f)
    ud = OD.direct(p, f, np.arange(p.shape[0]))
    e_dir = OD.rel_err(u, ud)
    uo = OF.fmm(OF.Plan(p, 4.0, OF.FMMParams(eps=1e-8, sketch=800, eps_op_factor=0.1)), f)
    e_fmm = OD.rel_err(u, uo)
    print(f"eps 1e-8, K 4: vs direct {e_dir:.3e}, vs oracle FMM {e_fmm:.3e}, oracle vs direct "
          f"{OD.rel_err(uo, ud):.3e}")
    assert e_dir <= 1e-8, e_dir
    # same skeletons and operators, FP64 on both sides: only the rounding order
    # differs (the library's FP64 GEMMs vs numpy products, atomics), amplified by the inverse
    # factors R^-1 whose condition reaches 1 / eps_op; measured 1.2e-10
    assert e_fmm <= 1e-9, e_fmm


def test_sphere_k8_eps1e8_all_targets():
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(8.0, 0)
    assert p.shape[0] == 20106
    g = Plan(p, 8.0, 1e-8)
    f = workloads.densities(p.shape[0], 1, 0)
    u = _apply(g, f)
    ud = OD.direct(p, f, np.arange(p.shape[0]))
    e_dir = OD.rel_err(u, ud)
    print(f"eps 1e-8, K 8: vs direct {e_dir:.3e}, ranks {g.stats()['rank']}")
    assert e_dir <= 1e-8, e_dir


def test_fp64_entry_points_agree(sphere4):
    import torch
    from paper_1311_4257_gb300 import DfmmError, apply_batched, lib
    p, g = sphere4
    f = workloads.densities(p.shape[0], 2, 3)
    u = _apply(g, f)
    uh = g.apply_host(f)
    assert uh.dtype == np.complex128
    assert OD.rel_err(uh, u) <= 1e-14
    fd = torch.as_tensor(f, device="cuda")
    ub = apply_batched([g, g], [fd, fd[:1].contiguous()])
    torch.cuda.synchronize()
    assert OD.rel_err(ub[0].cpu().numpy(), u) <= 1e-14
    assert OD.rel_err(ub[1].cpu().numpy(), u[:1]) <= 1e-14
    L = lib()
    L.dfmm_apply_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p]
    L.dfmm_apply_noalloc.restype = ctypes.c_int
    L.dfmm_noalloc_capacity.restype = ctypes.c_int64
    if g.workspace_bytes(2) <= L.dfmm_noalloc_capacity():
        un = torch.empty_like(fd)
        s = torch.cuda.current_stream().cuda_stream
        assert L.dfmm_apply_noalloc(g._h, fd.data_ptr(), un.data_ptr(), 2, s) == 0
        torch.cuda.synchronize()
        assert OD.rel_err(un.cpu().numpy(), u) <= 1e-14
    # the GMRES driver works on complex64 vectors: FP64 plans are refused
    with pytest.raises(DfmmError):
        g.solve(torch.ones(p.shape[0], dtype=torch.complex64, device="cuda"))


def test_fp64_captured_and_merged_batch_forms(sphere4):
    """A captured apply (dfmm_graph_*) and the merged batch (dfmm_batch_*, with a
    second FP64 plan of another geometry) on complex128 buffers equal the plain
    applies; the FP64 stages run per plan inside the batch's waves."""
    import torch
    from paper_1311_4257_gb300 import Batch, Plan
    p, g = sphere4
    f = workloads.densities(p.shape[0], 2, 5)
    u = _apply(g, f)
    fd = torch.as_tensor(f, device="cuda")
    ud = torch.empty_like(fd)
    gr = g.graph(fd, ud)
    gr.launch()
    torch.cuda.synchronize()
    assert OD.rel_err(ud.cpu().numpy(), u) <= 1e-14
    gr.close()
    p2 = workloads.sphere(4.0, 6, n=3000)
    g2 = Plan(p2, 4.0, 1e-8)
    f2 = workloads.densities(p2.shape[0], 1, 6)
    u2 = _apply(g2, f2)
    b = Batch([g, g2], [fd, torch.as_tensor(f2, device="cuda")])
    us = b.launch()
    torch.cuda.synchronize()
    assert OD.rel_err(us[0].cpu().numpy(), u) <= 1e-14
    assert OD.rel_err(us[1].cpu().numpy(), u2) <= 1e-14
    b.close()
