"""The skeleton pivot selection on the GPU (skeleton_gpu.cu) against the host form.

Both forms draw the same samples and the same +-1 sketch and apply the same
pivot rule (largest remaining column norm, recomputed every step, first index
among equal norms) to the QR of the sketch and to the two QRs that pick the far
check points.  Only the FP64 rounding differs, so on inputs without near-tied
pivots the selected index sets, hence the skeleton points, must be identical;
the host form is itself pinned to the oracle's skeletons (tests/test_abi.py).
"""
import numpy as np
import pytest

import workloads
from oracle import direct as OD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_4257_gb300 import build
    build.build()


TYPES = [(0.25, -1, 8.0), (0.5, -1, 8.0), (0.5, -1, 64.0), (1.0, 0, 8.0), (1.0, 3, 8.0), (2.0, 0, 8.0),
         (2.0, 7, 8.0), (4.0, 0, 64.0), (4.0, 21, 64.0), (8.0, 5, 64.0)]


@pytest.mark.parametrize("eps_op", [3e-5, 3e-6])
def test_device_selection_equals_host(eps_op):
    """eps 1e-4 and 1e-5 (eps_op = 0.3 eps): the same skeleton points as the host."""
    from paper_1311_4257_gb300.dfmm import representation
    for w, cell, w_top in TYPES:
        rh, bh, ah = representation(w, cell, w_top, eps_op)
        rd, bd, ad = representation(w, cell, w_top, eps_op, device=True)
        assert rd == rh, (w, cell, w_top, rd, rh)
        assert np.array_equal(bd, bh), (w, cell, w_top)
        assert np.array_equal(ad, ah), (w, cell, w_top)


def _fresh(w, cell, w_top, n_far=800, n_box=300):
    from oracle import skeleton as S
    st = S.Stream(4242)
    X = S.region_lf(st, w, w_top, n_far) if cell < 0 else S.region_hf(st, w, cell, w_top, n_far)
    return X, S.box_samples(st, w, n_box)


def _ls_error(b2, a2, r, X, Y):
    """Error of the least-squares form of Eq. 2 on fresh samples: the field of
    box sources Y at far points X from the state fitted at the 2r weighted
    check points a2, with the r equivalent points b = b2[:r]."""
    from oracle.kernel import G
    b = b2[:r]
    wa = np.linalg.norm(a2, axis=1)[:, None]
    coef = np.linalg.lstsq(wa * G(a2, b), wa * G(a2, Y), rcond=None)[0]
    wt = np.linalg.norm(X, axis=1)[:, None]
    exact = G(X, Y)
    return np.linalg.norm(wt * (exact - G(X, b) @ coef)) / np.linalg.norm(wt * exact)


@pytest.mark.parametrize("eps_op,sketch", [(3e-7, 0), (1e-9, 800)])
def test_device_selection_tight_tolerances(eps_op, sketch):
    """eps 1e-6 and the FP64 form's 1e-8: the later pivots are picked among column
    norms that agree to the rounding of the previous steps, so the device and
    host choices may part there (reading A15: both are valid skeletons).  Both
    must have the same rank and represent the kernel on fresh samples within
    20 eps_op (or, where FP64 itself limits the check, as well as the host's)."""
    from paper_1311_4257_gb300.dfmm import representation
    types = TYPES if sketch == 0 else [(1.0, 0, 8.0), (0.5, -1, 8.0), (2.0, 0, 8.0)]
    for w, cell, w_top in types:
        rh, bh, ah = representation(w, cell, w_top, eps_op, sketch_rows=sketch)
        rd, bd, ad = representation(w, cell, w_top, eps_op, sketch_rows=sketch, device=True)
        assert rd == rh, (w, cell, w_top, rd, rh)
        same_b = int(np.argmin(np.all(bd == bh, axis=1))) if not np.array_equal(bd, bh) else 2 * rh
        same_a = int(np.argmin(np.all(ad == ah, axis=1))) if not np.array_equal(ad, ah) else 2 * rh
        X, Y = _fresh(w, cell, w_top)
        eh, ed = _ls_error(bh, ah, rh, X, Y), _ls_error(bd, ad, rd, X, Y)
        print(f"w {w} cell {cell} top {w_top} eps_op {eps_op:g}: r {rh}, equal points b2 {same_b}/{2 * rh}, "
              f"a2 {same_a}/{2 * rh}; error host {eh:.2e} device {ed:.2e}")
        assert ed <= max(20 * eps_op, 2 * eh), (w, cell, ed, eh)


def test_plans_with_either_selection_agree():
    """A K = 16 plan (HF levels w = 2, 4, 8) at eps 1e-5 with the selection on the
    GPU and on the host: same ranks, and the same potentials up to the order of
    the floating-point additions."""
    import torch
    from paper_1311_4257_gb300 import Plan
    p = workloads.sphere(16.0, 1)
    f = torch.as_tensor(workloads.densities(p.shape[0], 1, 5).astype(np.complex64), device="cuda")
    gd = Plan(p, 16.0, 1e-5)   # the default: selection on the GPU
    gh = Plan(p, 16.0, 1e-5, skeleton_host=1)
    sd, sh = gd.stats(), gh.stats()
    assert sd["rank"] == sh["rank"]
    ud, uh = gd.apply(f), gh.apply(f)
    torch.cuda.synchronize()
    assert OD.rel_err(ud.cpu().numpy().astype(np.complex128), uh.cpu().numpy().astype(np.complex128)) < 1e-6
    print(f"K 16 skeleton phase: GPU {sd['plan_phase_seconds'][1]:.2f} s, host {sh['plan_phase_seconds'][1]:.2f} s")
