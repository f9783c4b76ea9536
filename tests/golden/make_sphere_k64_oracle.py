"""Writes sphere_k64_oracle.txt: the oracle's directional FMM (Alg. 1, FP64) and
the FP64 direct sum of Eq. 1 at 1000 sampled targets of the sphere of diameter
K = 64 (N = 1,286,796 points, seed 1; densities seed 64, one right-hand side;
eps 1e-5).  Test infrastructure: it calls only `oracle/` and the seeded input
generators (`workloads.py`).  About 10 minutes on an 8-core host:

    python tests/golden/make_sphere_k64_oracle.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads                                  # noqa: E402
from oracle import direct as OD                   # noqa: E402
from oracle import fmm as OF                      # noqa: E402

K, SEED, FSEED, EPS, NT, TSEED = 64.0, 1, 64, 1e-5, 1000, 6464
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sphere_k64_oracle.txt")


def main():
    p = workloads.sphere(K, SEED)
    f = workloads.densities(p.shape[0], 1, FSEED)
    t = np.sort(np.random.default_rng(TSEED).choice(p.shape[0], NT, replace=False))
    t0 = time.time()
    u_fmm = OF.fmm(OF.Plan(p, K, OF.FMMParams(eps=EPS)), f)[0, t]
    t1 = time.time()
    u_dir = OD.direct(p, f, t, chunk=8)[0]
    t2 = time.time()
    err = np.linalg.norm(u_fmm - u_dir) / np.linalg.norm(u_dir)
    with open(OUT, "w") as fh:
        fh.write(f"# sphere K={K:g} N={p.shape[0]} seed {SEED}, densities seed {FSEED} (nrhs 1), eps {EPS:g}\n")
        fh.write(f"# targets: {NT} drawn with numpy default_rng({TSEED}).choice(N, {NT}, replace=False), sorted\n")
        fh.write(f"# oracle FMM vs direct sum on these targets: {err:.3e} (FMM {t1 - t0:.0f} s, direct {t2 - t1:.0f} s)\n")
        fh.write("# target  fmm_re  fmm_im  direct_re  direct_im\n")
        for i, k in enumerate(t):
            vals = (u_fmm[i].real, u_fmm[i].imag, u_dir[i].real, u_dir[i].imag)
            fh.write(f"{k} " + " ".join(repr(float(v)) for v in vals) + "\n")
    print(f"wrote {OUT}: FMM vs direct {err:.3e}, FMM {t1 - t0:.0f} s, direct {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
