#!/usr/bin/env python
"""Benchmark of the directional FMM matvec on GB300.

Workload (default): a sphere of diameter K = 64 wavelengths, N = 1,286,796
uniform surface points (seed 1, 100 points per square wavelength), complex64
standard-normal densities, eps = 1e-5, one right-hand side.  A step is one
full matvec u = G f (every stage of Alg. 1 plus the near field) through the
C ABI, with the plan resident.  Metric: points x RHS per second.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (direct sum of Eq. 1 on a bounded target sample per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec points*RHS/s at <=1e-5 rel err, chosen vs plain; p50/p99 latency"
WORKLOADS = {
    "sphere_K64": dict(K=64.0, seed=1, eps=1e-5, desc="sphere diameter 64, N=1,286,796 (seed 1), eps 1e-5"),
    "sphere_K8": dict(K=8.0, seed=0, eps=1e-6, desc="sphere diameter 8, N=20,106 (seed 0), eps 1e-6"),
    "sphere_K8_eps1e8": dict(K=8.0, seed=0, eps=1e-8,
                             desc="sphere diameter 8, N=20,106 (seed 0), eps 1e-8 (FP64 form, complex128)"),
    "sphere_K16": dict(K=16.0, seed=1, eps=1e-5, desc="sphere diameter 16, N=80,424 (seed 1), eps 1e-5"),
    "sphere_K32": dict(K=32.0, seed=1, eps=1e-5, desc="sphere diameter 32, N=321,699 (seed 1), eps 1e-5"),
    "ellipsoid_K128": dict(K=128.0, seed=2, eps=1e-5, axes=(64.0, 32.0, 16.0),
                           desc="ellipsoid semi-axes (64, 32, 16), K=128, N=1,625,002 (seed 2), eps 1e-5"),
}


def points_of(wl):
    import workloads
    if "axes" in wl:
        return workloads.ellipsoid(*wl["axes"], seed=wl["seed"])
    return workloads.sphere(wl["K"], wl["seed"])


def peaks():
    p = {"hbm_gbs": 6778.0, "bf16_tflops": 1884.5, "sm_max_mhz": 2070.0, "source": "measured"}
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p.update({k: m[k] for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz") if k in m})
    except Exception:
        p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    # FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock
    p["fp32_tflops"] = 152 * 128 * 2 * p["sm_max_mhz"] * 1e6 / 1e12
    return p


class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.out.flush()
        rows = [l.split(",") for l in open(self.out.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.out.name)
        sm = sorted(float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 9 for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def traffic_for(kernel: str, source: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    this workload with the current kernel source (null otherwise)."""
    # the kernel source and the plan builder (which fixes operators and tiles)
    h = hashlib.sha256()
    for name in source.split("+"):
        h.update(open(os.path.join(ROOT, "paper_1311_4257_gb300", "csrc", name), "rb").read())
    h = h.hexdigest()[:12]
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))) if os.path.isdir(os.path.join(ROOT, "profiles")) else []:
        if not fn.endswith(".md"):
            continue
        t = open(os.path.join(ROOT, "profiles", fn)).read()
        m = re.search(r"traffic\[%s @ %s\]\s*=\s*([0-9.eE+]+)\s+bytes per launch\s+\(%s %s\)" % (
            kernel, re.escape(workload), re.escape(source), h), t)
        if m:
            return float(m.group(1))
    return None


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over the ranks of the process group (x itself on one rank)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def cpu_oracle_sample(points, f, ntgt: int, seed: int, pool=None):
    """The oracle's direct sum (FP64 numpy) on ntgt targets: over the processes of
    `pool` (one per host core) if given, else in this process (one core)."""
    import numpy as np
    from oracle.direct import direct
    t = np.random.default_rng(seed).choice(points.shape[0], ntgt, replace=False)
    t0 = time.perf_counter()
    ref = pool.run(t) if pool is not None else direct(points, f, t, chunk=8)
    dt = time.perf_counter() - t0
    return t, ref, dt


def oracle_pool(points, f):
    """Worker processes for the oracle's direct sum, one per host core."""
    from oracle.direct import DirectPool
    return DirectPool(points, f, os.cpu_count() or 1)


def run_reference(args, wl):
    import numpy as np
    import workloads
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K = wl["K"]
    p = points_of(wl)
    N = p.shape[0]
    f = workloads.densities(N, args.nrhs, wl["seed"])
    ntgt = args.ref_targets or 400
    pool = oracle_pool(p, f)
    for _ in range(args.warmup and 1):
        cpu_oracle_sample(p, f, max(8, ntgt // 8), 99, pool)
    times = []
    for s in range(args.steps):
        _, _, dt = cpu_oracle_sample(p, f, ntgt, 1000 + s, pool)
        times.append(dt)
    pool.close()
    tot = sum(times)
    value = ntgt * args.nrhs * args.steps / tot
    cores = pool.workers
    line = {"metric": METRIC, "value": value, "unit": "points*RHS/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl["desc"], "N": N, "K": K, "eps": wl["eps"], "nrhs": args.nrhs,
                       "method": "oracle direct sum of Eq. 1 (FP64 numpy), bounded target sample per step"},
            "cpu_baseline": {"value": value, "unit": "points*RHS/s", "cores": cores, "kind": "oracle",
                             "sample": f"{ntgt} targets x {N} sources per step (direct sum), "
                                       f"targets split over {cores} processes"},
            "e2e": {"value": value, "unit": "points*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, wl):
    import numpy as np
    import torch
    import workloads
    from paper_1311_4257_gb300 import Plan
    from paper_1311_4257_gb300 import build as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()
    probes = None
    if rank == 0 and not args.no_probes:
        # measured denominators (FP32 / FP64 FMA, MUFU, tcgen05 TF32 and F16), with the SM clock beside them
        from paper_1311_4257_gb300.dfmm import measure_peaks
        measure_peaks()   # warm-up: clocks ramp, modules load
        pclk = Clocks(local)
        pclk.start()
        probes = measure_peaks()
        probes["clocks"] = pclk.stop()
    K = wl["K"]
    p = points_of(wl)
    N = p.shape[0]
    nrhs = args.nrhs
    f = workloads.densities(N, nrhs, wl["seed"])
    t0 = time.perf_counter()
    plan = Plan(p, K, wl["eps"], cache_dir=args.cache_dir, m2l_mode={"auto": 0, "fp32": 1, "tc": 2}[args.form])
    plan_s = time.perf_counter() - t0
    st = plan.stats()
    fd = torch.as_tensor(f.astype(plan.np_dtype), device="cuda")
    ud = torch.empty_like(fd)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.apply(fd, ud)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    e0.record(stream)
    for _ in range(args.steps):
        plan.apply(fd, ud)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-step latency distribution (separately, events around each step)
    for _ in range(min(args.steps, 20)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.apply(fd, ud)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    lat.sort()
    ms_max = max_over_ranks(ms, dist)
    value = whole_job_rate(N * nrhs, world, ms_max)
    # the same steps as one captured CUDA graph each (dfmm_graph_*)
    graph_ms = None
    if world == 1:
        gr = plan.graph(fd, ud)
        for _ in range(2):
            gr.launch()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            gr.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1) / args.steps
        gr.close()
    # end to end through the host-buffer entry point (pinned buffers)
    fh = torch.as_tensor(f.astype(plan.np_dtype)).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    plan.apply_host_ptr(fh.data_ptr(), uh.data_ptr(), nrhs)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(args.steps):
        plan.apply_host_ptr(fh.data_ptr(), uh.data_ptr(), nrhs)
    e2e_ms = 1e3 * (time.perf_counter() - te) / args.steps
    # per-kernel timing with CUDA events recorded by the library on this stream
    plan.profile_start()
    nprof = 3
    for _ in range(nprof):
        plan.apply(fd, ud)
    prof = plan.profile_stop()
    torch.cuda.synchronize()
    pk = peaks()
    if probes:
        pk["fp32_tflops"] = probes["fp32_fma_tflops"]
        pk["fp32_source"] = "measured (dfmm_measure_peaks, FP32 FMA probe)"
    else:
        pk["fp32_source"] = "derived: 152 SM x 128 lanes x 2 x max SM clock"
    tc = (args.form == "tc") or (args.form == "auto" and wl["eps"] >= 1e-5)
    fp64 = plan.arith == 64   # FP64 form (eps < 1e-6): CUDA-core FP64 arithmetic throughout
    if fp64:
        pk["fp32_tflops"] = probes["fp64_fma_tflops"] if probes else 1.25
        pk["fp32_source"] = ("measured (dfmm_measure_peaks, FP64 FMA probe)" if probes else
                             "GB300 nominal FP64 rate 1.25 TFLOP/s (the probe measures 1.25)")
    # roofline of each stage family: translations on the tensor pipe (useful flops
    # against the FP16 peak / 3 MMAs) or the FP32 pipe, P2P on the FP32 pipe,
    # row streams and permutes on HBM
    gemm_fams = ("m2l_hf", "m2l_lf", "m2m", "l2l", "p2l_proj")
    stages = {}
    for name, v in prof.items():
        per = v["ms"] / nprof
        entry = {"launches_per_step": v["launches"] // nprof, "ms_per_step": per}
        if v["flops"] > 0:
            entry["tflops"] = v["flops"] / (v["ms"] / 1e3) / 1e12
        if v["bytes"] > 0:
            entry["gbs"] = v["bytes"] / (v["ms"] / 1e3) / 1e9
        if name in gemm_fams and "tflops" in entry:
            pkv = pk["bf16_tflops"] / 3 if tc else pk["fp32_tflops"]
            entry["frac"] = entry["tflops"] / pkv
            entry["bound"] = "tensor (FP16 peak / 3)" if tc else ("fp64 FMA" if fp64 else "fp32 FMA")
        elif name in ("p2p", "p2l_eval") and "tflops" in entry:
            entry["frac"] = entry["tflops"] / pk["fp32_tflops"]
            entry["bound"] = ("fp64" if fp64 else "fp32") + " FMA (16 + 8 nrhs flops per interaction)"
            if name == "p2p" and probes and not fp64:
                # each interaction issues one reciprocal square root and one sine + cosine
                # pair on the special-function unit: the measured rates bound the kernel
                # (once per pass of up to 4 right-hand sides)
                passes = -(-nrhs // (1 if nrhs == 1 else (2 if nrhs == 2 else 4)))
                t_mufu = st["p2p_interactions"] * passes * (1.0 / (probes["sincos_gops"] * 1e9) +
                                                            1.0 / (probes["rsqrt_gops"] * 1e9))
                entry["mufu_bound_ms"] = 1e3 * t_mufu
                entry["frac_of_mufu_bound"] = 1e3 * t_mufu / per
        elif "gbs" in entry:
            entry["frac"] = entry["gbs"] / pk["hbm_gbs"]
            entry["bound"] = "hbm"
        stages[name] = entry
    # the dominant kernel: the translation-stage GEMM, over all its launches
    gfam = [k for k in ("m2l_hf", "m2l_lf", "m2m", "l2l", "p2l_proj") if k in prof]
    g_ms = sum(prof[k]["ms"] for k in gfam)
    g_flops = sum(prof[k]["flops"] for k in gfam)
    launches = sum(prof[k]["launches"] for k in gfam)
    achieved = g_flops / (g_ms / 1e3) / 1e12
    share = g_ms / sum(v["ms"] for v in prof.values())
    if tc:
        # the scaled FP16 split issues 3 MMAs (hi hi, hi lo, lo hi) per useful
        # multiply-add; FP16 dense runs at the BF16 rate (measured)
        f16 = pk["bf16_tflops"]
        roofline = {"kernel": "gemm_cx_kernel (all translation stages; split-complex form)", "bound": "tensor",
                    "achieved": achieved,
                    "peak": f16 / 3, "unit": "TFLOP/s", "frac": achieved / (f16 / 3),
                    "issued_tflops": 3 * achieved, "issued_frac_of_f16_peak": 3 * achieved / f16,
                    "peak_source": "measured bf16 dense %.1f TF/s (FP16 runs at the same rate), / 3 MMAs per "
                                   "useful product" % pk["bf16_tflops"]}
    else:
        roofline = {"kernel": "gemm64_kernel (all translation stages)" if fp64 else
                    "gemm_stage_kernel (all translation stages)", "bound": "alu", "achieved": achieved,
                    "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "frac": achieved / pk["fp32_tflops"],
                    "peak_source": "%s CUDA-core peak, %s" % ("FP64" if fp64 else "FP32", pk["fp32_source"])}
    roofline.update({"traffic": traffic_for("gemm_cx_kernel", "m2l_cx.cu+dfmm.cpp", args.workload) if tc else
                     (None if fp64 else traffic_for("gemm_stage_kernel", "apply.cu+dfmm.cpp", args.workload)),
                     "launches_per_step": launches / nprof, "ms_per_launch": g_ms / launches,
                     "flops_per_launch": g_flops / launches, "share_of_step": share})
    out = {"metric": METRIC, "value": value, "unit": "points*RHS/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c128 (fp64)" if fp64 else "c64 (fp32)", "data": "synthetic",
           "config": {"workload": wl["desc"], "N": N, "K": K, "eps": wl["eps"], "nrhs": nrhs,
                      "form": "tensor cores (tcgen05, scaled FP16 hi/lo split, one accumulator per component)" if tc else
                      ("FP64 CUDA cores" if fp64 else "FP32 CUDA cores"),
                      "parallelism": "replicas" if world > 1 else "1 gpu",
                      "l2": "inputs larger than L2 (plan %.1f GB resident, states re-zeroed each step)" % (st["plan_bytes"] / 1e9),
                      "plan_seconds": plan_s,
                      "plan_phase_seconds": dict(zip(("tree_lists", "skeletons", "rep_upload", "operators", "rows",
                                                      "near_field", "tc_images", "operators_on_device"),
                                                     st["plan_phase_seconds"]))},
           "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
           "graph_ms_per_step": graph_ms,
           "e2e": {"value": N * nrhs / (e2e_ms / 1e3), "unit": "points*RHS/s",
                   "h2d_bytes_per_step": fd.element_size() * N * nrhs, "d2h_bytes_per_step": fd.element_size() * N * nrhs},
           "gpu_launches": plan.launches(nrhs) * args.steps,
           "clocks": clocks, "roofline": roofline, "stages": stages, "probes": probes}
    if args.compare and rank == 0 and not fp64:
        # the plain form (FP32 CUDA cores, one RHS) and the batched chosen form (16 RHS)
        # (own output buffers: ud keeps the chosen form's potentials for the error below)
        plain = Plan(p, K, wl["eps"], cache_dir=args.cache_dir, m2l_mode=1)
        u_plain = torch.empty_like(fd)
        for _ in range(2):
            plain.apply(fd, u_plain)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            plain.apply(fd, u_plain)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / 5
        del plain
        if tc:
            # the separate-accumulator variant (tc_accumulate 2): the hi*hi terms and the
            # cross terms in their own tensor-memory accumulators, one tile at a time
            fast = Plan(p, K, wl["eps"], cache_dir=args.cache_dir, tc_accumulate=2)
            u_fast = torch.empty_like(fd)
            for _ in range(2):
                fast.apply(fd, u_fast)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                fast.apply(fd, u_fast)
            e1.record(stream)
            torch.cuda.synchronize()
            out["two_accumulator_form"] = {"value": N / (e0.elapsed_time(e1) / args.steps / 1e3),
                                           "unit": "points*RHS/s", "ms_per_step": e0.elapsed_time(e1) / args.steps}
            del fast
        f16 = torch.as_tensor(workloads.densities(N, 16, wl["seed"] + 1).astype(np.complex64), device="cuda")
        u16 = torch.empty_like(f16)
        for _ in range(2):
            plan.apply(f16, u16)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            plan.apply(f16, u16)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / 5
        out["plain_vs_chosen"] = {"plain_fp32_nrhs1": N / (pms / 1e3), "chosen_nrhs1": value,
                                  "chosen_nrhs16": 16 * N / (bms / 1e3),
                                  "speedup_nrhs1": value / (N / (pms / 1e3)),
                                  "speedup_nrhs16": 16 * N / (bms / 1e3) / (N / (pms / 1e3)),
                                  "unit": "points*RHS/s"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(p, f)
        t, ref, dt = cpu_oracle_sample(p, f, args.ref_targets or 1600, 1001, pool)
        pool.close()
        u = ud.cpu().numpy()
        err = float(np.linalg.norm(u[:, t] - ref) / np.linalg.norm(ref))
        out["rel_err_vs_direct_sum"] = {"value": err, "targets": int(len(t))}
        if "two_accumulator_form" in out:
            uf = u_fast.cpu().numpy()
            out["two_accumulator_form"]["rel_err_vs_direct_sum"] = float(np.linalg.norm(uf[:, t] - ref) /
                                                                         np.linalg.norm(ref))
        t1, _, dt1 = cpu_oracle_sample(p, f, max(8, (args.ref_targets or 1600) // 16), 1002)
        out["cpu_baseline"] = {"value": len(t) * nrhs / dt, "unit": "points*RHS/s", "cores": pool.workers,
                               "kind": "oracle",
                               "sample": f"direct sum of Eq. 1 (FP64 numpy) for {len(t)} targets x {N} sources, "
                                         f"targets split over {pool.workers} processes",
                               "one_core": {"value": len(t1) * nrhs / dt1, "targets": int(len(t1))}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_stage_errors(args, wl):
    """Error of the tensor-core splits: for the FP16 split, one plan per translation
    family with only that family on the tensor cores (options.tc_stages); then every
    family on the tensor cores with each split (FP16, 3xBF16, 3xTF32).  Each against
    the FP32 CUDA-core form of the same points and against the FP64 direct sum, with
    the apply time of each form beside it."""
    import numpy as np
    import torch
    import workloads
    from oracle.direct import rel_err
    from paper_1311_4257_gb300 import Plan
    from paper_1311_4257_gb300 import build as B
    B.build()
    p = points_of(wl)
    N = p.shape[0]
    f = workloads.densities(N, 1, wl["seed"])
    fd = torch.as_tensor(f.astype(np.complex64), device="cuda")
    pool = oracle_pool(p, f)
    t, ref, _ = cpu_oracle_sample(p, f, args.ref_targets or 1600, 1001, pool)
    pool.close()
    forms = [("fp32_cuda_cores", dict(m2l_mode=1)),
             ("fp16_m2l_hf", dict(m2l_mode=2, tc_stages=1)), ("fp16_m2l_lf", dict(m2l_mode=2, tc_stages=2)),
             ("fp16_m2m", dict(m2l_mode=2, tc_stages=4)), ("fp16_l2l", dict(m2l_mode=2, tc_stages=8)),
             ("fp16_p2l_proj", dict(m2l_mode=2, tc_stages=16)),
             ("fp16_all", dict(m2l_mode=2)), ("bf16_all_3xBF16", dict(m2l_mode=2, tc_precision=1)),
             ("tf32_all_3xTF32", dict(m2l_mode=2, tc_precision=2))]
    out, u32 = {}, None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, kw in forms:
        plan = Plan(p, wl["K"], wl["eps"], cache_dir=args.cache_dir, **kw)
        u = plan.apply(fd)
        for _ in range(2):
            plan.apply(fd, u)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            plan.apply(fd, u)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        u = u.cpu().numpy().astype(np.complex128)
        del plan
        torch.cuda.empty_cache()
        if u32 is None:
            u32 = u
        out[name] = {"vs_direct_sum_fp64": rel_err(u[:, t], ref), "vs_fp32_form": rel_err(u, u32), "ms": ms}
    print(json.dumps({"metric": "relative error of the tensor-core splits (scaled hi / lo: FP16, 3xBF16, 3xTF32)",
                      "workload": wl["desc"], "N": N, "eps": wl["eps"], "direct_sum_targets": int(len(t)),
                      "stages": out}), flush=True)


def _plain_rate(plans_pts, cache_dir, max_cols: int = 4):
    """Points x RHS per second of the plain form: FP32 CUDA-core plans, one
    right-hand side per apply, one apply at a time, over each geometry (at
    most max_cols columns each, so the comparison stays short)."""
    import numpy as np
    import torch
    import workloads
    from paper_1311_4257_gb300 import Plan
    pts_rhs, secs = 0.0, 0.0
    for p, K, eps, cols in plans_pts:
        plain = Plan(p, K, eps, cache_dir=cache_dir, m2l_mode=1)
        f1 = torch.as_tensor(workloads.densities(p.shape[0], 1, 77).astype(np.complex64), device="cuda")
        plain.apply(f1)
        torch.cuda.synchronize()
        c = min(cols, max_cols)
        t0 = time.perf_counter()
        for _ in range(c):
            plain.apply(f1)
        torch.cuda.synchronize()
        secs += time.perf_counter() - t0
        pts_rhs += p.shape[0] * c
        plain.close()
    return pts_rhs / secs


def run_batch12(args):
    """The batched form: twelve geometries of uneven size and uneven RHS
    counts in one dfmm_apply_batched call per step."""
    import numpy as np
    import torch
    import workloads
    from paper_1311_4257_gb300 import Plan, apply_batched
    from paper_1311_4257_gb300 import build as B
    from oracle import direct as OD
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    geo = workloads.batch_geometries()
    t0 = time.perf_counter()
    plans = [Plan(p, K, 1e-5, cache_dir=args.cache_dir) for _, p, K, _ in geo]
    plan_s = time.perf_counter() - t0
    fs = [torch.as_tensor(workloads.densities(p.shape[0], r, 60 + k).astype(np.complex64), device="cuda")
          for k, (_, p, _, r) in enumerate(geo)]
    us = [torch.empty_like(f) for f in fs]
    for _ in range(args.warmup):
        apply_batched(plans, fs, us)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        apply_batched(plans, fs, us)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    work = sum(p.shape[0] * r for _, p, _, r in geo)
    # the same work one geometry at a time (all its RHS in one apply)
    e0.record()
    for pl, f, u in zip(plans, fs, us):
        pl.apply(f, u)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    # accuracy: every geometry against the direct sum on 50 targets, first RHS
    errs = {}
    for (name, p, _, r), u, f in zip(geo, us, fs):
        t = np.random.default_rng(5).choice(p.shape[0], 50, replace=False)
        ud = OD.direct(p, f[:1].cpu().numpy().astype(np.complex128), t, chunk=8)
        errs[name] = OD.rel_err(u[:1].cpu().numpy()[:, t].astype(np.complex128), ud)
    # the merged form: one launch per translation stage across the 12 geometries,
    # autotuned tile orders, the whole batch replayed as one captured graph
    from paper_1311_4257_gb300 import Batch
    us2 = [torch.empty_like(f) for f in fs]
    t0 = time.perf_counter()
    batch = Batch(plans, fs, us2, graph=True, tune=True)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        batch.launch()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    ms_m = e0.elapsed_time(e1) / args.steps
    dev = max(OD.rel_err(a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128))
              for a, b in zip(us2, us))
    merged = {"ms_per_step": ms_m, "points_rhs_per_s": work / (ms_m / 1e3), "setup_seconds": setup_s,
              "launches_of_the_single_applies": int(sum(pl.launches(r) for pl, (_, _, _, r) in zip(plans, geo))),
              "max_rel_diff_vs_stream_form": dev, **batch.stats()}
    batch.close()
    plain = _plain_rate([(p, K, 1e-5, r) for _, p, K, r in geo], args.cache_dir) if args.compare else None
    line = {"metric": METRIC, "value": work / (ms / 1e3), "unit": "points*RHS/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 (fp32)", "data": "synthetic",
            "config": {"workload": "batch of 12 geometries (spheres K=8..48, ellipsoids K=16..64, tori R=8..32; "
                                   "seeds 10-21; nrhs 1/4/16/32 round-robin), eps 1e-5",
                       "points": int(sum(p.shape[0] for _, p, _, _ in geo)), "points_x_rhs": int(work),
                       "plan_seconds": plan_s},
            "sequential_same_work_ms": ms_seq,
            "merged_graph_form": merged,
            "plain_fp32_single_rhs_rate": plain,
            "speedup_vs_plain": (work / (ms / 1e3)) / plain if plain else None,
            "rel_err_vs_direct_sum_50_targets": errs}
    print(json.dumps(line), flush=True)


def run_solve(args):
    """GMRES around the resident matvec: x + (4 / K) (a / 4 pi) G x = b on the
    sphere K = 64 (a = area per point), to the plan's tolerance."""
    import numpy as np
    import torch
    import workloads
    from paper_1311_4257_gb300 import Plan
    from paper_1311_4257_gb300 import build as B
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    wl = WORKLOADS["sphere_K64"]
    p = points_of(wl)
    plan = Plan(p, wl["K"], wl["eps"], cache_dir=args.cache_dir)
    b = torch.as_tensor(workloads.densities(p.shape[0], 1, 11)[0].astype(np.complex64), device="cuda")
    # identity plus the single-layer sum scaled by 4 / K, so that |beta G| stays
    # near 1 at every size (unscaled, (1/2) I + S stagnates at K = 64)
    alpha, beta = 1.0, (1.0 / workloads.POINTS_PER_SQ_WAVELENGTH) / (4 * np.pi) * (4.0 / wl["K"])
    plan.solve(b, alpha, beta, tol=1e-2)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, it, rr = plan.solve(b, alpha, beta, tol=wl["eps"], restart=60, maxit=300)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    line = {"metric": "GMRES solve of x + (4/K)(a/4pi) G x = b, seconds to rel. residual <= eps",
            "value": sec, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * sec,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32)",
            "data": "synthetic", "config": {"workload": wl["desc"], "restart": 60},
            "matvecs": it, "true_relative_residual": rr, "ms_per_iteration": 1e3 * sec / max(1, it + 1)}
    print(json.dumps(line), flush=True)


def run_served8(args):
    """The served form: a Poisson request stream over eight resident plans,
    served by the library's request server."""
    import numpy as np
    import torch
    import workloads
    from paper_1311_4257_gb300 import Plan, Server
    from paper_1311_4257_gb300 import build as B
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    B.build()
    geo = workloads.served_geometries()
    t0 = time.perf_counter()
    plans = [Plan(p, K, 1e-5, cache_dir=args.cache_dir) for _, p, K in geo]
    plan_s = time.perf_counter() - t0
    n = args.requests
    rng = np.random.default_rng(30)
    which = rng.integers(0, len(plans), n)
    nrhs = rng.integers(1, 17, n)
    arrive = workloads.poisson_arrivals(n, args.rate, 30)
    # host buffers: one pinned density block of 16 RHS per plan, and a ring of
    # 8 result buffers per plan (a request writes slot k mod 8)
    fh = [torch.as_tensor(workloads.densities(pl.N, 16, 90 + k).astype(np.complex64)).pin_memory()
          for k, pl in enumerate(plans)]
    uh = [[torch.empty((16, pl.N), dtype=torch.complex64).pin_memory() for _ in range(8)] for pl in plans]
    budget = int(args.budget_gb * (1 << 30))

    def serve(times, count):
        srv = Server(streams=4, budget_bytes=budget, max_rhs=16)
        tick = []
        start = time.perf_counter()
        for k in range(count):
            if times is not None:
                dt = times[k] - (time.perf_counter() - start)
                if dt > 0:
                    time.sleep(dt)
            w = int(which[k])
            tick.append(srv.submit(plans[w], fh[w].data_ptr(), uh[w][k % 8].data_ptr(), int(nrhs[k])))
        for t in tick:
            srv.wait(t, timeout=600.0)
        st = srv.stats()
        srv.close()
        return st

    serve(arrive[:16] - arrive[0], 16)      # warm-up
    st = serve(arrive, n)
    sat = serve(None, n)                     # all requests at once: capacity
    work = float(sum(plans[w].N * r for w, r in zip(which, nrhs)))
    # the same stream at 60% of the measured capacity: latency without backlog
    cap_rate = sat["points_rhs_done"] / sat["wall_seconds"] / (work / n)
    light = serve(workloads.poisson_arrivals(n, 0.6 * cap_rate, 32), n)
    plain = _plain_rate([(p, K, 1e-5, 16) for _, p, K in geo], args.cache_dir) if args.compare else None
    line = {"metric": METRIC, "value": sat["points_rhs_done"] / sat["wall_seconds"], "unit": "points*RHS/s",
            "n_gpus": 1, "steps": n, "warmup": 20, "ms_per_step": 1e3 * sat["wall_seconds"] / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32)",
            "data": "synthetic",
            "config": {"workload": "served: %d requests over 8 resident plans (spheres K=16/32/64, ellipsoids "
                                   "K=32/128, tori R=16/32, cube edge 48; seeds 40-47), nrhs U{1..16}, eps 1e-5"
                                   % n, "server": "4 streams, max 16 RHS per apply, %.0f GB arena" % args.budget_gb,
                       "plan_seconds": plan_s, "points_x_rhs": work},
            "poisson": {"rate_req_per_s": args.rate, "latency_p50_ms": st["latency_p50_ms"],
                        "latency_p99_ms": st["latency_p99_ms"], "applies": st["applies"],
                        "points_rhs_per_s": st["points_rhs_done"] / st["wall_seconds"],
                        "max_concurrent_applies": st["max_concurrent_applies"]},
            "saturated": {"latency_p50_ms": sat["latency_p50_ms"], "latency_p99_ms": sat["latency_p99_ms"],
                          "applies": sat["applies"], "max_concurrent_applies": sat["max_concurrent_applies"]},
            "poisson_at_60pct_capacity": {"rate_req_per_s": 0.6 * cap_rate, "latency_p50_ms": light["latency_p50_ms"],
                                          "latency_p99_ms": light["latency_p99_ms"], "applies": light["applies"],
                                          "points_rhs_per_s": light["points_rhs_done"] / light["wall_seconds"]},
            "plain_fp32_single_rhs_rate": plain,
            "speedup_vs_plain": (sat["points_rhs_done"] / sat["wall_seconds"]) / plain if plain else None}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere_K64", choices=sorted(WORKLOADS) + ["batch12", "served8", "solve_K64"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--ref-targets", type=int, default=None,
                    help="oracle targets per sample (default: 1600 beside the GPU arm, 400 per reference step)")
    ap.add_argument("--cache-dir", default=os.path.join(tempfile.gettempdir(), "dfmm_cache"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="auto", choices=["auto", "fp32", "tc"])
    ap.add_argument("--compare", dest="compare", action="store_true", default=True,
                    help="also time the plain FP32 form and 16 RHS (default)")
    ap.add_argument("--no-compare", dest="compare", action="store_false")
    ap.add_argument("--no-probes", action="store_true", help="skip the peak-rate probes")
    ap.add_argument("--requests", type=int, default=2000, help="served8: requests in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="served8: Poisson arrival rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="served8: the server's device arena")
    ap.add_argument("--stage-errors", action="store_true",
                    help="instead of timing: the error each translation family's tensor-core split adds")
    args = ap.parse_args()
    os.makedirs(args.cache_dir, exist_ok=True)
    if args.workload in ("batch12", "served8", "solve_K64"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched, served and solve forms have no "
                              "oracle timing; use a single-geometry workload"}), flush=True)
        elif int(os.environ.get("RANK", "0")) == 0:
            {"batch12": run_batch12, "served8": run_served8, "solve_K64": run_solve}[args.workload](args)
        return
    wl = WORKLOADS[args.workload]
    if args.stage_errors:
        if int(os.environ.get("RANK", "0")) == 0:
            run_stage_errors(args, wl)
        return
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
