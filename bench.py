#!/usr/bin/env python3
"""Benchmark of the polyspectrum estimator on GB300.

One step = one poly_estimate of one 256^3 lognormal field with 64 unit-width
shells (n = 3, 24,432 triangle bins): forward transform, 64 shell fields,
product-sum contraction, reduction and normalisation (counts are plan-time).
The metric is configs/s = output bins per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank estimates its own field (weak scaling, no collective on
the data path); rank 0 prints one JSON line.  `--impl reference` times the FP64
CPU oracle (the plain definition of the method) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bispectrum configs/s at 256³ N_max=64, split-BF16 vs FP32 on GB300 at rel err ≤1e-5"
N, L, NSHELL, ORDER, SEED, WIDTH, ELL = 256, 1000.0, 64, 3, 2, 1.0, 0
WORKLOAD = "bispectrum, 256^3 lognormal field (seed 2), 64 unit shells k_F..64k_F, n=3, 24432 bins"


def set_workload(n: int, nshell: int, order: int, width: float = 1.0, ell: int = 0):
    """Other sizes (profiling cases, trispectrum, multipoles); the default is the metric's workload."""
    global N, NSHELL, ORDER, WORKLOAD, WIDTH, ELL
    if (n, nshell, order, width, ell) == (N, NSHELL, ORDER, WIDTH, ELL):
        return
    N, NSHELL, ORDER, WIDTH, ELL = n, nshell, order, width, ell
    WORKLOAD = (f"order-{order} polyspectrum{f', multipole ell={ell} (first leg)' if ell else ''}, {n}^3 lognormal "
                f"field (seed 2), {nshell} shells of width {width:g} k_F (not the metric workload)")
SAMPLE_SHELLS = (59, 60, 61, 62, 63, 64)  # CPU baseline sample: the bins among these shells


TC_SOURCES = ["contract_tc.cu", "tc.cuh", "common.cuh"]
CC_SOURCES = ["contract_cc.cu", "common.cuh"]
FIELD_SOURCES = ["fields_impl.cuh", "fields_f32.cu", "fft.cuh", "common.cuh"]
ADJ_SOURCES = ["adjoint_tc.cu", "tc.cuh", "common.cuh"]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1904_11055_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def workload_key(n: int, nshell: int, order: int, width: float = 1.0, ell: int = 0, prec: str = "") -> str:
    return f"n{order}-{n}cube-{nshell}x{width:g}" + (f"-ell{ell}" if ell else "") + (f"-{prec}" if prec else "")


def traffic_for(kernel: str, src_files, key: str, config: int | None = None):
    """DRAM bytes per launch from a committed ncu summary of this kernel on this workload, if it was
    captured from the current source and, for the tensor-core contraction, at the same launch shape
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(f"{kernel}@{key}")
    except Exception:
        return None
    if not rec or rec.get("source_hash") != source_hash(*src_files):
        return None
    if config is not None and rec.get("contraction_config") not in (None, config):
        return None
    return rec.get("bytes_per_launch")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(delta_f32):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import numpy as np

    import fieldgen
    import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    edges = fieldgen.unit_edges(NSHELL, WIDTH)
    allb = oracle.enumerate_bins(edges, ORDER)
    sel = np.array([i for i, b in enumerate(allb) if set(b.tolist()) <= set(SAMPLE_SHELLS)])
    t0 = time.perf_counter()
    ref = oracle.estimate(delta_f32.astype(np.float64), L, edges, ORDER, bins=allb[sel])
    dt = time.perf_counter() - t0
    # the small case on one thread: 64^3 Gaussian field (cut above 16 k_F), 16 unit shells, all 508 bins
    oracle.set_threads(1)
    d1, e1 = fieldgen.field("gaussian_cut16", 64, 1, np.float64), fieldgen.unit_edges(16)
    t1 = time.perf_counter()
    ref64 = oracle.estimate(d1, L, e1, 3)
    nb1 = len(ref64["B"])
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    t2 = time.perf_counter()
    oracle.estimate(d1, L, e1, 3)
    dt2 = time.perf_counter() - t2
    cpu_baseline.ref64 = ref64
    cpu_baseline.rate64 = {"one_thread": nb1 / dt1, "all_cores": nb1 / dt2, "cores": cores}
    return {"value": len(sel) / dt, "unit": "configs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} bins among shells {SAMPLE_SHELLS[0]}-{SAMPLE_SHELLS[-1]} of the 256^3 field "
                      f"(full forward FFT, 6 shell + 6 counting fields, FP64), {dt:.1f} s",
            "one_thread": {"value": nb1 / dt1, "unit": "configs/s", "cores": 1, "seconds": dt1,
                           "workload": "64^3 Gaussian field cut above 16 k_F, 16 unit shells, all 508 bins, "
                                       "counts included, FP64"}}, sel, ref


def cufft_fields_ms(torch, d, edges, reps=3):
    """The shell fields through cuFFT (torch.fft), as a timed cross-check of the library's pruned transforms:
    one full R2C, then per shell a mask multiply and a full C2R into one reused buffer (N_max x N^3 outputs
    written, as the library writes).  Device-timed median of `reps`."""
    N = d.shape[0]
    f = torch.fft.fftfreq(N, d=1.0 / N, device=d.device)
    fz = torch.fft.rfftfreq(N, d=1.0 / N, device=d.device)
    q2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2
    e2 = torch.tensor([float(x) ** 2 for x in edges], device=d.device, dtype=q2.dtype)
    smap = torch.bucketize(q2, e2, right=True) - 1  # shell s: e_s^2 <= |q|^2 < e_{s+1}^2
    smap[q2 == 0] = -1
    out = torch.empty_like(d)
    ms = []
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        F = torch.fft.rfftn(d)
        for s in range(len(edges) - 1):
            out.copy_(torch.fft.irfftn(torch.where(smap == s, F, 0), s=(N, N, N), norm="forward"))
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms[1:])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import fieldgen
    import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    edges = fieldgen.unit_edges(NSHELL, WIDTH)
    delta = fieldgen.field("lognormal", N, SEED, np.float32).astype(np.float64)
    allb = oracle.enumerate_bins(edges, ORDER)
    shells = (63, 64)  # per step: the 4 bins among the two outermost shells (keeps K steps within minutes)
    sel = allb[[i for i, b in enumerate(allb) if set(b.tolist()) <= set(shells)]]
    for _ in range(args.warmup):
        oracle.estimate(delta, L, edges, ORDER, bins=sel)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.estimate(delta, L, edges, ORDER, bins=sel)
    dt = time.perf_counter() - t0
    val = len(sel) * args.steps / dt
    sample = f"{len(sel)} bins among shells 63-64 of the 256^3 field per step (full forward FFT, FP64)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "configs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "N_max": NSHELL, "order": ORDER, "sample": sample},
        "cpu_baseline": {"value": val, "unit": "configs/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def time_precision(ps, torch, plan, d, args, flush_buf, dist_ok):
    """Device-timed K steps (L2 flushed between steps); returns per-step ms and stage means."""
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.estimate(d)
    ps.poly_plan_set_timing(plan.handle, True)
    plan.estimate(d)
    torch.cuda.synchronize()
    launches0 = ps.poly_plan_stats(plan.handle)["launches"]
    out = torch.empty(plan.nbins, dtype=torch.float64, device=d.device)
    step_ms, stages = [], []
    if dist_ok:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush_buf.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.estimate(d, out=out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stages.append(ps.poly_plan_stats(plan.handle))
    torch.cuda.synchronize()
    if dist_ok:
        torch.distributed.barrier()
    time_precision.last_out = out.cpu().numpy()
    launches = ps.poly_plan_stats(plan.handle)["launches"] - launches0
    ps.poly_plan_set_timing(plan.handle, False)
    mean = {k: statistics.fmean(s[k] for s in stages) for k in ("ms_forward", "ms_fields", "ms_contract", "ms_reduce")}
    mean["contract_flops"] = stages[-1]["contract_flops"]
    return step_ms, mean, launches


def _contract_roofline(prec, useful_flops, ms_contract, peaks, fma, peak_src, burst=False):
    """Roofline of the contraction stage: tensor pipe (split-BF16) or CUDA-core FMA (FP32, FP64)."""
    achieved = useful_flops / (ms_contract * 1e-3) / 1e12
    if prec == "split_bf16":
        key = "bf16_tflops" if burst else "bf16_tflops_sustained"
        peak = peaks.get(key, peaks.get("bf16_tflops"))
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"bf16 dense {'burst' if burst else 'sustained'}, {peak_src}"}
    f = fma["f64" if prec == "fp64" else "f32"]["tflops"]
    return {"bound": "alu", "achieved": achieved, "peak": f, "unit": "TFLOP/s", "frac": achieved / f,
            "peak_source": f"{'FP64' if prec == 'fp64' else 'FP32'} FMA, measured by poly_diag_fma_peak in this run"}


def _median_ms(torch, fn, reps, warm=1):
    for _ in range(warm):
        fn()
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def config1_record(ps, torch, np, peaks, fma, peak_src, flush_buf):
    """64^3 Gaussian field (P ~ k^-1.5 cut above 16 k_F, seed 1), 16 unit shells, n = 3, all 508 bins: the
    plain FP64 method and the FP32 / split-BF16 paths, each against the FP64 oracle on every bin."""
    from types import SimpleNamespace

    import fieldgen

    e1 = fieldgen.unit_edges(16)
    d1 = fieldgen.field("gaussian_cut16", 64, 1, np.float64)
    ref = getattr(cpu_baseline, "ref64", None)
    rec = {"workload": "bispectrum, 64^3 Gaussian field P~k^-1.5 cut above 16 k_F (seed 1), 16 unit shells, n=3, "
                       "all polygon bins", "precisions": {},
           "l2": "256 MiB buffer written between timed steps (L2 flushed)"}
    c_n = (L ** 3) ** 2 / float(64 ** 3) ** 3
    for prec in ("fp64", "fp32", "split_bf16"):
        plan = ps.Plan(64, L, 3, e1, prec)
        d = torch.from_numpy(d1).cuda().to(plan.real_dtype)
        step_ms, stage, launches = time_precision(ps, torch, plan, d, SimpleNamespace(steps=10, warmup=3), flush_buf,
                                                  False)
        B = time_precision.last_out
        ms = statistics.median(step_ms)
        r = {"ms_per_step": ms, "value": plan.nbins / (ms * 1e-3), "unit": "configs/s", "stage_ms": stage,
             "gpu_launches": launches, "steps": 10, "warmup": 3,
             "roofline": _contract_roofline(prec, plan.nbins * 64 ** 3 * 3, stage["ms_contract"], peaks, fma,
                                            peak_src, burst=True)}
        if ref is not None:
            r["error_vs_oracle"] = float(np.max(np.abs(B - ref["B"]) / (c_n * ref["scale"])))
            r["counts_bit_exact"] = bool(np.array_equal(plan.counts, ref["counts"]))
        rec["precisions"][prec] = r
        rec["nbins"] = plan.nbins
        plan.close()
    if ref is not None:
        rec["cpu_oracle"] = {"unit": "configs/s", "kind": "oracle", "sample": "all bins, counts included",
                             **cpu_baseline.rate64}
    return rec


def config3_record(ps, torch, np, peaks, fma, peak_src, flush_buf, delta_np, d):
    """The trispectrum as the paper defines it: 256^3 lognormal field, 32 shells of width 1.5 k_F, n = 4, split-BF16
    and FP32 paths, error against the FP64 oracle on the bins among the two outermost shells; the disconnected part;
    and the full-shape trispectrum (Eq. Tkfull) of bin (10, 10, 10, 10) with diagonal bins of width 1.5 k_F."""
    from types import SimpleNamespace

    import fieldgen
    import oracle

    e3 = fieldgen.unit_edges(32, 1.5)
    allb = oracle.enumerate_bins(e3, 4)
    sel = np.array([i for i, b in enumerate(allb) if set(b.tolist()) <= {31, 32}])
    t0 = time.perf_counter()
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.estimate(delta_np.astype(np.float64), L, e3, 4, bins=allb[sel])
    t_or = time.perf_counter() - t0
    c_n = (L ** 3) ** 3 / float(256 ** 3) ** 4
    rec = {"workload": "trispectrum, 256^3 lognormal field (seed 2), 32 shells of width 1.5 k_F up to 48 k_F, n=4",
           "precisions": {}, "l2": "256 MiB buffer written between timed steps (L2 flushed)",
           "cpu_oracle": {"value": len(sel) / t_or, "unit": "configs/s", "kind": "oracle", "cores": os.cpu_count(),
                          "sample": f"{len(sel)} bins among shells 31-32 (full forward FFT, FP64), {t_or:.1f} s"}}
    kfull = (10, 10, 10, 10)
    for prec, steps in (("split_bf16", 10), ("fp32", 3)):
        torch.cuda.synchronize()
        tp = time.perf_counter()
        plan = ps.Plan(256, L, 4, e3, prec)
        torch.cuda.synchronize()
        plan_ms = (time.perf_counter() - tp) * 1e3
        code = plan.tune(d)[0] if prec == "split_bf16" else 0
        step_ms, stage, launches = time_precision(ps, torch, plan, d, SimpleNamespace(steps=steps, warmup=3),
                                                  flush_buf, False)
        B = time_precision.last_out
        ms = statistics.median(step_ms)
        roof = _contract_roofline(prec, plan.nbins * 256 ** 3 * 4, stage["ms_contract"], peaks, fma, peak_src)
        if prec == "split_bf16":
            roof["traffic"] = traffic_for("tc_contract", TC_SOURCES, workload_key(256, 32, 4, 1.5), code)
        r = {"ms_per_step": ms, "value": plan.nbins / (ms * 1e-3), "unit": "configs/s", "nbins": plan.nbins,
             "steps": steps, "warmup": 3, "stage_ms": stage, "gpu_launches": launches, "roofline": roof,
             "plan_ms": plan_ms, "contraction_shape": code,
             "error_vs_oracle": float(np.max(np.abs(B[sel] - ref["B"]) / (c_n * ref["scale"]))),
             "counts_bit_exact_on_sample": bool(np.array_equal(plan.counts[sel], ref["counts"]))}
        if prec == "split_bf16":
            r["disconnected_ms"] = _median_ms(torch, lambda: plan.disconnected(d), 3)
            # full-shape trispectrum of one bin, diagonals |q1 - q2|, |q1 - q3| in bins of width 1.5 k_F
            de = np.concatenate([[0.0], (np.arange(22) + 0.5) * 1.5])
            out = {}

            def full():
                out["T"], out["C"], out["S"] = plan.trispectrum_full(d, kfull, de, scale=True)

            fms = _median_ms(torch, full, 3)
            C = out["C"].cpu().numpy()
            T, S = out["T"].cpu().numpy(), out["S"].cpu().numpy()
            b = int(np.flatnonzero((plan.bins == np.asarray(kfull)).all(axis=1))[0])
            r["full_shape"] = {
                "bin": list(kfull), "ndiag": int(len(de) - 1), "ms": fms, "quadrilaterals": int(C.sum()),
                "quadrilaterals_per_s": float(C.sum()) / (fms * 1e-3),
                "counts_sum_equals_count_b": bool(C.sum() == plan.counts[b]),
                "sum_error_vs_estimate": float(abs((T * C).sum() - B[b] * plan.counts[b]) / (S * C).sum()),
                "note": "poly_trispectrum_full on the same field and plan, device-timed median of 3; the sum over "
                        "diagonal bins of T*count against B_b*count_b of the same step, in units of sum scale*count"}
        rec["precisions"][prec] = r
        plan.close()
    return rec


def config4_record(ps, torch, np):
    """Checks of the hand-written adjoint at the sizes the oracle and finite differences reach: 64 voxels of a 64^3
    field (16 unit shells, FP64 plan) by central differences, and the FP32 / split-BF16 / FP64 gradients of a 32^3
    field (8 unit shells) against the FP64 oracle gradient."""
    import fieldgen
    import oracle

    rec = {}
    N, e = 64, fieldgen.unit_edges(16)
    d = fieldgen.field("gaussian_cut16", N, 4, np.float64)
    plan = ps.Plan(N, L, 3, e, "fp64")
    w = np.random.default_rng(5).standard_normal(plan.nbins)
    dev = torch.from_numpy(d).cuda()
    wt = torch.from_numpy(w).cuda()
    g = plan.backward(dev, wt).cpu().numpy().reshape(-1)
    vox = np.random.default_rng(6).choice(N ** 3, size=64, replace=False)
    h = 1e-3 * float(d.std())
    flat = dev.view(-1)
    worst = 0.0
    for v in vox:
        flat[v] += h
        lp = float(torch.dot(plan.estimate(dev), wt))
        flat[v] -= 2 * h
        lm = float(torch.dot(plan.estimate(dev), wt))
        flat[v] += h
        worst = max(worst, abs((lp - lm) / (2 * h) - g[v]) / np.abs(g).max())
    plan.close()
    rec["finite_differences_64cube"] = {"voxels": 64, "max_error_over_max_grad": worst, "precision": "fp64"}
    N, e = 32, fieldgen.unit_edges(8)
    d = fieldgen.field("lognormal", N, 9, np.float64)
    errs = {}
    for prec in ("fp64", "fp32", "split_bf16"):
        plan = ps.Plan(N, 500.0, 3, e, prec)
        w = np.random.default_rng(7).standard_normal(plan.nbins)
        if prec == "fp64":
            ref = oracle.gradient(d, 500.0, e, 3, plan.bins, plan.counts, w)
        dt = torch.from_numpy(d).cuda().to(plan.real_dtype)
        g = plan.backward(dt, torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)
        errs[prec] = float(np.abs(g - ref).max() / np.abs(ref).max())
        plan.close()
    rec["oracle_gradient_32cube"] = {"max_error_over_max_grad": errs, "shells": 8}
    return rec


def rows_f_record(ps, torch, np, peaks, fma, peak_src, flush_buf, delta_np, d):
    """SURVEY row (f) measurements beside the configurations: the redshift-space quadrupole (ell = 2) of the
    metric workload, split-BF16 and FP32, against the oracle on the triangles among five shells; and an
    order-5 plan whose counts need the integer closure maps (128^3, 20 unit shells)."""
    from types import SimpleNamespace

    import fieldgen
    import oracle

    rec = {}
    e = fieldgen.unit_edges(64)
    c3 = 5 * (L ** 3) ** 2 / float(256 ** 3) ** 3
    q = {"workload": "quadrupole (ell = 2, line of sight z) bispectrum, 256^3 lognormal field (seed 2), 64 unit "
                     "shells, n=3", "precisions": {}}
    sel_ref = None
    for prec, steps in (("split_bf16", 10), ("fp32", 3)):
        plan = ps.Plan(256, L, 3, e, prec, ell=2)
        code = plan.tune(d)[0] if prec == "split_bf16" else 0
        step_ms, stage, launches = time_precision(ps, torch, plan, d, SimpleNamespace(steps=steps, warmup=3),
                                                  flush_buf, False)
        B = time_precision.last_out
        if sel_ref is None:
            shells = {64, 40, 33, 17, 2}
            idx = np.array([i for i, b in enumerate(plan.bins) if set(b.tolist()) <= shells])
            sel_ref = (idx, oracle.estimate_ell(delta_np.astype(np.float64), L, e, 3, 2, plan.bins[idx]))
        idx, ref = sel_ref
        ms = statistics.median(step_ms)
        q["precisions"][prec] = {
            "ms_per_step": ms, "value": plan.nbins / (ms * 1e-3), "unit": "configs/s", "steps": steps, "warmup": 3,
            "stage_ms": stage, "gpu_launches": launches, "contraction_shape": code,
            "roofline": _contract_roofline(prec, plan.nbins * 256 ** 3 * 3, stage["ms_contract"], peaks, fma, peak_src),
            "error_vs_oracle": float(np.max(np.abs(B[idx] - ref["B"]) / (c3 * ref["scale"]))),
            "bins_checked": int(len(idx))}
        plan.close()
    rec["f3_quadrupole_256cube"] = q
    # order 5 at 128^3 with 20 unit shells: counts up to 1e13 come from the integer closure maps
    e5 = fieldgen.unit_edges(20)
    d5 = torch.from_numpy(fieldgen.field("lognormal", 128, 2, np.float32)).cuda()
    f2 = {"workload": "order-5 polyspectrum, 128^3 lognormal field (seed 2), 20 unit shells", "precisions": {},
          "note": "plan creation includes the integer closure-map counts (the FP64 counting-field sums cannot be "
                  "rounded safely at these counts); the first plan computes them, the second reuses them"}
    for prec in ("fp32", "split_bf16"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = ps.Plan(128, L, 5, e5, prec)
        torch.cuda.synchronize()
        plan_ms = (time.perf_counter() - t0) * 1e3
        code = plan.tune(d5)[0] if prec == "split_bf16" else 0
        step_ms, stage, launches = time_precision(ps, torch, plan, d5, SimpleNamespace(steps=3, warmup=3),
                                                  flush_buf, False)
        ms = statistics.median(step_ms)
        r = {"ms_per_step": ms, "value": plan.nbins / (ms * 1e-3), "unit": "configs/s", "stage_ms": stage,
             "plan_ms": plan_ms, "contraction_shape": code,
             "roofline": _contract_roofline(prec, plan.nbins * 128 ** 3 * 5, stage["ms_contract"], peaks, fma,
                                            peak_src)}
        if prec == "fp32":
            top = np.argsort(plan.counts)[-3:]
            ref = oracle.counts_exact(128, e5, 5, plan.bins[top])
            f2["nbins"] = plan.nbins
            f2["max_count"] = int(plan.counts.max())
            f2["counts_bit_exact_on_largest_3"] = bool(np.array_equal(plan.counts[top], ref))
            B32 = time_precision.last_out
        else:
            # split-BF16 against the FP32 path on every bin, in units of the FP32 estimate's scale
            sc = plan.estimate(d5, scale=True)[1].cpu().numpy()
            B16 = time_precision.last_out
            c5 = (L ** 3) ** 4 / float(128 ** 3) ** 5
            with np.errstate(invalid="ignore", divide="ignore"):
                rel = np.abs(B16 - B32) / (c5 * sc)
            r["max_diff_vs_fp32_over_scale"] = float(np.nanmax(rel[plan.counts > 0]))
        f2["precisions"][prec] = r
        plan.close()
    rec["f2_order5_128cube"] = f2
    return rec


def run_ours(args):
    import numpy as np
    import torch

    import fieldgen
    import paper_1904_11055_gb300 as ps
    from paper_1904_11055_gb300 import build as psbuild
    from paper_1904_11055_gb300 import sharding

    rank, world, local = sharding.rank_env()
    torch.cuda.set_device(local)
    dist_ok = world > 1
    if dist_ok:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not dist_ok:
        psbuild.build()
    if dist_ok:
        torch.distributed.barrier()
    peaks, peak_src = load_peaks()
    fma = {"f32": ps.diag_fma_peak(False), "f64": ps.diag_fma_peak(True)}  # measured CUDA-core peaks

    delta_np = fieldgen.field("lognormal", N, sharding.field_seed(SEED, rank), np.float32)
    d = torch.from_numpy(delta_np).cuda()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    edges = fieldgen.unit_edges(NSHELL, WIDTH)

    precisions = [args.precision] if args.precision != "auto" else ["split_bf16", "fp32"]
    results = {}
    for prec in precisions:
        try:
            torch.cuda.synchronize()
            t_plan = time.perf_counter()
            plan = ps.Plan(N, L, ORDER, edges, prec, ell=ELL)
            torch.cuda.synchronize()
            plan_ms = (time.perf_counter() - t_plan) * 1e3
        except ps.PolyError as e:
            if e.status == 6:
                results[prec] = {"unavailable": str(e)}
                continue
            raise
        # the contraction's launch shape, tuned once on this field (a user's plan.tune call; it reorders only
        # the final FP64 sums), outside the timed steps
        if prec == "split_bf16" and args.tc_config >= 0:
            plan.set_config(args.tc_config)  # a fixed shape (0: the plan's default), e.g. for profiling runs
            tuned = (args.tc_config, 0.0)
        else:
            tuned = plan.tune(d) if prec == "split_bf16" else (0, 0.0)
        step_ms, stage, launches = None, None, None
        with ClockSampler(local) as clk:
            step_ms, stage, launches = time_precision(ps, torch, plan, d, args, flush_buf, dist_ok)
        # every rank estimated its own field K times: units of all ranks over the slowest rank's time
        value = sharding.job_rate(plan.nbins * args.steps, sum(step_ms) / 1e3)
        total_ms = sharding.max_over_ranks(sum(step_ms))
        # end to end through the host-buffer entry point (pinned input, H2D + D2H every step)
        pinned = torch.from_numpy(delta_np).pin_memory().numpy()
        out_h = np.empty(plan.nbins)
        ps.poly_estimate_host(plan.handle, pinned, out_h, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ps.poly_estimate_host(plan.handle, pinned, out_h, None)
        e2e_s = time.perf_counter() - t0
        e2e_rate = sharding.job_rate(plan.nbins * args.steps, e2e_s)
        n3 = N ** 3
        useful_flops = plan.nbins * n3 * ORDER
        if prec == "split_bf16":
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            achieved = useful_flops / (stage["ms_contract"] * 1e-3) / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic_for("tc_contract", TC_SOURCES, workload_key(N, NSHELL, ORDER, WIDTH, ELL),
                                           tuned[0]),
                    "kernel": "tc_contract",
                    "peak_source": f"bf16 dense sustained, {peak_src}"}
        else:
            peak = fma["f32"]["tflops"]
            achieved = useful_flops / (stage["ms_contract"] * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic_for("contract_cc", CC_SOURCES, workload_key(N, NSHELL, ORDER, WIDTH, ELL, prec)),
                    "kernel": "contract_cc_kernel",
                    "peak_source": "FP32 FMA, measured by poly_diag_fma_peak in this run"}
        roof["executed_tflops"] = stage["contract_flops"] / (stage["ms_contract"] * 1e-3) / 1e12
        roof["useful_over_executed"] = useful_flops / stage["contract_flops"]
        field_bytes = NSHELL * n3 * 4 + n3 * 4
        fields_roof = {"bound": "hbm", "achieved": field_bytes / (stage["ms_fields"] * 1e-3) / 1e9,
                       "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": field_bytes / (stage["ms_fields"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                       "traffic": traffic_for("fields", FIELD_SOURCES, workload_key(N, NSHELL, ORDER, WIDTH, ELL)),
                       "kernel": "fields stage: xpass_kernel + inv_plane_kernel (8- and 16-warp launches), bytes per step",
                       "peak_source": peak_src}
        # the adjoint (dL/d delta for L = sum_b w_b B_b), device-timed, on this rank's field
        w = torch.from_numpy(np.random.default_rng(5).standard_normal(plan.nbins)).cuda()
        grad = torch.empty_like(d)
        bms = []
        if ORDER <= 4 and ELL == 0:  # the adjoint covers monopole plans of orders 2 to 4
            plan.backward(d, w, grad)
            torch.cuda.synchronize()
        for _ in range(3 if ORDER <= 4 and ELL == 0 else 0):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.backward(d, w, grad)
            b.record()
            torch.cuda.synchronize()
            bms.append(a.elapsed_time(b))
        cufft_ms = cufft_fields_ms(torch, d, edges) if prec == precisions[0] and ELL == 0 else None
        dms = []
        for _ in range(3 if ORDER == 4 and ELL == 0 else 0):  # the trispectrum's disconnected part (optional output)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.disconnected(d)
            b.record()
            torch.cuda.synchronize()
            dms.append(a.elapsed_time(b))
        results[prec] = {"value": value, "ms_per_step": total_ms / args.steps, "roofline": roof,
                         "disconnected_ms": statistics.median(dms) if dms else None, "cufft_fields_ms": cufft_ms,
                         "B": time_precision.last_out,
                         "plan_ms": plan_ms, "backward_ms": statistics.median(bms) if bms else None,
                         "tuned_config": {"code": tuned[0], "contract_ms": round(tuned[1], 4)},
                         "fields_roofline": fields_roof, "stage_ms": stage, "gpu_launches": launches,
                         "clocks": clk.summary(),
                         "e2e": {"value": e2e_rate, "unit": "configs/s",
                                 "h2d_bytes_per_step": n3 * 4, "d2h_bytes_per_step": plan.nbins * 8},
                         "nbins": plan.nbins}
        plan.close()
    if rank != 0:
        if dist_ok:
            torch.distributed.destroy_process_group()
        return
    head_prec = next((p for p in precisions if "value" in results.get(p, {})), None)
    if head_prec is None:
        print(json.dumps({"metric": METRIC, "error": "no precision available", "results": results}), flush=True)
        return
    h = results[head_prec]
    line = {
        "metric": METRIC, "value": h["value"], "unit": "configs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3" if head_prec == "split_bf16" else "f32", "data": "synthetic",
        "fields_per_s": 1e3 * world / h["ms_per_step"],
        "config": {"workload": WORKLOAD, "N": N, "N_max": NSHELL, "order": ORDER, "nbins": h["nbins"], "L": L,
                   "precision": head_prec, "l2": "256 MiB buffer written between timed steps (L2 flushed)",
                   "parallelism": f"replica per GPU x{world}" if world > 1 else "1 GPU",
                   "contraction_shape": h["tuned_config"]},
        "roofline": h["roofline"], "fields_roofline": h["fields_roofline"], "stage_ms": h["stage_ms"],
        "e2e": h["e2e"], "gpu_launches": h["gpu_launches"], "clocks": h["clocks"],
        "plan_ms": {"value": h["plan_ms"], "note": "plan creation with the FP64 counts (the first plan of the "
                    "process; later plans with the same shells reuse the cached counts); outside the timed step"},
        "backward_ms": {"value": h["backward_ms"], "note": "poly_backward, dL/d delta of sum_b w_b B_b on the same "
                        "field, device-timed median of 3"},
        "cufft_cross_check": {"fields_ms": h["cufft_fields_ms"], "library_fields_ms": h["stage_ms"]["ms_forward"] +
                              h["stage_ms"]["ms_fields"],
                              "note": "the same shell fields through cuFFT (torch.fft: full R2C, per-shell mask, full "
                                      "C2R), device-timed median of 3, against the library's forward + shell-field "
                                      "stages"},
        **({"disconnected_ms": {"value": h["disconnected_ms"], "note": "poly_trispectrum_disconnected on the same "
                                "field (forward transform, shell powers, per-bin pairings), device-timed median of 3"}}
           if ORDER == 4 and ELL == 0 else {}),
        "precisions": {p: ({k: r[k] for k in ("value", "ms_per_step", "roofline", "stage_ms", "e2e", "plan_ms",
                                              "backward_ms")}
                           if "value" in r else r) for p, r in results.items()},
    }
    if world == 1 and not args.no_cpu_baseline and (N, NSHELL, ORDER) == (256, 64, 3) and ELL == 0:
        line["cpu_baseline"], sel, ref = cpu_baseline(delta_np)
        # the error of every precision against the FP64 oracle on the same bins, in units of the tolerance scale
        # c_n sum_x |prod D| / (N^3 count) (bars: 1e-5 split-BF16, 1e-4 FP32)
        c_n = (L ** 3) ** (ORDER - 1) / float(N ** 3) ** ORDER
        line["error_vs_oracle"] = {
            p: float(np.max(np.abs(r["B"][sel] - ref["B"]) / (c_n * ref["scale"]))) for p, r in results.items()
            if "B" in r}
        line["error_vs_oracle"]["bins"] = int(len(sel))
    if world == 1 and not args.no_configs and (N, NSHELL, ORDER, WIDTH) == (256, 64, 3, 1.0) and ELL == 0:
        line["configs"] = {
            "1_bispectrum_64cube": config1_record(ps, torch, np, peaks, fma, peak_src, flush_buf),
            "3_trispectrum_256cube": config3_record(ps, torch, np, peaks, fma, peak_src, flush_buf, delta_np, d),
            "4_gradient": {"backward_ms_256cube": {p: r.get("backward_ms") for p, r in results.items()},
                           **config4_record(ps, torch, np)},
            "5_mocks": mocks_record(SimpleNamespace(steps=3, warmup=3)),
        }
        line["rows_f"] = rows_f_record(ps, torch, np, peaks, fma, peak_src, flush_buf, delta_np, d)
    line["fma_peak_measured"] = fma
    print(json.dumps(line), flush=True)
    if dist_ok:
        torch.distributed.destroy_process_group()


MOCKS = ((128, 256), (96, 128), (160, 128))  # (grid size, realisations)
MOCK_SHELLS = 32
MOCK_METRIC = ("mock realisations/s: 512 lognormal mocks (256 x 128^3, 128 x 96^3, 128 x 160^3), "
               "32 unit shells, bispectrum, split-BF16, one captured graph vs 512 sequential calls")


def run_mocks(args):
    """Batched mixed-size mocks: one poly_estimate_batched (captured graph) per step."""
    line = mocks_record(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def mocks_record(args):
    """The batched-mocks workload; returns the JSON record on rank 0 (None on other ranks)."""
    import numpy as np
    import torch

    import fieldgen
    import paper_1904_11055_gb300 as ps

    from paper_1904_11055_gb300 import sharding

    rank, world, local = sharding.rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    e = fieldgen.unit_edges(MOCK_SHELLS)
    plans = {n: ps.Plan(n, L, 3, e, "split_bf16", ps.POLY_ALLOW_ALIAS if 3 * MOCK_SHELLS >= n else 0)
             for n, _ in MOCKS}
    # 8 distinct seeded fields per size, one device buffer per realisation
    host = {n: [fieldgen.field("lognormal", n, 1000 + 8 * k + j, np.float32) for j in range(8)]
            for k, (n, _) in enumerate(MOCKS)}
    # this rank's share of each grid size's realisations (weak scaling: whole realisations per GPU)
    bplans, fields = [], []
    for n, count in MOCKS:
        a, b = sharding.unit_range(count, world, rank)
        for r in range(a, b):
            bplans.append(plans[n])
            fields.append(torch.from_numpy(host[n][r % 8]).cuda())
    outs = [torch.empty(p.nbins, dtype=torch.float64, device="cuda") for p in bplans]
    seq_outs = [torch.empty_like(o) for o in outs]
    tuned = {n: plans[n].tune(fields[[p.N for p in bplans].index(n)]) for n, _ in MOCKS}
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def sequential():
        for p, f, o in zip(bplans, fields, seq_outs):
            p.estimate(f, out=o)

    def batched():
        ps.estimate_batched(bplans, fields, outs)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ms = []
        for _ in range(args.steps):
            flush_buf.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    with ClockSampler(torch.cuda.current_device()) as clocks:
        if world > 1:
            torch.distributed.barrier()
        t_batch = timed(batched)
        t_seq = timed(sequential)
    identical = all(torch.equal(a, b) for a, b in zip(outs, seq_outs))
    # every rank ran its own share: realisations of all ranks over the slowest rank's step time
    rate_batch = sharding.job_rate(len(bplans), t_batch / 1e3)
    rate_seq = sharding.job_rate(len(bplans), t_seq / 1e3)
    identical = sharding.sum_over_ranks(0.0 if identical else 1.0) == 0.0
    t_batch, t_seq = sharding.max_over_ranks(t_batch), sharding.max_over_ranks(t_seq)
    if world > 1:
        torch.distributed.destroy_process_group()
    for p in plans.values():
        p.close()
    if rank != 0:
        return None
    line = {"metric": MOCK_METRIC, "value": rate_batch, "unit": "realisations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3",
            "data": "synthetic: 8 seeded lognormal fields per grid size (seeds 1000+), one device buffer per mock",
            "config": {"workload": "batched mocks", "mocks": {f"{n}^3": c for n, c in MOCKS}, "nshell": MOCK_SHELLS,
                       "order": 3, "bins": {f"{n}^3": plans[n].nbins for n, _ in MOCKS},
                       "l2": "256 MiB buffer written between timed steps (L2 flushed)",
                       "tuned_config": {f"{n}^3": {"code": c, "contract_ms": round(m, 4)} for n, (c, m) in tuned.items()}},
            "sequential": {"value": rate_seq, "ms_per_step": t_seq},
            "speedup_vs_sequential": t_seq / t_batch, "bit_identical_to_sequential": identical,
            "clocks": clocks.summary()}
    return line


FULL_K, FULL_NSHELL, FULL_WIDTH = (10, 10, 10, 10), 32, 1.5
FULL_METRIC = ("full-shape trispectrum quadrilaterals/s: bin (10,10,10,10) of 32 shells of width 1.5 k_F, 256^3, "
               "22 x 22 diagonal bins of width 1.5 k_F (Eq. Tkfull)")


def run_fullshape(args):
    """One full-shape trispectrum bin per step (poly_trispectrum_full on the trispectrum workload's shells)."""
    import numpy as np
    import torch

    import fieldgen
    import paper_1904_11055_gb300 as ps
    from paper_1904_11055_gb300 import build as psbuild

    psbuild.build()
    e = fieldgen.unit_edges(FULL_NSHELL, FULL_WIDTH)
    de = np.concatenate([[0.0], (np.arange(22) + 0.5) * FULL_WIDTH])
    K = 0
    while (K + 1) ** 2 < e[-1] ** 2:
        K += 1
    order = 4 if 4 * K < N else 2  # a smaller grid (profiling) takes a power-spectrum plan: same shells
    plan = ps.Plan(N, L, order, e, "split_bf16")
    delta_np = fieldgen.field("lognormal", N, SEED, np.float32)
    d = torch.from_numpy(delta_np).cuda()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}

    def step():
        out["T"], out["C"] = plan.trispectrum_full(d, FULL_K, de)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush_buf.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    quads = int(out["C"].sum().item())
    t = sum(ms) / 1e3
    match = np.flatnonzero((plan.bins == np.asarray(FULL_K)).all(axis=1)) if order == 4 else []
    line = {"metric": FULL_METRIC, "value": quads * args.steps / t, "unit": "quadrilaterals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"full-shape trispectrum, {N}^3 lognormal field (seed 2)", "bin": list(FULL_K),
                       "ndiag": int(len(de) - 1), "quadrilaterals_per_step": quads,
                       "l2": "256 MiB buffer written between timed steps (L2 flushed)"},
            "counts_sum_equals_count_b": bool(quads == plan.counts[match[0]]) if len(match) else None,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "split_bf16", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tc-config", type=int, default=-1,
                    help="split-BF16 contraction shape code instead of tuning (0: the plan's default)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the sub-records of the other workloads (64^3 FP64, trispectrum, gradient, mocks)")
    ap.add_argument("--N", type=int, default=N, help="grid size (default: the metric workload)")
    ap.add_argument("--nshell", type=int, default=NSHELL)
    ap.add_argument("--order", type=int, default=ORDER)
    ap.add_argument("--width", type=float, default=1.0, help="shell width in k_F (the trispectrum workload: 1.5)")
    ap.add_argument("--ell", type=int, default=0, help="redshift-space multipole of the first leg (even; FP32/FP64)")
    ap.add_argument("--workload", default="metric", choices=["metric", "mocks", "fullshape"],
                    help="mocks: 512 mixed-size realisations through poly_estimate_batched; fullshape: one bin of "
                         "the full-shape trispectrum")
    args = ap.parse_args()
    set_workload(args.N, args.nshell, args.order, args.width, args.ell)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mocks":
        run_mocks(args)
    elif args.workload == "fullshape":
        run_fullshape(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
