#!/usr/bin/env python
"""Benchmark of the FMM-LU hot path on one GB300 (or N replicas).

One step = the whole hot path on one synthetic input, through the C ABI:
fmmlu_build_tree + fmmlu_factor + fmmlu_solve + fmmlu_solve_adjoint on the
50,000-point ellipsoid (semi-axes 1, 2, 0.5; k = 2 pi; eps = 1e-6; complex128,
leaf 64, 300 proxy points). The metric is points per second of that step
(the paper's S = n / t, for factor plus both solves), higher is better.

Timing: W warm-up steps, then K steps, each preceded by an L2 flush (a 256 MiB
write) outside its CUDA-event window; barrier + synchronize on both sides;
max over ranks. Every kernel launch inside the timed steps is bracketed by
CUDA events on its stream (opts.profile = 1) to obtain the dominant kernel's
average launch duration for the roofline line. `e2e` repeats the step from
pinned host buffers with the host-to-device copies of the inputs and the
device-to-host copies of both solutions inside the timed region.

--impl reference times the CPU oracle (numpy/SciPy FP64) as it stands on this
machine's host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = ("factor s & solve ms vs N at eps 1e-6/1e-4, mixed+batched vs plain FP64 GPU, "
          "% roofline")
UNIT = "points/s"
FP64_PEAK_TFLOPS = 1.25     # GB300 dense FP64 (nominal table of the profiling recipe)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def sample_workload(name: str):
    spec = synth.WORKLOADS[name]
    return spec


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line.strip())
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def is_tensor_kernel(name: str) -> bool:
    """Kernels whose flops are bf16 tensor-core products (exact digit split)."""
    return name.endswith("_tc") or name == "gram"


def measured_peaks() -> dict:
    """Roofline denominators: the measured copy bandwidth and cuBLAS bf16 rate
    of this GPU type (MEASURED_PEAKS.json), else the profiling fallback."""
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {"hbm": (float(m["hbm_gbs"]), "of measured hbm_gbs"),
                "bf16_sustained": (float(m["bf16_tflops_sustained"]),
                                   "of measured bf16_tflops_sustained (kernel timed inside a long step)")}
    except Exception:
        return {"hbm": (6800.0, "of fallback (6.8 TB/s)"),
                "bf16_sustained": (1700.0, "of fallback (1.7 PFLOP/s sustained)")}


# translation unit (and its local headers) of each tensor-core kernel class
_KERNEL_FILES = {name: ("tcgemm.cu", "device_common.cuh", "fmmlu_internal.h")
                 for name in ("schur_tc", "gram", "gemm_g1_tc", "gemm_g3_tc", "gemm_w_tc",
                              "gemm_xrr_tc", "ns_tc", "root_w_tc", "root_schur_tc", "tc_split")}


def kernel_source_hash(kernel: str | None = None) -> str:
    """Hash of the sources a kernel is compiled from (all of csrc/ when the
    kernel is not in the table): recorded DRAM counters stay valid while it
    does not change."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2201_07325_gb300", "csrc")
    files = _KERNEL_FILES.get(kernel) or [f for f in os.listdir(d)
                                          if f.endswith((".cu", ".cuh", ".h"))]
    for f in sorted(files):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it still
    matches the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))
    except Exception:
        return None
    e = rec.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value of x over all ranks (the slowest replica's time);
    x itself when there is no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args, rank, world):
    import torch
    import paper_2201_07325_gb300 as pkg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    spec = synth.WORKLOADS[args.workload]
    k, eps = spec["k"], spec["eps"]
    surf = synth.make_surface(args.workload)
    b_np = synth.make_rhs(args.workload, surf)
    if b_np.ndim == 2:
        b_np = np.ascontiguousarray(b_np.T)          # (nrhs, n)
    nrhs = 1 if b_np.ndim == 1 else b_np.shape[0]
    n = surf.n
    pkg.load_library()
    precision = {"fp64": pkg.PRECISION_FP64, "mixed": pkg.PRECISION_MIXED,
                 "auto": pkg.PRECISION_AUTO}[args.precision]
    opts = pkg.fmmlu_default_opts(leaf_size=64, precision=precision, profile=1)
    pts = torch.from_numpy(surf.points).to(dev)
    nrm = torch.from_numpy(surf.normals).to(dev)
    wts = torch.from_numpy(surf.weights).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    x = torch.empty_like(b)
    y = torch.empty_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def one_step(handles, evs=None):
        if evs:
            evs[0].record(st)
        t = pkg.fmmlu_build_tree(pts, opts)
        if evs:
            evs[1].record(st)
        h = pkg.fmmlu_factor(t, pts, nrm, wts, k, eps, opts)
        pkg.fmmlu_free(t)
        if evs:
            evs[2].record(st)
        pkg.fmmlu_solve(h, b, x, n)
        if evs:
            evs[3].record(st)
        pkg.fmmlu_solve_adjoint(h, b, y, n)
        if evs:
            evs[4].record(st)
        handles.append(h)

    for _ in range(args.warmup):
        hs = []
        one_step(hs)
        for h in hs:
            pkg.fmmlu_free(h)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    comp = np.zeros(4)
    total_ms = 0.0
    launches0 = pkg.fmmlu_kernel_launches()
    kern = {}
    last_stats = None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        hs = []
        one_step(hs, evs)
        torch.cuda.synchronize()
        barrier()
        ts = [evs[i].elapsed_time(evs[i + 1]) for i in range(4)]
        comp += np.array(ts)
        total_ms += evs[0].elapsed_time(evs[4])
        last_stats = pkg.fmmlu_stats(hs[0])
        for name, e in last_stats["kernels"].items():
            acc = kern.setdefault(name, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
            for f in acc:
                acc[f] += e[f]
        keep_x = x.clone()
        for h in hs:
            pkg.fmmlu_free(h)
    launches = pkg.fmmlu_kernel_launches() - launches0
    clocks = sampler.stop()
    step_ms = max_over_ranks(total_ms / args.steps, dist, dev)
    value = n * world / (step_ms / 1e3)

    # residual of the last solution (dense on-the-fly product, outside timing)
    yv = torch.empty_like(keep_x)
    pkg.fmmlu_matvec(pts, nrm, wts, k, k, keep_x, yv)
    residual = float(torch.linalg.vector_norm(yv - b) / torch.linalg.vector_norm(b))

    # repeated solves with one factorization (the serving case): after the
    # first solve of each direction the sweeps replay as one CUDA graph
    opts_rep = pkg.fmmlu_default_opts(leaf_size=64, precision=precision)
    t = pkg.fmmlu_build_tree(pts, opts_rep)
    h = pkg.fmmlu_factor(t, pts, nrm, wts, k, eps, opts_rep)
    pkg.fmmlu_free(t)
    rep = {}
    for name, fn in (("solve", pkg.fmmlu_solve), ("adjoint", pkg.fmmlu_solve_adjoint)):
        for _ in range(3):
            fn(h, b, x, n)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(st)
        for _ in range(reps):
            fn(h, b, x, n)
        e1.record(st)
        torch.cuda.synchronize()
        rep[name] = e0.elapsed_time(e1) / reps
    pkg.fmmlu_free(h)

    # end to end from pinned host buffers
    hp = [torch.from_numpy(a).pin_memory() for a in (surf.points, surf.normals, surf.weights)]
    hb = torch.from_numpy(b_np).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    hy = torch.empty_like(hb).pin_memory()
    e2e_ms = 0.0
    opts_np = pkg.fmmlu_default_opts(leaf_size=64, precision=precision)
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dp, dn, dw = (a.to(dev, non_blocking=True) for a in hp)
        db = hb.to(dev, non_blocking=True)
        dx = torch.empty_like(db)
        dy = torch.empty_like(db)
        t = pkg.fmmlu_build_tree(dp, opts_np)
        h = pkg.fmmlu_factor(t, dp, dn, dw, k, eps, opts_np)
        pkg.fmmlu_free(t)
        pkg.fmmlu_solve(h, db, dx, n)
        pkg.fmmlu_solve_adjoint(h, db, dy, n)
        hx.copy_(dx, non_blocking=True)
        hy.copy_(dy, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        e2e_ms += e0.elapsed_time(e1)
        pkg.fmmlu_free(h)
    e2e_ms = max_over_ranks(e2e_ms / e2e_steps, dist, dev)
    h2d = sum(a.numel() * a.element_size() for a in hp) + hb.numel() * hb.element_size()
    d2h = 2 * hb.numel() * hb.element_size()

    # roofline of the dominant kernel over the timed region
    dom = max(kern.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    fp32_path = precision == pkg.PRECISION_MIXED or (precision == pkg.PRECISION_AUTO
                                                     and eps >= 1e-5)
    fp32_kernels = ({"cpqr", "assemble_id"} if fp32_path else set()) | {"xrr_inverse32"}
    peaks = measured_peaks()
    if is_tensor_kernel(dname):
        # exact-split products on the bf16 tensor cores: the bf16 flops of the
        # digit-pair products against the measured sustained bf16 rate
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        peak, src = peaks["bf16_sustained"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "kernel": dname, "peak_source": src}
    elif d["flops"] > 0:
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        peak = FP32_PEAK_TFLOPS if dname in fp32_kernels else FP64_PEAK_TFLOPS
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "kernel": dname,
                "peak_source": "fp32 FFMA units x clock" if dname in fp32_kernels
                else "nominal fp64 of the profiling recipe (1.25 TFLOP/s)"}
    else:
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
        peak, src = peaks["hbm"]
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak, "kernel": dname, "peak_source": src}
    tr = recorded_traffic(dname, args.workload)
    roof["traffic"] = tr
    roof["avg_launch_ms"] = d["ms"] / max(1, d["launches"])
    roof["launches"] = d["launches"]
    roof["share_of_step"] = d["ms"] / max(1e-9, total_ms)
    top = sorted(kern.items(), key=lambda kv: -kv[1]["ms"])[:8]

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not fp32_path else "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "k": k, "eps": eps,
                   "precision": args.precision, "nrhs": nrhs, "leaf_size": 64,
                   "n_proxy": 300, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "t_tree_ms": comp[0] / args.steps, "t_factor_s": comp[1] / args.steps / 1e3,
        "t_solve_ms": comp[2] / args.steps, "t_adjoint_ms": comp[3] / args.steps,
        "t_solve_repeat_ms": rep["solve"], "t_adjoint_repeat_ms": rep["adjoint"],
        "n0": last_stats["n0"], "factor_bytes": last_stats["factor_bytes"],
        "residual": residual,
        "e2e": {"value": n * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "top_kernels": {nm: {"ms_per_step": e["ms"] / args.steps,
                             "launches_per_step": e["launches"] / args.steps,
                             "tflops": (e["flops"] / (e["ms"] / 1e3) / 1e12) if e["ms"] else 0,
                             "unit": "bf16 TFLOP/s" if is_tensor_kernel(nm) else
                                     ("TFLOP/s" if e["flops"] else "GB/s"),
                             "gbs": (e["bytes"] / (e["ms"] / 1e3) / 1e9) if e["ms"] else 0}
                        for nm, e in top},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    if dist is not None:
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

SAMPLE_N = 2500


def oracle_step(workload: str, nsample: int = SAMPLE_N):
    """The oracle on a bounded sample of the workload: same surface family,
    k, eps, leaf size; N = nsample. Returns (seconds, points)."""
    from oracle import rss
    spec = synth.WORKLOADS[workload]
    surf = synth.make_surface(workload, nsample)
    b = synth.make_rhs(workload, surf)
    if b.ndim == 2:
        b = b[:, 0]
    t0 = time.perf_counter()
    F = rss.factor(surf.points, surf.normals, surf.weights, spec["k"], spec["eps"],
                   leaf_size=64)
    rss.solve(F, b)
    rss.solve_adjoint(F, b)
    return time.perf_counter() - t0, nsample


def single_core_oracle(workload: str, nsample: int = SAMPLE_N):
    """The oracle step in a child process limited to one thread (the paper's
    single-core setting); None when the child fails."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = ("import json, bench; s, p = bench.oracle_step(%r, %d); print(json.dumps([s, p]))"
            % (workload, nsample))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=300)
        sec, pts = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": pts / sec, "unit": UNIT, "cores": 1,
            "sample": f"oracle on {pts} points, one thread: {sec:.1f} s"}


def cpu_baseline(workload: str) -> dict:
    sec, pts = oracle_step(workload)
    out = {"value": pts / sec, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
           "sample": f"oracle (numpy/scipy fp64, dense current matrix) on {pts} points of "
                     f"the same surface family and k, eps, leaf 64: tree + factor + solve + "
                     f"adjoint in {sec:.1f} s"}
    one = single_core_oracle(workload)
    if one is not None:
        out["single_core"] = one
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_step(args.workload, 1200)
    tot, pts = 0.0, 0
    for _ in range(args.steps):
        s, p = oracle_step(args.workload, 1200)
        tot += s
        pts += p
    value = pts / tot
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_n": 1200,
                       "note": "CPU oracle on a bounded sample of the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle",
                             "sample": "oracle on 1200 points of the same surface family, "
                                       "k, eps, leaf 64 per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def factor_once(args) -> dict:
    """One tree + factorization of the workload (optionally at another size)
    with per-launch profiling on: the small case the ncu captures run."""
    import torch
    import paper_2201_07325_gb300 as pkg
    pkg.load_library()
    spec = synth.WORKLOADS[args.workload]
    s = synth.make_surface(args.workload, args.n)
    prec = {"fp64": pkg.PRECISION_FP64, "mixed": pkg.PRECISION_MIXED,
            "auto": pkg.PRECISION_AUTO}[args.precision]
    opts = pkg.fmmlu_default_opts(precision=prec, profile=1)
    pts, nrm, w = (torch.from_numpy(np.ascontiguousarray(a)).cuda()
                   for a in (s.points, s.normals, s.weights))
    t = pkg.fmmlu_build_tree(pts, opts)
    h = pkg.fmmlu_factor(t, pts, nrm, w, spec["k"], spec["eps"], opts)
    torch.cuda.synchronize()
    st = pkg.fmmlu_stats(h)
    pkg.fmmlu_free(h)
    pkg.fmmlu_free(t)
    return {"workload": args.workload, "n": s.n, "precision": args.precision, "n0": st["n0"],
            "kernels": st["kernels"]}


def scaling(args) -> list:
    """Factor and solve times against N on the ellipsoid (1, 2, 0.5) family
    at a fixed number of points per wavelength (k = 2 pi sqrt(N / 50,000),
    the regime of the paper's Table 2), plain fp64 at eps = 1e-6 and mixed at
    eps = 1e-4. Per size: one factorization to warm up (and tune), then one
    timed factorization; the solve is the mean of 5 graph replays after 3
    warm-up solves; residual by the dense on-the-fly product up to 100,000
    points."""
    import time
    import torch
    import paper_2201_07325_gb300 as pkg
    pkg.load_library()
    st = torch.cuda.current_stream()
    out = []
    sizes = [int(v) for v in args.sizes.split(",")]
    for prec_name, prec, eps in (("fp64", pkg.PRECISION_FP64, 1e-6),
                                 ("mixed", pkg.PRECISION_MIXED, 1e-4)):
        for n in sizes:
            s = synth.make_surface("ellipsoid50k", n)
            k = 2.0 * np.pi * float(np.sqrt(n / 50000.0))
            b = synth.make_rhs("ellipsoid50k", s, k)
            pts, nrm, w = (torch.from_numpy(np.ascontiguousarray(a)).cuda()
                           for a in (s.points, s.normals, s.weights))
            bt = torch.from_numpy(b).cuda()
            x = torch.empty_like(bt)
            opts = pkg.fmmlu_default_opts(precision=prec)
            for it in range(2):
                t = pkg.fmmlu_build_tree(pts, opts)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = pkg.fmmlu_factor(t, pts, nrm, w, k, eps, opts)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                pkg.fmmlu_free(t)
                if it == 0:
                    pkg.fmmlu_free(h)
            for _ in range(3):
                pkg.fmmlu_solve(h, bt, x, n)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(5):
                pkg.fmmlu_solve(h, bt, x, n)
            e1.record(st)
            torch.cuda.synchronize()
            stats = pkg.fmmlu_stats(h)
            row = {"n": n, "k": k, "precision": prec_name, "eps": eps,
                   "factor_s": t1 - t0, "solve_ms": e0.elapsed_time(e1) / 5,
                   "n0": stats["n0"], "factor_bytes": stats["factor_bytes"]}
            if n <= 100000:
                y = torch.empty_like(x)
                pkg.fmmlu_matvec(pts, nrm, w, k, k, x, y)
                row["residual"] = float(torch.linalg.vector_norm(y - bt)
                                        / torch.linalg.vector_norm(bt))
            pkg.fmmlu_free(h)
            print(json.dumps(row), flush=True)
            out.append(row)
            del pts, nrm, w, bt, x
            torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ellipsoid50k", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "auto"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--factor-once", action="store_true",
                    help="one profiled tree + factor of the workload (ncu captures); "
                         "prints the per-kernel algorithmic flops/bytes")
    ap.add_argument("--n", type=int, default=None,
                    help="with --factor-once: the same surface family at n points")
    ap.add_argument("--scaling", action="store_true",
                    help="factor and solve times against N (ellipsoid family, fixed points "
                         "per wavelength), one JSON line per size and precision")
    ap.add_argument("--sizes", default="12500,25000,50000,100000,200000,400000")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.factor_once:
        print(json.dumps(factor_once(args)))
        return
    if args.scaling:
        scaling(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
