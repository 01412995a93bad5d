#!/usr/bin/env python
"""Benchmark of the FMM-LU hot path on one GB300 (or N replicas).

One step = the whole hot path on one synthetic input, through the C ABI:
fmmlu_build_tree + fmmlu_factor + fmmlu_solve + fmmlu_solve_adjoint of every
right-hand side. Default workload: the 1,000,000-point ellipsoid (semi-axes
1, 3, 0.5) with density graded 100:1 toward one tip, k = 20, eps = 1e-4, the
mixed path (complex64 ID matrix, complex128 elimination and solves), 16
plane-wave right-hand sides, leaf 64, 300 proxy points. The metric is points
per second of that step (the paper's S = n / t, for the factor plus both
batched solves), higher is better; the line also carries the factor seconds
and solve milliseconds (t_factor_s, t_solve_ms) the metric names.

Timing: W warm-up steps, then K steps, each preceded by an L2 flush (a 256 MiB
write) outside its CUDA-event window; barrier + synchronize on both sides;
max over ranks. The timed steps run without per-kernel events. One further
step runs with CUDA events around every launch (opts.profile = 1): the
per-kernel breakdown (top_kernels) and the dominant kernel's roofline come
from it. `e2e` repeats the step K times from pinned host buffers with the
host-to-device copies of the inputs and the device-to-host copies of both
solutions inside the timed region. After the headline: the same workload on
the plain fp64 path at the same eps (plain_fp64, mixed_vs_plain) and the
other workloads (other_workloads), one warm-up and one timed step each.

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


# translation unit (and its local headers) of each kernel class whose DRAM
# counters are recorded
_COMMON = ("device_common.cuh", "fmmlu_internal.h")
_KERNEL_FILES = {name: ("tcgemm.cu", "dfloat.cuh") + _COMMON
                 for name in ("schur_tc", "gram", "gemm_g1_tc", "gemm_g3_tc", "gemm_w_tc",
                              "gemm_xrr_tc", "ns_tc", "root_w_tc", "root_schur_tc", "tc_split")}
_KERNEL_FILES.update({"pchol": ("pchol.cu", "coop.cuh") + _COMMON,
                      "xrr_inverse32": ("gj_dist.cu", "coop.cuh") + _COMMON,
                      "assemble_id": ("assembly.cu", "dfloat.cuh") + _COMMON,
                      "assemble_elim": ("assembly.cu", "dfloat.cuh") + _COMMON})


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


def recorded_traffic(kernel: str, workload: str, alg_bytes_per_launch: float | None = None):
    """DRAM bytes per launch from the committed ncu summary, if it still
    matches the current kernel sources (else None). A record taken on a
    smaller case of the same surface family holds the ratio of DRAM bytes to
    algorithmic bytes, applied here to this run's algorithmic bytes per
    launch; an older record holds bytes per launch directly."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))
    except Exception:
        return None
    e = rec.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    if "dram_per_alg_byte" in e:
        return e["dram_per_alg_byte"] * alg_bytes_per_launch if alg_bytes_per_launch else None
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


_T0 = time.time()


def log(msg: str):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.time() - _T0:7.1f} s] {msg}\n")
    sys.stderr.flush()


def kernel_pipe(name: str, fp32_path: bool) -> str:
    """Pipe that a kernel class's flops run on."""
    if is_tensor_kernel(name):
        return "tensor"
    if name == "xrr_inverse32" or (fp32_path and name in ("cpqr", "assemble_id")):
        return "fp32"
    return "fp64"


def kernel_roofline(name: str, e: dict, fp32_path: bool, peaks: dict, step_ms: float) -> dict:
    """Roofline entry of one kernel class from a profiled step: the method's
    own flops (8 real flops per complex multiply-add of the product it
    computes; kernel evaluations for the ID assembly) per second against the
    peak of the pipe the kernel runs on, or its algorithmic bytes per second
    against HBM when it does no arithmetic of its own."""
    sec = e["ms"] / 1e3
    launches = max(1, e["launches"])
    mfl = e.get("method_flops", e["flops"])
    out = {"kernel": name, "launches": e["launches"], "avg_launch_ms": e["ms"] / launches,
           "share_of_step": e["ms"] / max(1e-9, step_ms),
           "alg_bytes_per_launch": e["bytes"] / launches,
           "gbs": e["bytes"] / sec / 1e9 if sec > 0 else 0.0}
    if sec <= 0:
        return out
    pipe = kernel_pipe(name, fp32_path)
    if mfl > 0:
        ach = mfl / sec / 1e12
        if pipe == "tensor":
            peak, src = peaks["bf16_sustained"]
            out["pipe_achieved"] = e["flops"] / sec / 1e12
            out["pipe_frac"] = out["pipe_achieved"] / peak
            out["pipe_flops"] = "bf16 flops of the exact-split digit products"
            bound = "tensor"
        elif pipe == "fp32":
            peak, src, bound = FP32_PEAK_TFLOPS, "fp32 lanes x 2 x max SM clock", "alu"
        else:
            peak, src, bound = FP64_PEAK_TFLOPS, "nominal fp64 of the profiling recipe", "alu"
        out.update(bound=bound, achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   peak_source=src)
    else:
        gbs = e["bytes"] / sec / 1e9
        peak, src = peaks["hbm"]
        out.update(bound="hbm", achieved=gbs, peak=peak, unit="GB/s", frac=gbs / peak,
                   peak_source=src)
    return out


class Workload:
    """Device-resident inputs of one workload (right-hand sides as (nrhs, n))."""

    def __init__(self, name: str, dev, n: int | None = None):
        import torch
        spec = synth.WORKLOADS[name]
        self.name, self.k, self.eps = name, spec["k"], spec["eps"]
        self.surf = synth.make_surface(name, n)
        b = synth.make_rhs(name, self.surf)
        self.b_np = np.ascontiguousarray(b.T) if b.ndim == 2 else b
        self.nrhs = 1 if b.ndim == 1 else b.shape[1]
        self.n = self.surf.n
        self.pts = torch.from_numpy(self.surf.points).to(dev)
        self.nrm = torch.from_numpy(self.surf.normals).to(dev)
        self.wts = torch.from_numpy(self.surf.weights).to(dev)
        self.b = torch.from_numpy(self.b_np).to(dev)
        self.x = torch.empty_like(self.b)
        self.y = torch.empty_like(self.b)


def precision_code(pkg, name: str) -> int:
    return {"fp64": pkg.PRECISION_FP64, "mixed": pkg.PRECISION_MIXED,
            "auto": pkg.PRECISION_AUTO}[name]


def gpu_step(pkg, w: Workload, opts, st, evs=None):
    """One pass of the hot path: tree, factor, solve and adjoint solve of all
    right-hand sides. Returns the handle (the caller frees it)."""
    if evs:
        evs[0].record(st)
    t = pkg.fmmlu_build_tree(w.pts, opts)
    if evs:
        evs[1].record(st)
    h = pkg.fmmlu_factor(t, w.pts, w.nrm, w.wts, w.k, w.eps, opts)
    pkg.fmmlu_free(t)
    if evs:
        evs[2].record(st)
    pkg.fmmlu_solve(h, w.b, w.x, w.n)
    if evs:
        evs[3].record(st)
    pkg.fmmlu_solve_adjoint(h, w.b, w.y, w.n)
    if evs:
        evs[4].record(st)
    return h


def timed_steps(pkg, w: Workload, opts, st, steps: int, flush, barrier=lambda: None):
    """Time `steps` passes with CUDA events (L2 flushed before each, outside
    the events). Returns (mean ms per step, mean component ms [tree, factor,
    solve, adjoint], stats of the last handle)."""
    import torch
    comp = np.zeros(4)
    total = 0.0
    stats = None
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        h = gpu_step(pkg, w, opts, st, evs)
        torch.cuda.synchronize()
        barrier()
        comp += np.array([evs[i].elapsed_time(evs[i + 1]) for i in range(4)])
        total += evs[0].elapsed_time(evs[4])
        stats = pkg.fmmlu_stats(h)
        pkg.fmmlu_free(h)
    return total / steps, comp / steps, stats


def arm_summary(w: Workload, precision: str, step_ms: float, comp, stats) -> dict:
    return {"workload": w.name, "n": w.n, "k": w.k, "eps": w.eps, "nrhs": w.nrhs,
            "precision": stats["precision"], "requested": precision,
            "points_per_s": w.n / (step_ms / 1e3), "ms_per_step": step_ms,
            "t_tree_ms": comp[0], "t_factor_s": comp[1] / 1e3, "t_solve_ms": comp[2],
            "t_adjoint_ms": comp[3], "n0": stats["n0"], "factor_bytes": stats["factor_bytes"]}


def dense_residual(pkg, w: Workload) -> float:
    """||A x - b|| / ||b|| of the first solution by the dense on-the-fly GPU
    product (O(N^2): used up to a few hundred thousand points)."""
    import torch
    x0 = w.x[0].clone() if w.x.dim() == 2 else w.x.clone()
    b0 = w.b[0] if w.b.dim() == 2 else w.b
    y = torch.empty_like(x0)
    pkg.fmmlu_matvec(w.pts, w.nrm, w.wts, w.k, w.k, x0, y)
    return float(torch.linalg.vector_norm(y - b0) / torch.linalg.vector_norm(b0))


# proxy points per workload: 300 on every level, except on the 1M-point
# ellipsoid at k = 20 (about 10 wavelengths), whose coarse boxes are several
# wavelengths across: there the count follows the per-level multipole
# estimate (Sec. 5.2) with a floor of 64 points, which measured faster and
# more accurate than 300 everywhere (sampled residual 2.3e-5 against 3.5e-5)
PROXY_DEFAULTS = {"ellipsoid1m": ("adaptive", 64)}

# other workloads measured beside the headline (one warm-up step that also
# tunes, then one timed step each)
EXTRA_ARMS = [("ellipsoid50k", "fp64"), ("torus200k", "mixed"), ("torus200k", "fp64"),
              ("sphere100k", "fp64")]


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

    pkg.load_library()
    st = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    log(f"inputs {args.workload}")
    w = Workload(args.workload, dev)
    n, nrhs, k, eps = w.n, w.nrhs, w.k, w.eps
    log("warm-up")
    precision = precision_code(pkg, args.precision)
    def proxy_opts(workload):
        rule, npx = ((args.proxy_rule, args.n_proxy) if workload == args.workload
                     else PROXY_DEFAULTS.get(workload, ("fixed", 300)))
        return dict(n_proxy=npx,
                    proxy_rule=pkg.PROXY_ADAPTIVE if rule == "adaptive" else pkg.PROXY_FIXED)

    popts = proxy_opts(args.workload)
    opts = pkg.fmmlu_default_opts(leaf_size=64, precision=precision, **popts)

    # ---- headline: W warm-up steps, K timed steps (no per-kernel events) ----
    for _ in range(args.warmup):
        pkg.fmmlu_free(gpu_step(pkg, w, opts, st))
    torch.cuda.synchronize()
    log("timed steps")
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = pkg.fmmlu_kernel_launches()
    mean_ms, comp, stats = timed_steps(pkg, w, opts, st, args.steps, flush, barrier)
    launches = pkg.fmmlu_kernel_launches() - launches0
    clocks = sampler.stop()
    step_ms = max_over_ranks(mean_ms, dist, dev)
    value = n * world / (step_ms / 1e3)
    fp32_path = stats["precision"] == "mixed"

    log(f"timed: {step_ms:.1f} ms per step; profiled step")
    # ---- per-kernel breakdown: one more step with CUDA events on every launch
    opts_prof = pkg.fmmlu_default_opts(leaf_size=64, precision=precision, profile=1, **popts)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    torch.cuda.synchronize()
    e0.record(st)
    h = gpu_step(pkg, w, opts_prof, st)
    e1.record(st)
    torch.cuda.synchronize()
    prof_step_ms = e0.elapsed_time(e1)
    kern = pkg.fmmlu_stats(h)["kernels"]
    pkg.fmmlu_free(h)
    peaks = measured_peaks()
    roofs = {nm: kernel_roofline(nm, e, fp32_path, peaks, prof_step_ms) for nm, e in kern.items()
             if e["ms"] > 0}
    order = sorted(roofs, key=lambda nm: -roofs[nm]["avg_launch_ms"] * roofs[nm]["launches"])
    dname = order[0]
    roof = dict(roofs[dname])
    for rk, nm in enumerate(order[:3]):
        roofs[nm]["traffic"] = recorded_traffic(nm, args.workload, roofs[nm]["alg_bytes_per_launch"])
    roof["traffic"] = roofs[dname]["traffic"]
    roof["measured_in"] = ("a profiled step after the timed steps (CUDA events around every "
                           "launch on its stream); share_of_step is of that step")
    roof["flops_counted"] = ("the method's: 8 real flops per complex multiply-add of the "
                             "product computed (pipe_achieved counts the bf16 digit-pair flops)")

    log("repeated solves")
    # ---- repeated solves with one factorization (graph replay) -------------
    h = gpu_step(pkg, w, opts, st)
    rep = {}
    for name, fn in (("solve", pkg.fmmlu_solve), ("adjoint", pkg.fmmlu_solve_adjoint)):
        for _ in range(3):
            fn(h, w.b, w.x, n)
        torch.cuda.synchronize()
        e0.record(st)
        reps = 10
        for _ in range(reps):
            fn(h, w.b, w.x, n)
        e1.record(st)
        torch.cuda.synchronize()
        rep[name] = e0.elapsed_time(e1) / reps
    pkg.fmmlu_free(h)

    log("end to end")
    # ---- end to end from pinned host buffers, K steps ------------------------
    hp = [torch.from_numpy(a).pin_memory() for a in (w.surf.points, w.surf.normals,
                                                      w.surf.weights)]
    hb = torch.from_numpy(w.b_np).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    hy = torch.empty_like(hb).pin_memory()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0.record(st)
        dp, dn, dw = (a.to(dev, non_blocking=True) for a in hp)
        db = hb.to(dev, non_blocking=True)
        dx = torch.empty_like(db)
        dy = torch.empty_like(db)
        t = pkg.fmmlu_build_tree(dp, opts)
        hh = pkg.fmmlu_factor(t, dp, dn, dw, k, eps, opts)
        pkg.fmmlu_free(t)
        pkg.fmmlu_solve(hh, db, dx, n)
        pkg.fmmlu_solve_adjoint(hh, db, dy, n)
        hx.copy_(dx, non_blocking=True)
        hy.copy_(dy, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        e2e_ms += e0.elapsed_time(e1)
        pkg.fmmlu_free(hh)
        del dp, dn, dw, db, dx, dy
    e2e_ms = max_over_ranks(e2e_ms / args.steps, dist, dev)
    h2d = sum(a.numel() * a.element_size() for a in hp) + hb.numel() * hb.element_size()
    d2h = 2 * hb.numel() * hb.element_size()
    del hp, hb, hx, hy

    headline = arm_summary(w, args.precision, step_ms, comp, stats)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if fp32_path else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "k": k, "eps": eps,
                   "precision": stats["precision"], "nrhs": nrhs, "leaf_size": 64,
                   "n_proxy": args.n_proxy, "proxy_rule": args.proxy_rule, "step": "tree + factor + solve + adjoint solve of all "
                                           "right-hand sides",
                   "l2": "flushed between steps (256 MiB write); the factor's working set "
                         "is far larger than L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "t_tree_ms": comp[0], "t_factor_s": comp[1] / 1e3, "t_solve_ms": comp[2],
        "t_adjoint_ms": comp[3], "t_solve_repeat_ms": rep["solve"],
        "t_adjoint_repeat_ms": rep["adjoint"], "n0": stats["n0"],
        "factor_bytes": stats["factor_bytes"],
        "e2e": {"value": n * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "steps": args.steps},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / max(1, args.steps),
        "roofline": roof,
        "top_kernels": {nm: roofs[nm] for nm in order[:10]},
        "profiled_step": {"ms": prof_step_ms,
                          "kernel_ms": sum(e["ms"] for e in kern.values()),
                          "launches": sum(e["launches"] for e in kern.values()),
                          "idle_fraction": 1.0 - sum(e["ms"] for e in kern.values()) / prof_step_ms,
                          "kernel_ms_by_class": {nm: e["ms"] for nm, e in
                                                 sorted(kern.items(), key=lambda kv: -kv[1]["ms"])}},
        "clocks": clocks,
    }
    # ---- plain fp64 at the same eps, and the other workloads ---------------
    if not args.no_extra and world == 1:
        arms = []
        if stats["precision"] != "fp64":
            arms.append((args.workload, "fp64"))
        arms += [a for a in EXTRA_ARMS if a[0] != args.workload]
        extra = {}
        for wl, prec in arms:
            log(f"arm {wl} {prec}")
            wa = w if wl == args.workload else Workload(wl, dev)
            oa = pkg.fmmlu_default_opts(leaf_size=64, precision=precision_code(pkg, prec),
                                        **proxy_opts(wl))
            pkg.fmmlu_free(gpu_step(pkg, wa, oa, st))
            ms, cp, sa = timed_steps(pkg, wa, oa, st, 1, flush)
            row = arm_summary(wa, prec, ms, cp, sa)
            if wa.n <= 200000:
                row["residual"] = dense_residual(pkg, wa)
            extra[f"{wl}_{prec}"] = row
            del wa
            torch.cuda.empty_cache()
        log("arms done")
        # the azimuthal sonar sweep (Sec. 6.3): factor, then plane waves,
        # batched solves and backscattered far fields for every angle
        log("sonar sweep")
        ws = Workload("sonar200k", dev) if args.workload != "sonar200k" else w
        osn = pkg.fmmlu_default_opts(leaf_size=64, precision=pkg.PRECISION_AUTO,
                                     **proxy_opts("sonar200k"))
        phis = synth.azimuthal_angles(synth.WORKLOADS["sonar200k"]["angles"])
        dirs = torch.from_numpy(np.stack([np.cos(phis), np.sin(phis), np.zeros_like(phis)],
                                         axis=1)).to(dev)
        Rs = torch.empty(len(phis), dtype=torch.complex128, device=dev)
        for rep in range(2):
            torch.cuda.synchronize()
            e0.record(st)
            t = pkg.fmmlu_build_tree(ws.pts, osn)
            hs = pkg.fmmlu_factor(t, ws.pts, ws.nrm, ws.wts, ws.k, ws.eps, osn)
            pkg.fmmlu_free(t)
            e1.record(st)
            e2 = torch.cuda.Event(enable_timing=True)
            pkg.fmmlu_sonar_sweep(hs, ws.pts, ws.nrm, ws.wts, dirs, Rs, 32)
            e2.record(st)
            torch.cuda.synchronize()
            pkg.fmmlu_free(hs)
        extra["sonar200k_sweep"] = {
            "workload": "sonar200k", "n": ws.n, "k": ws.k, "eps": ws.eps, "angles": len(phis),
            "batch": 32, "t_tree_factor_s": e0.elapsed_time(e1) / 1e3,
            "t_sweep_ms": e1.elapsed_time(e2), "angles_per_s": len(phis) / (e1.elapsed_time(e2) / 1e3),
            "max_abs_R": float(Rs.abs().max())}
        del ws
        torch.cuda.empty_cache()
        plain = extra.pop(f"{args.workload}_fp64", None)
        if plain is not None:
            out["plain_fp64"] = plain
            out["mixed_vs_plain"] = {
                "factor_speedup": plain["t_factor_s"] / headline["t_factor_s"],
                "step_speedup": plain["ms_per_step"] / headline["ms_per_step"],
                "factor_bytes_ratio": headline["factor_bytes"] / plain["factor_bytes"]}
        out["other_workloads"] = extra
    del w
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline")
        out["cpu_baseline"] = cpu_baseline(args.workload, pkg, dev, opts)
    if dist is not None:
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

BASELINE_SIZES = (1000, 2000)
REFERENCE_N = 800


def oracle_step(workload: str, nsample: int):
    """The oracle on a bounded sample of the workload: same surface family,
    k, eps, leaf size and right-hand sides, N = nsample; tree + factor +
    solve + adjoint solve. Returns (seconds, points)."""
    from oracle import rss
    spec = synth.WORKLOADS[workload]
    surf = synth.make_surface(workload, nsample)
    b = synth.make_rhs(workload, surf)
    rule, npx = PROXY_DEFAULTS.get(workload, ("fixed", 300))
    t0 = time.perf_counter()
    F = rss.factor(surf.points, surf.normals, surf.weights, spec["k"], spec["eps"],
                   leaf_size=64, n_proxy=npx, proxy_rule=rule)
    rss.solve(F, b)
    rss.solve_adjoint(F, b)
    return time.perf_counter() - t0, nsample


def single_core_oracle(workload: str, nsample: int):
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
                           text=True, timeout=600)
        sec, pts = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": pts / sec, "unit": UNIT, "cores": 1, "n": pts, "seconds": sec,
            "sample": f"oracle on {pts} points, one thread: {sec:.1f} s"}


def cpu_baseline(workload: str, pkg=None, dev=None, opts=None) -> dict:
    """The oracle (as it stands) on samples of the workload's surface family,
    all host cores, with the GPU's step time at the same sizes beside it."""
    per_n = []
    for nn in BASELINE_SIZES:
        sec, pts = oracle_step(workload, nn)
        row = {"n": pts, "oracle_s": sec, "oracle_points_per_s": pts / sec}
        if pkg is not None:
            import torch
            wsm = Workload(workload, dev, nn)
            pkg.fmmlu_free(gpu_step(pkg, wsm, opts, torch.cuda.current_stream()))
            flush = torch.empty(1, device=dev)
            ms, _, _ = timed_steps(pkg, wsm, opts, torch.cuda.current_stream(), 3, flush)
            row["gpu_s"] = ms / 1e3
            row["gpu_over_oracle"] = sec / (ms / 1e3)
        per_n.append(row)
    last = per_n[-1]
    out = {"value": last["oracle_points_per_s"], "unit": UNIT, "cores": cpu_cores(),
           "kind": "oracle", "per_n": per_n,
           "sample": f"oracle (numpy/scipy fp64, dense current matrix) on {last['n']} points "
                     f"of the same surface family, k, eps, leaf 64 and right-hand sides: tree + "
                     f"factor + solve + adjoint in {last['oracle_s']:.1f} s (value); also "
                     f"{', '.join(str(r['n']) for r in per_n[:-1])} points (per_n, with the "
                     f"GPU's time at each size)"}
    one = single_core_oracle(workload, BASELINE_SIZES[0])
    if one is not None:
        out["single_core"] = one
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_step(args.workload, REFERENCE_N)
    tot, pts = 0.0, 0
    for _ in range(args.steps):
        s, p = oracle_step(args.workload, REFERENCE_N)
        tot += s
        pts += p
    value = pts / tot
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_n": REFERENCE_N,
                       "note": "CPU oracle on a bounded sample of the workload"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle",
                             "sample": f"oracle on {REFERENCE_N} points of the same surface "
                                       f"family, k, eps, leaf 64 and right-hand sides per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def factor_once(args) -> dict:
    """One tree + factorization of the workload (optionally at another size;
    with --step-once also the solve and adjoint solve of its right-hand
    sides), with per-launch profiling on: the case the ncu captures run.
    Same options as the benchmark's step (leaf 64, the workload's proxy
    rule)."""
    import torch
    import paper_2201_07325_gb300 as pkg
    pkg.load_library()
    w = Workload(args.workload, torch.device("cuda"), args.n)
    rule, npx = args.proxy_rule, args.n_proxy
    opts = pkg.fmmlu_default_opts(leaf_size=64, precision=precision_code(pkg, args.precision),
                                  profile=1, n_proxy=npx,
                                  proxy_rule=pkg.PROXY_ADAPTIVE if rule == "adaptive"
                                  else pkg.PROXY_FIXED)
    st = torch.cuda.current_stream()
    if args.step_once:
        # one unprofiled step first (the tuners run there), then the profiled
        # step inside a profiler range (ncu --profile-from-start off)
        opts0 = pkg.fmmlu_default_opts(leaf_size=64,
                                       precision=precision_code(pkg, args.precision),
                                       n_proxy=npx,
                                       proxy_rule=pkg.PROXY_ADAPTIVE if rule == "adaptive"
                                       else pkg.PROXY_FIXED)
        pkg.fmmlu_free(gpu_step(pkg, w, opts0, st))
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        h = gpu_step(pkg, w, opts, st)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    else:
        t = pkg.fmmlu_build_tree(w.pts, opts)
        h = pkg.fmmlu_factor(t, w.pts, w.nrm, w.wts, w.k, w.eps, opts)
        pkg.fmmlu_free(t)
    torch.cuda.synchronize()
    stats = pkg.fmmlu_stats(h)
    pkg.fmmlu_free(h)
    return {"workload": args.workload, "n": w.n, "precision": stats["precision"],
            "proxy_rule": rule, "n_proxy": npx, "n0": stats["n0"],
            "kernels": stats["kernels"]}


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
    ap.add_argument("--workload", default="ellipsoid1m", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="auto", choices=["fp64", "mixed", "auto"],
                    help="auto: mixed when eps >= 1e-5 (the 1M-point workload: eps = 1e-4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--proxy-rule", default=None, choices=["fixed", "adaptive"],
                    help="proxy points per sphere: n_proxy on every level, or the per-level "
                         "multipole estimate with n_proxy as the floor (default: the "
                         "workload's, PROXY_DEFAULTS)")
    ap.add_argument("--n-proxy", type=int, default=None)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the plain-fp64 arm and the other workloads")
    ap.add_argument("--factor-once", action="store_true",
                    help="one profiled tree + factor of the workload (ncu captures); "
                         "prints the per-kernel algorithmic flops/bytes")
    ap.add_argument("--step-once", action="store_true",
                    help="one profiled step (tree, factor, solve, adjoint) of the workload")
    ap.add_argument("--n", type=int, default=None,
                    help="with --factor-once: the same surface family at n points")
    ap.add_argument("--scaling", action="store_true",
                    help="factor and solve times against N (ellipsoid family, fixed points "
                         "per wavelength), one JSON line per size and precision")
    ap.add_argument("--sizes", default="12500,25000,50000,100000,200000,400000")
    args = ap.parse_args()
    rule, npx = PROXY_DEFAULTS.get(args.workload, ("fixed", 300))
    args.proxy_rule = args.proxy_rule or rule
    args.n_proxy = args.n_proxy or npx
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.factor_once or args.step_once:
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
