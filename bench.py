#!/usr/bin/env python
"""Benchmark of the multiple-scattering operator y = x - S (T + R) x and its solve.

Workload: 5000 dielectric discs (R = 0.25, kp = 2.4 pi) in the middle layer (d = 2) of the medium
k = (2 pi, 3 pi, 4 pi), p = 14 (29 coefficients per disc), 1024-node Sommerfeld contour, seeded
synthetic layout at ~20% area fraction.  A step is one operator application on one coefficient
vector already resident in device memory.  `value` is operator applications per second of the
mixed-precision operator (FP32 translation; the solve recovers FP64 accuracy by refinement), summed
over all ranks; the FP64 operator's rate, the solve times and the end-to-end rate through the
host-pointer C ABI are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 launch with torch.distributed.run: every rank runs an independent replica (the operator
of one layout does not shard without an exchange step), so scaling is weak.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import math
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "disc5000_p14_ns1024"
METRIC = "N=5000 solve time & operator applies/s, mixed/batched vs FP64 at <=1e-8 rel err"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12    # 152 SMs x 128 FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12      # 2 FP64 FMA per SM per clock on GB300


def _measured_peaks():
    """Measured copy bandwidth and cuBLAS BF16 throughput of this GPU pool, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 6800.0, "fallback"


BF16_PEAK_TFLOPS, HBM_PEAK_GBS, PEAK_SOURCE = _measured_peaks()
# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by the kernel's name and
# the SHA-256 of the source files it was built from (reported as null once they change).
TRAFFIC = {
    # k_translate_f32_sym<14>, 5000 discs: dram__bytes_read.sum 2.467 MB + dram__bytes_write.sum 0.068 MB
    # (profiles/translate_f32_sym_disc5000_p14_ns1024.md)
    "k_translate_f32_sym:ab0d5d3b92ae1b35": 2.5344e6,
}
KERNEL_SOURCES = ("mixed.cu", "ff_hankel.cuh")       # the FP32 translation kernels and their Hankel sequences
# the FP32 translation kernel of each tile shape (lsms_get_translation_tuning)
SHAPE_KERNEL = {0: "k_translate_f32_h2", 1: "k_translate_f32", 2: "k_translate_f32_sym"}


def translation_flop(n, p, nrhs=1):
    """Algorithmic FLOP of one all-pairs translation (Lemma 3.1): every ordered pair of distinct
    discs applies a P x P Toeplitz block to each right-hand side, 8 real flop per complex
    multiply-add."""
    P = 2 * p + 1
    return 8.0 * P * P * n * (n - 1) * nrhs


def fma_probe(fp64: bool) -> float:
    """Measured FMA TFLOP/s of this GPU (FP64 or FP32) from the benchmark's probe library
    libfmaprobe.so (built beside liblsms.so, outside its ABI)."""
    import ctypes

    from paper_1407_3868_gb300 import build as b
    lib = ctypes.CDLL(b.PROBE_LIB)
    lib.fma_probe_tflops.restype = ctypes.c_int
    lib.fma_probe_tflops.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    rc = lib.fma_probe_tflops(1 if fp64 else 0, ctypes.byref(v))
    if rc != 0:
        raise RuntimeError(f"fma_probe_tflops failed with CUDA error {rc}")
    return v.value


def max_over_ranks(vals, world, device):
    """Element-wise maximum of per-rank timings: the slowest replica sets the job's time."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processed units_per_rank in at most ms milliseconds."""
    return world * units_per_rank / (ms / 1e3)


def src_hash(paths) -> str:
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-solve", action="store_true", help="skip the solve timings")
    ap.add_argument("--no-fp64-solve", action="store_true", help="skip the FP64 solve (about 70 s)")
    ap.add_argument("--no-batched", action="store_true", help="skip the block and sweep measurements")
    ap.add_argument("--no-sweep", action="store_true", help="in the batched section, skip the 128-layout sweep")
    ap.add_argument("--full", action="store_true",
                    help="also solve the 64-source block and the 128-layout sweep (mixed, a few minutes)")
    ap.add_argument("--oracle-rows", type=int, default=2,
                    help="target rows per host core in each step of the reference arm (the oracle)")
    ap.add_argument("--baseline-rows", type=int, default=2,
                    help="target rows per host core in each pass of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing")
    ap.add_argument("--section", choices=["large", "example1", "translate", "batched"], default=None,
                    help="run one extra measurement alone and print its dict (for profiling); "
                         "translate: the mixed translation alone on --workload, --steps times")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# the oracle on every host core, on bounded samples of target rows
# ------------------------------------------------------------------------------------------------
def host_cpu() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform's name)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_workers() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_timing(workload: str, rows_per_worker: int, steps: int, warmup: int = 0,
                  workers: int | None = None) -> dict:
    """Time the oracle's operator application (`Problem.apply`, FP64 NumPy/SciPy) on every host core:
    a pool of worker processes (spawn, one BLAS thread each) splits the target particles, one chunk
    per worker.  A step is one pass over a bounded sample of rows_per_worker target rows per worker
    (rows spread over the layout); each worker also forms the global aggregate and per-node layer
    response once per pass, as a full application split the same way would.  Two calibration passes
    with one row per worker separate that global cost t_g from the cost per row t_r; a full
    application on the same pool takes t_g + ceil(N / workers) t_r."""
    import numpy as np

    from oracle import lsms_oracle as O
    from paper_1407_3868_gb300 import inputs
    w = inputs.WORKLOADS[workload]
    m = w.medium
    lam, wt = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    pr = O.Problem(O.Medium(m["k1"], m["k2"], m["k3"], m["d"], m["kp"], m["radius"]), w.p, w.centres(), lam, wt)
    x = inputs.random_coefficients(w.n, w.p, 1, 0)[0] / O.order_scale(w.p, m["k2"], m["radius"])
    workers = workers or host_workers()
    rows_per_worker = max(2, rows_per_worker)

    def spread(k):
        return sorted(set(np.linspace(0, w.n - 1, min(k, w.n)).astype(int).tolist()))

    with O.RowPool(pr, workers=workers) as rp:
        W = rp.workers
        one, sample = spread(W), spread(W * rows_per_worker)

        def timed_pass(rows):
            t0 = time.perf_counter()
            rp.apply(x, rows=rows, chunks=W)
            return time.perf_counter() - t0
        timed_pass(one)                                   # imports and first-touch in the workers
        t_one = min(timed_pass(one) for _ in range(2))
        for _ in range(warmup):
            timed_pass(sample)
        times = [timed_pass(sample) for _ in range(max(1, steps))]
    per_worker = len(sample) / W
    t_r = max(0.0, (statistics.mean(times) - t_one) / max(per_worker - len(one) / W, 1e-9))
    t_g = max(0.0, t_one - t_r * len(one) / W)
    full = t_g + math.ceil(w.n / W) * t_r
    return {"workers": W, "cpu": host_cpu(), "n": w.n, "rows_per_step": len(sample), "steps": len(times),
            "step_s": times, "t_global_s": t_g, "t_row_s": t_r, "full_apply_s": full}


def cpu_baseline_entry(s: dict) -> dict:
    return {"value": 1.0 / s["full_apply_s"], "unit": "applies/s", "cores": s["workers"], "kind": "oracle",
            "cpu": s["cpu"],
            "sample": (f"FP64 NumPy/SciPy oracle on {s['workers']} host cores ({s['cpu']}), one worker process "
                       f"per core: {s['steps']} passes over {s['rows_per_step']} of {s['n']} target rows "
                       f"({statistics.mean(s['step_s']):.2f} s each, incl. each worker's global aggregate and "
                       f"layer solves, {s['t_global_s']:.2f} s); one application = "
                       f"{s['t_global_s']:.2f} s + ceil({s['n']}/{s['workers']}) x {s['t_row_s']:.3f} s per "
                       f"row = {s['full_apply_s']:.1f} s")}


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# our implementation
# ------------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_3868_gb300 import inputs, lsms

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    # measured FMA ceilings of this GPU, beside the derived ALU peaks
    fma = {"fp32_tflops": fma_probe(False), "fp64_tflops": fma_probe(True),
           "probe": "libfmaprobe.so: 8 independent FMA chains per thread, 8 CTAs of 256 per SM"}
    w = inputs.WORKLOADS[args.workload]
    n, P = w.n, 2 * w.p + 1
    centres = w.centres()
    ctx = lsms.context_for(w, lsms.LSMS_MIXED)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    ctx.set_particles(centres)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    ctx.set_timing(True)
    b = torch.from_numpy(inputs.random_coefficients(n, w.p, 1, 100 + rank)).to(dev)
    y = torch.empty_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(flags, steps):
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        t_tr, launches = [], 0
        for i in range(steps):
            flush.fill_(float(i))
            e0[i].record(stream)
            ctx.apply_dev(b, y, flags, stream)
            e1[i].record(stream)
            ttr, _, launches = ctx.last_timing()       # waits for this step's events
            t_tr.append(ttr)
        torch.cuda.synchronize()
        ms = sum(e0[i].elapsed_time(e1[i]) for i in range(steps))
        return ms, t_tr, launches

    flags_mixed = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    flags_fp64 = lsms.APPLY_SCALED
    for _ in range(args.warmup):
        ctx.apply_dev(b, y, flags_mixed, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    ms_mixed, t_tr_mixed, launches = timed(flags_mixed, args.steps)
    shape = ctx.translation_tuning()[0]
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    # FP64 operator (fewer steps: ~0.2 s each)
    k64 = max(2, min(args.steps, 5))
    for _ in range(1):
        ctx.apply_dev(b, y, flags_fp64, stream)
    ms_fp64, t_tr_fp64, _ = timed(flags_fp64, k64)
    ms_mixed, ms_fp64 = max_over_ranks([ms_mixed, ms_fp64], world, dev)
    value = job_rate(args.steps, world, ms_mixed)
    fp64_rate = job_rate(k64, world, ms_fp64)

    # end to end through the host-pointer ABI: pinned host input, host output, copies inside
    xh = torch.from_numpy(inputs.random_coefficients(n, w.p, 1, 200 + rank)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xn, yn = xh.numpy(), yh.numpy()
    lib = lsms.load()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    for _ in range(2):
        lib.lsms_apply(ctx.h, 1, xn.ctypes.data_as(dp), yn.ctypes.data_as(dp))
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        rc = lib.lsms_apply(ctx.h, 1, xn.ctypes.data_as(dp), yn.ctypes.data_as(dp))
        assert rc == 0, rc
        _ = float(yn.real[0, 0, 0])
    e2e_s = time.perf_counter() - t0
    e2e = job_rate(args.steps, world, 1e3 * max_over_ranks([e2e_s], world, dev)[0])

    # roofline of the dominant kernel (the FP32 translation)
    flop = translation_flop(n, w.p)
    tr_ms = statistics.mean(t_tr_mixed)
    achieved = flop / (tr_ms / 1e3) / 1e12
    tr64_ms = statistics.mean(t_tr_fp64)
    key = src_hash([os.path.join(ROOT, "paper_1407_3868_gb300", "csrc", f) for f in KERNEL_SOURCES])
    traffic = TRAFFIC.get(SHAPE_KERNEL[shape] + ":" + key)

    solve = None
    u_ref_fp64 = None
    if not args.no_solve:
        # the mixed solve refines to 1e-8 (the refinement target of the mixed 5000-disc case) and,
        # for comparison, to 1e-10 (the FP64 solve's tolerance); fields are compared at the targets
        solve = {"mixed_tol": 1e-8, "fp64_tol": 1e-10, "set_particles_s": t_setup,
                 "timing": "wall clock around lsms_solve (create and set_particles excluded); mixed "
                           "at 1e-8: median of 3 after one warm-up solve"}
        u_m = {}
        for tol, key, reps in ((1e-8, "mixed", 3), (1e-8, "mixed_box_residual", 3), (1e-10, "mixed_tol1e-10", 1)):
            ctxm = lsms.context_for(w, lsms.LSMS_MIXED)
            ctxm.set_particles(centres)
            if key == "mixed_box_residual":
                # the FP64 refinement residual through boxes of width 4 (truncation ~1e-12); the
                # inner solves keep the all-pairs mixed operator
                ctxm.set_fmm(4.0)
                ctxm.set_fmm_scope(lsms.FMM_RESIDUAL)
            if reps > 1:
                ctxm.solve(w.sources, tol=tol, maxiter=2000)
            times = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info_m = ctxm.solve(w.sources, tol=tol, maxiter=2000)
                times.append(time.perf_counter() - t0)
            solve[key + "_s"] = statistics.median(times)
            if reps > 1:
                solve[key + "_s_all"] = times
            u_m[key] = ctxm.eval_field(w.targets, 0, lsms.FIELD_SCATTERED)
            solve[key + "_iters"] = info_m["iters"]
            solve[key + "_refinements"] = info_m["outer_iters"]
            solve[key + "_rel_res_fp64"] = info_m["rel_res_fp64"]
            ctxm.close()
        if not args.no_fp64_solve:
            ctxd = lsms.context_for(w, lsms.LSMS_FP64)
            ctxd.set_particles(centres)
            t0 = time.perf_counter()
            _, info_d = ctxd.solve(w.sources, tol=1e-10, maxiter=2000)
            solve["fp64_s"] = time.perf_counter() - t0
            solve["fp64_iters"] = info_d["iters"]
            solve["fp64_rel_res"] = info_d["rel_res_fp64"]
            u_d = ctxd.eval_field(w.targets, 0, lsms.FIELD_SCATTERED)
            u_ref_fp64 = u_d
            for key in u_m:
                solve[key + "_vs_fp64_field_rel_err"] = float(np.linalg.norm(u_m[key] - u_d) / np.linalg.norm(u_d))
            solve["speedup_mixed_vs_fp64"] = solve["fp64_s"] / solve["mixed_s"]
            ctxd.close()
    ctx.close()
    batched = stack = inclusions = contrast = large = boxes = example1 = None
    if world == 1 and not args.no_batched:
        # the further workloads, after the headline: a failure in one is reported in its own key
        # (and on stderr) without losing the headline line
        batched = guarded("batched", run_batched, args, dev, flush)
        stack = guarded("stack", run_stack, args, w, dev, flush)
        inclusions = guarded("inclusions", run_inclusions, args, w, dev, flush)
        contrast = guarded("contrast_sweep", run_contrast, args)
        large = guarded("large", run_large, args, dev, flush)
        boxes = guarded("boxes", run_boxes, args, w, dev, flush, u_ref_fp64)
        example1 = guarded("example1", run_example1, args)

    c2 = None
    if world == 1 and not args.no_solve:
        c2 = guarded("c2", run_c2, args)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "discs": n, "p": w.p, "contour_nodes": w.n_nodes,
                   "operator": "mixed (FP32 translation)", "nrhs": 1,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "batched": batched,
        "stack": stack,
        "inclusions": inclusions,
        "contrast_sweep": contrast,
        "large": large,
        "boxes": boxes,
        "example1": example1,
        "fma_probe": fma,
        "fp64": {"value": fp64_rate, "unit": "applies/s", "ms_per_step": ms_fp64 / k64, "dtype": "f64",
                 "translate_ms": tr64_ms,
                 "translate_frac_of_fp64_peak": (flop / (tr64_ms / 1e3) / 1e12) / FP64_PEAK_TFLOPS},
        "speedup_mixed_vs_fp64": value / fp64_rate,
        "roofline": {"kernel": SHAPE_KERNEL[shape], "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": traffic, "flop_per_launch": flop, "launch_ms": tr_ms,
                     "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "measured_fma_peak": fma["fp32_tflops"], "frac_of_measured_fma": achieved / fma["fp32_tflops"]},
        "e2e": {"value": e2e, "unit": "applies/s", "h2d_bytes_per_step": n * P * 16,
                "d2h_bytes_per_step": n * P * 16},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_entry(oracle_timing(w.name, args.baseline_rows, 2))
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    # the solve results last: the end of the line is what a truncated log keeps
    line["c2"] = c2
    line["solve"] = solve
    return line


def guarded(name, fn, *args):
    """fn(*args), or {"error": ...} (also printed to stderr) if it raises."""
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 - any failure of a further workload is reported, not raised
        msg = f"{type(e).__name__}: {e}"
        print(f"bench: section {name} failed: {msg}", file=sys.stderr)
        return {"error": msg[-500:]}


def time_device(fn, steps, flush=None):
    import torch
    ms = 0.0
    for i in range(steps):
        if flush is not None:
            flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    return ms / steps


GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "disc1000_p12_ns512_oracle.txt")


def load_oracle_solution(path=GOLDEN_C2):
    """The oracle's stored solution of the 1000-disc workload: (discs, beta rows, {field kind: values})."""
    import numpy as np
    beta, fields = {}, {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, a, b, *rest = line.split()
            if tag == "beta":
                beta[(int(a), int(b))] = complex(float(rest[0]), float(rest[1]))
            else:
                fields.setdefault(tag, {})[int(a)] = complex(float(b), float(rest[0]))
    discs = sorted({j for j, _ in beta})
    p = max(n for _, n in beta)
    B = np.array([[beta[(j, n)] for n in range(-p, p + 1)] for j in discs])
    return discs, B, {k: np.array([v[t] for t in sorted(v)]) for k, v in fields.items()}


def run_c2(args):
    """The plain FP64 GPU method on 1000 discs (p = 12, 512 contour nodes, tol 1e-10) and the mixed
    solve at 1e-8, each timed (one warm-up solve first) and compared with the oracle's solution of
    the same discrete problem (dense LU, stored in tests/golden): beta on every tenth disc in the
    scaled norm and the scattered and particle fields at the 64 targets, as 2-norm and element-wise
    relative errors."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    w = inputs.WORKLOADS["disc1000_p12_ns512"]
    discs, B, U = load_oracle_solution()
    from scipy import special
    hs = np.abs(special.hankel1(np.arange(-w.p, w.p + 1), w.medium["k2"] * w.medium["radius"]))   # scaled norm
    out = {"workload": w.name, "discs": w.n, "p": w.p, "contour_nodes": w.n_nodes,
           "oracle": "stored dense-LU solution (tests/golden), scaled residual 2.6e-14"}
    for prec, key, tol in ((lsms.LSMS_FP64, "fp64_solve", 1e-10), (lsms.LSMS_MIXED, "mixed_solve", 1e-8)):
        ctx = lsms.context_for(w, prec)
        ctx.set_particles(w.centres())
        ctx.solve(w.sources, tol=tol, maxiter=2000)                       # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        beta, info = ctx.solve(w.sources, tol=tol, maxiter=2000)
        t = time.perf_counter() - t0
        got = beta[0][discs]
        wgt = hs
        row = {"tol": tol, "s": t, "iters": info["iters"], "refinements": info["outer_iters"],
               "rel_res_fp64": info["rel_res_fp64"],
               "beta_rel_err": float(np.linalg.norm((got - B) * wgt) / np.linalg.norm(B * wgt)),
               "beta_max_err": float(np.max(np.abs((got - B) * wgt)) / np.max(np.abs(B * wgt)))}
        for kind, which in (("scattered", lsms.FIELD_SCATTERED), ("particle", lsms.FIELD_PARTICLE)):
            u = ctx.eval_field(w.targets, 0, which)
            row[kind + "_field_rel_err"] = float(np.linalg.norm(u - U[kind]) / np.linalg.norm(U[kind]))
            row[kind + "_field_max_err"] = float(np.max(np.abs(u - U[kind])) / np.max(np.abs(U[kind])))
        out[key] = row
        ctx.close()
    out["speedup_mixed_vs_fp64"] = out["fp64_solve"]["s"] / out["mixed_solve"]["s"]
    # the oracle-size configuration (16 discs, p = 10, 256 nodes, tol 1e-12): a solve of a few dozen
    # small Arnoldi steps, where the GMRES iteration's graph-resident loop matters
    w1 = inputs.WORKLOADS["disc16_p10_ns256"]
    ctx = lsms.context_for(w1, lsms.LSMS_FP64)
    ctx.set_particles(w1.centres())
    ctx.solve(w1.sources, tol=1e-12, maxiter=500)                         # warm-up
    ts = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = ctx.solve(w1.sources, tol=1e-12, maxiter=500)
        ts.append(time.perf_counter() - t0)
    ctx.close()
    out["c1_fp64_solve"] = {"workload": w1.name, "discs": w1.n, "tol": 1e-12, "s": statistics.median(ts),
                            "iters": info["iters"], "timing": "wall clock around lsms_solve, median of 5"}
    return out


def run_batched(args, dev, flush):
    """Batched forms: 64 sources on one 2000-disc layout (block of right-hand sides) and a design
    sweep of 128 layouts (log-uniform N in [200, 4000]) applied as one graph launch."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    out = {}
    # block of right-hand sides
    w = inputs.WORKLOADS["disc2000_p12_ns768_src64"]
    ctx = lsms.context_for(w, lsms.LSMS_MIXED)
    ctx.set_particles(w.centres())
    nrhs = len(w.sources)
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, nrhs, 0)).to(dev)
    y = torch.empty_like(x)
    fl_m = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    P = 2 * w.p + 1
    flop = translation_flop(w.n, w.p, nrhs)
    blk = {"workload": w.name, "discs": w.n, "p": w.p, "contour_nodes": w.n_nodes, "rhs": nrhs}
    for tcmin, key in ((48, "mixed"), (0, "mixed_cuda_cores")):
        ctx.set_tc_translation(tcmin)
        ctx.apply_dev(x, y, fl_m)
        torch.cuda.synchronize()
        ms_m = time_device(lambda: ctx.apply_dev(x, y, fl_m), 5, flush)
        ctx.set_timing(1)
        tr = []
        for _ in range(3):
            ctx.apply_dev(x, y, fl_m)
            tr.append(ctx.last_timing()[0])
        ctx.set_timing(0)
        tr_ms = statistics.mean(tr)
        blk[key] = {"ms_per_block_apply": ms_m, "rhs_applies_per_s": nrhs * 1e3 / ms_m,
                    "translate_ms": tr_ms, "translate_tflops_algorithmic": flop / (tr_ms / 1e3) / 1e12,
                    "translation": "tensor cores (split-BF16 tcgen05)" if tcmin else "FP32 CUDA cores"}
    ctx.set_tc_translation(48)
    ctx.apply_dev(x, y, lsms.APPLY_SCALED)
    torch.cuda.synchronize()
    ms_d = time_device(lambda: ctx.apply_dev(x, y, lsms.APPLY_SCALED), 1, flush)
    blk["fp64"] = {"ms_per_block_apply": ms_d, "rhs_applies_per_s": nrhs * 1e3 / ms_d}
    blk["speedup_mixed_vs_fp64"] = ms_d / blk["mixed"]["ms_per_block_apply"]
    # the tensor-core translation: algorithmic flops against the measured BF16 peak, and the MMA
    # work it issues (six BF16 plane products on the real embedding: per step two 128 x 128 tiles
    # with K = 2P padded to 64, a group of 2 floor(128 / P) targets against one source)
    tg = 2 * (128 // P)
    ngroups = (w.n + tg - 1) // tg
    issued = 2.0 * 6 * 2 * 128 * 128 * 64 * ngroups * w.n * ((nrhs + 63) // 64)
    tms = blk["mixed"]["translate_ms"]
    blk["roofline"] = {"kernel": "k_translate_tc", "bound": "tensor", "achieved": flop / (tms / 1e3) / 1e12,
                       "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": flop / (tms / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
                       "issued_tensor_tflops": issued / (tms / 1e3) / 1e12,
                       "issued_frac": issued / (tms / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
                       "peak_note": f"{PEAK_SOURCE} cuBLAS BF16 burst"}
    if not args.no_solve:
        for tol, key in ((1e-8, "mixed_solve"), (1e-10, "mixed_solve_tol1e-10")):
            if tol < 1e-8 and not args.full:
                continue
            t0 = time.perf_counter()
            _, info = ctx.solve(w.sources, tol=tol, maxiter=1000)
            blk[key] = {"tol": tol, "s": time.perf_counter() - t0, "iters": info["iters"],
                        "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
    ctx.close()
    out["block_rhs"] = blk
    if args.no_sweep:
        return out
    # design sweep over 128 layouts
    lay = inputs.sweep_layouts()
    h = inputs.widened_half_width(max(len(c) for c in lay))
    ws = inputs.Workload("sweep128_p12_ns512", 0, 12, 512, 152.0, -h, h, 0, np.array([[0.0, 1.0]]),
                         inputs.observation_points(-h, h, 64, 1.5), 1e-10)
    b = lsms.context_for(ws, lsms.LSMS_MIXED)
    b.set_layouts(lay)
    tuning = b.autotune()
    ntot = sum(len(c) for c in lay)
    x = torch.from_numpy(inputs.random_coefficients(ntot, ws.p, 1, 0)[0]).to(dev)
    y = torch.empty_like(x)
    for _ in range(2):
        b.apply_dev(x, y, fl_m)
    torch.cuda.synchronize()
    ms_m = time_device(lambda: b.apply_dev(x, y, fl_m), 5, flush)
    for _ in range(2):
        b.apply_dev(x, y, lsms.APPLY_SCALED)
    torch.cuda.synchronize()
    ms_d = time_device(lambda: b.apply_dev(x, y, lsms.APPLY_SCALED), 1, flush)
    waves, items = b.batch_translation()
    sweep_flop = sum(translation_flop(len(c), ws.p) for c in lay)
    sw = {"workload": ws.name, "layouts": len(lay), "discs": ntot, "p": ws.p, "contour_nodes": ws.n_nodes,
          "autotuned": {"layouts_two_lane_tiles": sum(1 for sh, _ in tuning if sh == 0),
                        "layouts_four_lane_tiles": sum(1 for sh, _ in tuning if sh == 1),
                        "layouts_unordered_pair_tiles": sum(1 for sh, _ in tuning if sh == 2),
                        "split_mults": sorted({m for _, m in tuning}),
                        "batched_translation": {"waves": waves, "work_items": items}},
          "mixed": {"ms_per_sweep_apply": ms_m, "layout_applies_per_s": len(lay) * 1e3 / ms_m,
                    "launch": "one CUDA graph: the layouts' translations in one kernel launch (work items "
                              "largest layout first), their reflected couplings in 128 branches",
                    "translation_flop": sweep_flop,
                    "apply_frac_of_fp32_peak": sweep_flop / (ms_m / 1e3) / 1e12 / FP32_PEAK_TFLOPS},
          "fp64": {"ms_per_sweep_apply": ms_d, "layout_applies_per_s": len(lay) * 1e3 / ms_d}}
    sw["speedup_mixed_vs_fp64"] = ms_d / ms_m
    if not args.no_solve:
        t0 = time.perf_counter()
        _, info = b.solve(ws.sources, tol=1e-8, maxiter=1000)
        sw["mixed_solve"] = {"tol": 1e-8, "s": time.perf_counter() - t0, "iters_max": info["iters"],
                             "refinements_max": info["outer_iters"],
                             "rel_res_fp64_max": info["rel_res_fp64"]}
    b.close()
    out["sweep"] = sw
    return out


def run_stack(args, w, dev, flush):
    """The bench layout in a five-layer medium (discs in layer 3): mixed operator applications and
    the mixed solve at 1e-8.  Only the per-node layer response differs from the three-layer run."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    st, m = inputs.STACK5, w.medium
    ctx = lsms.Context(0, 0, 0, 0, m["kp"], m["radius"], w.p, w.n_nodes, b=w.b, t_max=w.t_max,
                       panel_order=16, precision=lsms.LSMS_MIXED, stack=(st["ks"], st["ds"], st["layer"]))
    centres = w.centres() - np.array([0.0, inputs.STACK5_DEPTH])
    ctx.set_particles(centres)
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, 1, 300)).to(dev)
    y = torch.empty_like(x)
    fl_m = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    for _ in range(3):
        ctx.apply_dev(x, y, fl_m)
    torch.cuda.synchronize()
    ms = time_device(lambda: ctx.apply_dev(x, y, fl_m), max(args.steps, 3), flush)
    out = {"workload": w.name + "_stack5", "wavenumbers": st["ks"], "thicknesses": st["ds"],
           "particle_layer": st["layer"], "mixed": {"ms_per_apply": ms, "applies_per_s": 1e3 / ms}}
    if not args.no_solve:
        t0 = time.perf_counter()
        _, info = ctx.solve(w.sources, tol=1e-8, maxiter=2000)      # sources stay in layer 1
        out["mixed_solve"] = {"tol": 1e-8, "s": time.perf_counter() - t0, "iters": info["iters"],
                              "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
    ctx.close()
    return out


def run_inclusions(args, w, dev, flush):
    """The bench layout with five-lobed star inclusions (Sec. 4; Sec. 6 Eq. "par1"), each turned
    by a seeded angle: the prototype's scattering matrix from the host Nystrom solve, then mixed
    operator applications and the mixed solve at 1e-8 with the rotated dense matrices."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    s, m = inputs.STAR5, w.medium
    t0 = time.perf_counter()
    smat = lsms.inclusion_scattering_matrix(w.p, m["k2"], m["kp"], m["radius"],
                                            inputs.star_curve(s["a1"], s["a2"], s["a3"], s["n_pts"]))
    t_matrix = time.perf_counter() - t0
    ctx = lsms.context_for(w, lsms.LSMS_MIXED)
    ctx.set_particles(w.centres())
    ctx.set_scattering_matrix(smat)
    ctx.set_orientations(inputs.orientations(w.n, 7))
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, 1, 400)).to(dev)
    y = torch.empty_like(x)
    fl_m = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    for _ in range(3):
        ctx.apply_dev(x, y, fl_m)
    torch.cuda.synchronize()
    ms = time_device(lambda: ctx.apply_dev(x, y, fl_m), max(args.steps, 3), flush)
    out = {"workload": w.name + "_star5", "shape": dict(s), "matrix_setup_s": t_matrix,
           "mixed": {"ms_per_apply": ms, "applies_per_s": 1e3 / ms}}
    if not args.no_solve:
        t0 = time.perf_counter()
        _, info = ctx.solve(w.sources, tol=1e-8, maxiter=2000)
        out["mixed_solve"] = {"tol": 1e-8, "s": time.perf_counter() - t0, "iters": info["iters"],
                              "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
        # the same stars with a lossy interior, k_p (1 + 0.3i) (complex k_p in Muller's system)
        kp_abs = m["kp"] * (1 + 0.3j)
        t0 = time.perf_counter()
        smat_abs = lsms.inclusion_scattering_matrix(w.p, m["k2"], kp_abs, m["radius"],
                                                    inputs.star_curve(s["a1"], s["a2"], s["a3"], s["n_pts"]))
        t_abs = time.perf_counter() - t0
        ctx.set_scattering_matrix(smat_abs)
        t0 = time.perf_counter()
        _, info = ctx.solve(w.sources, tol=1e-8, maxiter=2000)
        out["absorbing_mixed_solve"] = {"kp": [kp_abs.real, kp_abs.imag], "matrix_setup_s": t_abs, "tol": 1e-8,
                                        "s": time.perf_counter() - t0, "iters": info["iters"],
                                        "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
    ctx.close()
    return out


def run_contrast(args):
    """Contrast sweep (Sec. 6, Example 2): 200 rotated three-lobed inclusions in a layer of
    thickness 12 between half-spaces of k = 1, the layer's k2 from 1 to 20 (guided-mode media for
    k2 > 1), FP64 GMRES to 1e-6 for each k2.  Per k2: context and layout setup, the inclusion's
    scattering matrix (host), the solve; the sweep total."""
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    cfg = inputs.CONTRAST
    sh = cfg["shape"]
    centres = inputs.contrast_layout()
    theta = inputs.orientations(cfg["n"], 22)
    curve = inputs.star_curve(sh["a1"], sh["a2"], sh["a3"], sh["n_pts"])
    b = inputs.contour_b(cfg["x_hi"] - cfg["x_lo"])
    rows = []
    t_all = time.perf_counter()
    for k2 in cfg["k2_values"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = lsms.Context(cfg["k1"], k2, cfg["k3"], cfg["d"], cfg["kp"], cfg["radius"], cfg["p"],
                           cfg["n_nodes"], b=b, t_max=inputs.contrast_t_max(k2), panel_order=16,
                           precision=lsms.LSMS_FP64)
        ctx.set_particles(centres)
        t1 = time.perf_counter()
        smat = lsms.inclusion_scattering_matrix(cfg["p"], k2, cfg["kp"], cfg["radius"], curve)
        ctx.set_scattering_matrix(smat)
        ctx.set_orientations(theta)
        t2 = time.perf_counter()
        _, info = ctx.solve([[0.0, 1.0]], tol=cfg["tol"], maxiter=3000, raise_on_error=False)
        t3 = time.perf_counter()
        ctx.close()
        rows.append({"k2": k2, "setup_s": t1 - t0, "matrix_s": t2 - t1, "solve_s": t3 - t2,
                     "iters": info["iters"], "rel_res": info["rel_res_fp64"], "status": info["status"]})
    return {"workload": "contrast200_p10_ns2048", "inclusions": cfg["n"], "p": cfg["p"],
            "contour_nodes": cfg["n_nodes"], "tol": cfg["tol"], "precision": "fp64",
            "total_s": time.perf_counter() - t_all, "per_k2": rows}


def run_boxes(args, w, dev, flush, u_ref=None):
    """The bench layout with the translation through boxes (width 4, 614 boxes): mixed and FP64
    operator applications, the mixed solve at 1e-8 and the FP64 solve at 1e-10, and the scattered
    field against the all-pairs FP64 solve (u_ref)."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    out = {"workload": w.name + "_boxes", "box_width": 4.0}
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, 1, 600)).to(dev)
    y = torch.empty_like(x)
    fl_m = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    for prec, key, flags, tol in ((lsms.LSMS_MIXED, "mixed", fl_m, 1e-8),
                                  (lsms.LSMS_FP64, "fp64", lsms.APPLY_SCALED, 1e-10)):
        ctx = lsms.context_for(w, prec)
        ctx.set_particles(w.centres())
        ctx.set_fmm(4.0)
        out["boxes"], out["order"] = ctx.fmm_info()
        for _ in range(3):
            ctx.apply_dev(x, y, flags)
        torch.cuda.synchronize()
        ms = time_device(lambda: ctx.apply_dev(x, y, flags), max(3, min(args.steps, 10)), flush)
        row = {"ms_per_apply": ms, "applies_per_s": 1e3 / ms}
        if not args.no_solve:
            if prec == lsms.LSMS_MIXED:
                ctx.solve(w.sources, tol=tol, maxiter=2000)          # warm-up (graphs, workspaces)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = ctx.solve(w.sources, tol=tol, maxiter=2000, raise_on_error=False)
            row["solve"] = {"tol": tol, "s": time.perf_counter() - t0, "iters": info["iters"],
                            "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"],
                            "status": info["status"]}
            if u_ref is not None:
                u = ctx.eval_field(w.targets, 0, lsms.FIELD_SCATTERED)
                row["solve"]["field_rel_err_vs_all_pairs_fp64"] = float(np.linalg.norm(u - u_ref) /
                                                                        np.linalg.norm(u_ref))
        out[key] = row
        ctx.close()
    return out


def run_example1(args):
    """Sec. 6 Example 1's configuration: 5000 rotated three-lobed inclusions, k = (1, 3, 1), a layer 32
    thick (a guided-mode layer), kp = 2, p = 10, 2048 contour nodes; the mixed solve to 1e-6 (the
    paper's tolerance; its serial CPU code with FMM needed 127 s on a laptop, context only)."""
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    e = inputs.EXAMPLE1
    sh = e["shape"]
    curve = inputs.star_curve(sh["a1"], sh["a2"], sh["a3"], sh["n_pts"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = lsms.Context(e["k1"], e["k2"], e["k3"], e["d"], e["kp"], e["radius"], e["p"], e["n_nodes"],
                       b=inputs.contour_b(e["x_hi"] - e["x_lo"]), t_max=e["t_max"], panel_order=16,
                       precision=lsms.LSMS_MIXED)
    ctx.set_particles(inputs.example1_layout())
    ctx.set_scattering_matrix(lsms.inclusion_scattering_matrix(e["p"], e["k2"], e["kp"], e["radius"], curve))
    ctx.set_orientations(inputs.orientations(e["n"], 32))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = {"workload": "example1_star5000_p10_ns2048", "setup_s": t_setup,
           "paper_context": "Sec. 6 Example 1: 127 s to 6 digits on a 2.3 GHz laptop (serial, FMM)"}
    if not args.no_solve:
        ctx.solve([[0.0, 1.0]], tol=e["tol"], maxiter=3000, raise_on_error=False)      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = ctx.solve([[0.0, 1.0]], tol=e["tol"], maxiter=3000, raise_on_error=False)
        out["mixed_solve"] = {"tol": e["tol"], "s": time.perf_counter() - t0, "iters": info["iters"],
                              "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"],
                              "status": info["status"]}
    ctx.close()
    return out


def run_large(args, dev, flush):
    """N >> 5000: 50,000 discs (the bench medium and density, p = 14, 1024 nodes, 24,544 wide).
    Operator applications with the translation through boxes (width 4, FP64; the contour part
    mixed) against the all-pairs FP32 translation, the box translation alone, and the mixed
    solve at 1e-8 with boxes."""
    import numpy as np
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    n, p = 50000, 14
    h = inputs.widened_half_width(n)
    w = inputs.Workload("disc50000_p14_ns1024", n, p, 1024, 163.0, -h, h, 6, np.array([[0.0, 1.0]]),
                        inputs.observation_points(-h, h, 64, 1.5), 1e-8)
    ctx = lsms.context_for(w, lsms.LSMS_MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.set_particles(w.centres())
    torch.cuda.synchronize()
    t_particles = time.perf_counter() - t0
    x = torch.from_numpy(inputs.random_coefficients(n, p, 1, 500)).to(dev)
    y = torch.empty_like(x)
    fl_m = lsms.APPLY_SCALED | lsms.APPLY_MIXED
    out = {"workload": w.name, "discs": n, "p": p, "contour_nodes": w.n_nodes, "set_particles_s": t_particles}
    for _ in range(2):
        ctx.apply_dev(x, y, fl_m)
    torch.cuda.synchronize()
    out["all_pairs_mixed"] = {"ms_per_apply": time_device(lambda: ctx.apply_dev(x, y, fl_m), 3, flush),
                              "translation": "FP32 all pairs"}
    t0 = time.perf_counter()
    ctx.set_fmm(4.0)
    torch.cuda.synchronize()
    nb, q = ctx.fmm_info()
    out["boxes"] = {"box_width": 4.0, "boxes": nb, "order": q, "setup_s": time.perf_counter() - t0}
    for _ in range(2):
        ctx.apply_dev(x, y, fl_m)
    torch.cuda.synchronize()
    ms = time_device(lambda: ctx.apply_dev(x, y, fl_m), max(3, min(args.steps, 10)), flush)
    def staged(flags):
        ctx.set_timing(True)
        tr, near, far = [], [], []
        for _ in range(3):
            flush.fill_(1.0)
            ctx.apply_dev(x, y, flags)
            tr.append(ctx.last_timing()[0])
            pairs, f_ms, n_ms = ctx.fmm_stats()
            far.append(f_ms)
            near.append(n_ms)
        ctx.set_timing(False)
        return pairs, statistics.mean(tr), statistics.mean(far), statistics.mean(near)

    pairs, tr_ms, far_ms, near_ms = staged(fl_m)
    out["boxes_mixed"] = {"ms_per_apply": ms, "translate_ms": tr_ms, "far_ms": far_ms, "near_ms": near_ms,
                          "translation": "through boxes: far field FP32 (shifts, FFT convolution), near field FP32"}
    # the near field (ordered pairs in adjacent boxes, 8 P^2 flop each) against the peak of its precision
    P = 2 * p + 1
    flop = 8.0 * P * P * pairs

    def roof(kernel, ms_, peak, note):
        ach = flop / (ms_ / 1e3) / 1e12
        return {"kernel": kernel, "bound": "alu", "pairs": pairs, "flop_per_launch": flop, "launch_ms": ms_,
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "peak_note": note}
    out["roofline_near_mixed"] = roof("k_pair_seq_f32 (+ the FP32 copy of the coefficients)", near_ms,
                                      FP32_PEAK_TFLOPS, "derived FP32: 152 SMs x 128 lanes x 2 x 2070 MHz")
    pairs, tr64, far64, near64 = staged(lsms.APPLY_SCALED)
    out["boxes_fp64_stages"] = {"translate_ms": tr64, "far_ms": far64, "near_ms": near64}
    out["roofline_near_fp64"] = roof("k_fmm_near", near64, FP64_PEAK_TFLOPS,
                                     "derived FP64: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz")
    ms64 = time_device(lambda: ctx.apply_dev(x, y, lsms.APPLY_SCALED), 3, flush)
    out["boxes_fp64"] = {"ms_per_apply": ms64}
    out["speedup_boxes_vs_all_pairs_mixed"] = out["all_pairs_mixed"]["ms_per_apply"] / ms
    if not args.no_solve:
        t0 = time.perf_counter()
        _, info = ctx.solve(w.sources, tol=1e-8, maxiter=3000, raise_on_error=False)
        out["mixed_solve"] = {"tol": 1e-8, "s": time.perf_counter() - t0, "iters": info["iters"],
                              "refinements": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"],
                              "status": info["status"]}
    ctx.close()
    return out


def run_translate_only(args):
    """The mixed translation alone (Lemma 3.1 in FP32: float conversion, the pair kernel, the partial
    sums' reduction, the near pairs) on --workload's first right-hand side, --steps applications
    after --warmup; the kernel's CUDA-event time and its algorithmic rate."""
    import torch

    from paper_1407_3868_gb300 import inputs, lsms
    w = inputs.WORKLOADS[args.workload]
    ctx = lsms.context_for(w, lsms.LSMS_MIXED)
    ctx.set_particles(w.centres())
    x = torch.from_numpy(inputs.random_coefficients(w.n, w.p, 1, 100)).cuda()
    y = torch.empty_like(x)
    flags = lsms.APPLY_SCALED | lsms.APPLY_MIXED | lsms.APPLY_NO_REFLECTION
    for _ in range(args.warmup):
        ctx.apply_dev(x, y, flags)
    ctx.set_timing(True)
    tr = []
    for _ in range(args.steps):
        ctx.apply_dev(x, y, flags)
        tr.append(ctx.last_timing()[0])
    shape = ctx.translation_tuning()[0]
    ctx.close()
    ms = statistics.mean(tr)
    flop = translation_flop(w.n, w.p)
    return {"workload": w.name, "kernel": SHAPE_KERNEL[shape], "steps": args.steps, "translate_ms": ms, "flop": flop,
            "tflops": flop / (ms / 1e3) / 1e12, "frac_of_fp32_peak": flop / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS}


def run_reference(args, rank):
    """The reference arm: the oracle (there is no reference code) on every host core, K timed steps
    after W warm-up steps, each step one pass over a bounded sample of target rows (oracle_timing).
    ms_per_step is the measured time of a step; value is the oracle's full applications per second
    derived from the same passes."""
    if rank != 0:
        return None
    s = oracle_timing(args.workload, args.oracle_rows, args.steps, args.warmup)
    value = 1.0 / s["full_apply_s"]
    cb = cpu_baseline_entry(s)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": 1,
            "steps": len(s["step_s"]), "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(s["step_s"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "operator": "FP64 oracle",
                                             "step": f"{s['rows_per_step']} of {s['n']} target rows"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.section == "large":
        import torch

        import __graft_entry__
        __graft_entry__.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"section": "large", "large": run_large(args, dev, flush)}))
        return
    if args.section == "translate":
        import torch

        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(torch.device("cuda", local_rank))
        print(json.dumps({"section": "translate", "translate": run_translate_only(args)}))
        return
    if args.section == "batched":
        import torch

        import __graft_entry__
        __graft_entry__.build()
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"section": "batched", "batched": run_batched(args, dev, flush)}))
        return
    if args.section == "example1":
        import torch

        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(torch.device("cuda", local_rank))
        print(json.dumps({"section": "example1", "example1": run_example1(args)}))
        return
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
