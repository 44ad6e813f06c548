"""Benchmark: CMG Fiedler solves/s on the 100^3 7-point grid (1M vertices).

A step is one pass of the whole method (Alg. 1): cmg_setup (heavy edge
coarsening + Galerkin products on every level) and cmg_fiedler (coarsest
solve, prolongation and power iteration on every level, final vector,
Rayleigh quotient and residual) on the synthetic 100x100x100 grid with
U[0.5, 1.5] edge weights (seed 1412), inputs resident in device memory.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain sequential FP64 restatement of the method) on the same workload.
With N > 1 ranks (torchrun), every rank solves its own replica of the
workload (the method does not shard a single graph; replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "grid3d_100x100x100_uniform[0.5,1.5]_seed1412", "n": 1_000_000,
            "edges": 2_970_000, "nnz": 5_940_000, "precision": "fp64", "tol": 1e-8,
            "coarse_size": 25}
# The timed step is one whole CMG solve; inputs (71 MB of CSR) are smaller than
# L2 (129 MB), so L2 is flushed between timed steps.
METRIC = "Fiedler solves/s (CMG setup + solve, 3D grid 1M vertices)"
UNIT = "solves/s"


def make_graph():
    from paper_1412_0565_gb300 import inputs
    return inputs.grid3d(100, 100, 100, "uniform", seed=1412)


def sweep_bytes(n, nnz, fp32=False):
    """Algorithmic bytes of one power-iteration sweep: the CSR stream
    (col int32 + weight), the row pointers, one read of x and one write of y."""
    if fp32:
        return 8 * nnz + 12 * n
    return 12 * nnz + 20 * n


def level_launch_bytes(n, nnz, sweeps, n_coarse, fp32=False):
    """Algorithmic bytes of one power-iteration launch on a level: the start
    vector (prolongation reads agg and the coarse vector, writes x; a second
    pass re-reads x) plus `sweeps` sweeps."""
    e = 4 if fp32 else 8
    start = (4 * n + e * n_coarse + e * n) + e * n
    return start + sweeps * sweep_bytes(n, nnz, fp32)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


PROFILE = os.path.join(ROOT, "profiles", "k_power_sell_f32_grid3d_100_level0.md")
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)
PROFILED_SOURCES = [os.path.join(ROOT, "paper_1412_0565_gb300", "csrc", f)
                    for f in ("refine.cu", "pi_common.cuh", "ffloat.cuh")]


def kernel_fingerprint():
    """sha256 (16 hex digits) of the profiled kernel sources with comments and
    whitespace removed: a comment edit keeps the capture valid, a code edit
    does not."""
    import hashlib
    import re
    parts = []
    for f in PROFILED_SOURCES:
        src = open(f).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        parts.append(" ".join(src.split()))
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per level-0 launch from the committed ncu summary, or None
    when the kernel code changed since that capture."""
    try:
        text = open(PROFILE).read()
        h = kernel_fingerprint()
        fields = dict(line.strip("- ").split(": ", 1) for line in text.splitlines()
                      if line.startswith("- ") and ": " in line)
        if fields.get("kernel_code_sha256_16") != h:
            return None, "kernel changed since the ncu capture"
        return int(fields["traffic_bytes_per_launch"]), "dram read+write per launch, ncu (profiles/)"
    except Exception as e:  # missing or malformed summary
        return None, f"no ncu summary ({type(e).__name__})"


def cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for l in f:
                if l.lower().startswith(("model name", "cpu model")):
                    model = l.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return model or os.uname().machine


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks of the job (each rank's timed total:
    the job takes as long as its slowest replica)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, total_ms: float, world: int, device: str = "cuda") -> float:
    """Units all ranks processed (each rank the same count: replicas) per
    second of the slowest rank's timed total."""
    return world * units_per_rank / (max_over_ranks(total_ms, world, device) / 1e3)


def oracle_solve(rp, col, w):
    import oracle
    h = oracle.Hierarchy(rp, col, w, seed=1412)
    r = h.solve()
    return r


def run_reference(args):
    """Reference arm: the CPU oracle (single thread) on the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    rp, col, w = make_graph()
    for _ in range(args.warmup):
        oracle_solve(rp, col, w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(rp, col, w)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(WORKLOAD, l2="input 71 MB < L2; CPU run"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full CMG solves (setup+solve) of the 1M-vertex "
                                   f"grid, single-threaded C oracle, {cpu_info()}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1412_0565_gb300 import cmg
    cmg.load()
    rp, col, w = make_graph()
    n, nnz = len(rp) - 1, int(rp[-1])
    drp = torch.from_numpy(rp).cuda()
    dcol = torch.from_numpy(col).cuda()
    dw = torch.from_numpy(w).cuda()
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def measure(precision, steps, warmup):
        """Timed steps of setup + solve with device-resident inputs."""
        opts = cmg.options(seed=1412, timing=1, precision=precision)
        u = torch.empty(n, dtype=torch.float64, device="cuda")
        kinds = {}

        def step(mid=None):
            h = cmg.Hierarchy(drp, dcol, dw, opts=opts, stream=sid)
            if mid is not None:
                mid.record(stream)
            _, lam, st = h.fiedler(u_out=u, stream=sid)
            if not kinds:
                kinds["k"] = h.level_kernels()
            h.close()
            return lam, st

        for _ in range(max(3, warmup)):
            step()
        barrier()
        l0 = cmg.kernel_launches()
        step_ms, setup_ms, stats = [], [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            em = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lam, st = step(em)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            setup_ms.append(e0.elapsed_time(em))
            stats.append(st)
        barrier()
        launches = cmg.kernel_launches() - l0
        total = max_over_ranks(sum(step_ms), world)
        srt = sorted(step_ms)
        return {"value": world * steps / (total / 1e3), "ms_per_step": total / steps,
                "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                "setup_ms": statistics.median(setup_ms),
                "solve_ms": statistics.median(a - b for a, b in zip(step_ms, setup_ms)),
                "stats": stats, "launches": launches, "u": u.cpu().numpy(), "lam": lam,
                "kinds": kinds["k"]}

    with ClockSampler(local) as clk:
        r32 = measure("fp32", args.steps, args.warmup)
        r64 = measure("fp64", args.steps, args.warmup)
    clocks = clk.summary()

    # ---- roofline of the dominant kernel: the level-0 power-iteration launch
    def roofline(r, fp32):
        st0 = r["stats"][-1]
        ns, nnzs, sweeps = st0["n"], st0["nnz"], st0["sweeps"]
        L = len(ns)
        ms0 = statistics.median(s["level_ms"][0] for s in r["stats"])
        by0 = level_launch_bytes(ns[0], nnzs[0], sweeps[0], ns[1] if L > 1 else 0, fp32)
        tot_b = sum(level_launch_bytes(ns[j], nnzs[j], sweeps[j], ns[j + 1] if j + 1 < L else 0, fp32)
                    for j in range(L))
        tot_ms = statistics.median(sum(s["level_ms"]) for s in r["stats"])
        return ms0, by0, tot_b, tot_ms, st0

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    if not hbm_peak:
        hbm_peak = 6800.0
    ms0, by0, tot_b, tot_ms, st32 = roofline(r32, True)
    achieved0 = by0 / (ms0 * 1e-3) / 1e9
    traffic, traffic_note = profiled_traffic()
    roof = {"bound": "hbm", "kernel": "k_power_sell<float, int>, level-0 launch",
            "achieved": achieved0, "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
            "frac": achieved0 / hbm_peak, "traffic": traffic, "traffic_note": traffic_note,
            "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved0 / NOMINAL_HBM_GBS,
            "bytes_per_launch": by0,
            "launch_ms": ms0, "sweeps_per_launch": st32["sweeps"][0],
            "all_levels": {"bytes": tot_b, "ms": tot_ms, "achieved": tot_b / (tot_ms * 1e-3) / 1e9}}
    ms0_64, by0_64, tot_b64, tot_ms64, st64 = roofline(r64, False)

    # accuracy of the FP32-sweep form against the plain FP64 form
    u32, u64 = r32["u"], r64["u"]
    cosang = abs(float(np.dot(u32, u64))) / (np.linalg.norm(u32) * np.linalg.norm(u64))
    acc = {"lambda2_rel_diff": abs(r32["lam"] - r64["lam"]) / abs(r64["lam"]),
           "angle_rad": float(np.arccos(min(1.0, cosang))),
           "note": "FP32-sweep result vs plain FP64 GPU result, tolerance-mode sweep counts differ"}

    # ---- end to end through the public API with host buffers (FP32 form)
    e2e_ms = []
    # inputs and the result buffer in pinned host memory (filled once, outside
    # the timed region), so the copies inside it are plain DMA transfers
    try:
        rp_h, col_h, w_h, hu = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
                                for a in (rp, col, w, np.empty(n, dtype=np.float64)))
        pinned = True
    except Exception:
        rp_h, col_h, w_h, hu = (np.ascontiguousarray(a) for a in (rp, col, w, np.empty(n, dtype=np.float64)))
        pinned = False
    for _ in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = cmg.Hierarchy(rp_h, col_h, w_h, seed=1412, precision="fp32", stream=sid)
        h.fiedler(u_out=hu, stream=sid)
        h.close()
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = whole_job_rate(len(e2e_ms), sum(e2e_ms), world)

    batch = None
    if not args.no_batch and world == 1:
        batch = run_batch(args, stream, flush)
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(args)
    chung_lu = None
    if not args.no_chung_lu and world == 1:
        chung_lu = run_chung_lu(args, stream, flush)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            reps, t0 = 0, time.perf_counter()
            while reps < 3 or (time.perf_counter() - t0 < 10 and reps < 8):
                oracle_solve(rp, col, w)
                reps += 1
            dt = time.perf_counter() - t0
            cpu = {"value": reps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{reps} full CMG solves (setup+solve, FP64) of the same 1M-vertex grid, "
                             f"single-threaded C oracle on {cpu_info()}"}
        line = {
            "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": r32["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sweeps, f64 final sweep / Rayleigh quotient, float-float reductions",
            "data": "synthetic",
            "config": dict(WORKLOAD, precision="fp32-sweep",
                           l2="256 MB buffer written between timed steps (flush)",
                           parallelism=f"replicas{world}"),
            "latency_ms": {"p50": r32["p50_ms"], "p99": r32["p99_ms"]},
            "split_ms": {"setup": r32["setup_ms"], "solve": r32["solve_ms"]},
            "levels": {"n": st32["n"], "nnz": st32["nnz"], "sweeps": st32["sweeps"],
                       "kernel": [KERNEL_KIND[k] for k in r32["kinds"][0]],
                       "level_ms": [round(x, 4) for x in st32["level_ms"]]},
            "lambda2": st32["lambda2"], "residual": st32["residual"],
            "fp64": {"value": r64["value"], "ms_per_step": r64["ms_per_step"],
                     "latency_ms": {"p50": r64["p50_ms"], "p99": r64["p99_ms"]},
                     "split_ms": {"setup": r64["setup_ms"], "solve": r64["solve_ms"]},
                     "sweeps": st64["sweeps"], "level_ms": [round(x, 4) for x in st64["level_ms"]],
                     "lambda2": st64["lambda2"], "residual": st64["residual"],
                     "level0_launch": {"ms": ms0_64, "bytes": by0_64,
                                       "achieved_gbs": by0_64 / (ms0_64 * 1e-3) / 1e9},
                     "gpu_launches": r64["launches"]},
            "fp32_vs_fp64": acc,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (n + 1) + 12 * nnz, "d2h_bytes_per_step": 8 * n,
                    "host_memory": "pinned" if pinned else "pageable"},
            "gpu_launches": r32["launches"],
            "clocks": clocks,
            "batch": batch,
            "serving": serving,
            "chung_lu": chung_lu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


BATCH_WORKLOAD = ("4096 graphs, n log-uniform [500, 20000], random geometric (mean degree 8) / "
                  "near-square 2D grid / Barabasi-Albert m=4 round-robin, U[0.5,1.5] weights, seed 1412")
SERVE_WORKLOAD = ("requests drawn uniformly from {P} graphs with log n ~ Normal truncated to "
                  "[ln 1e3, ln 2e6] (families and weights as the batch), Poisson arrivals")


def _pool_workers():
    return max(1, min(16, os.cpu_count() or 1))


def run_batch(args, stream, flush):
    """Batched form (many graphs per launch): setup + solve of the whole batch
    per step; FP32 sweep form against the batched and the plain FP64 forms."""
    import torch
    from paper_1412_0565_gb300 import cmg, inputs
    t0 = time.perf_counter()
    graphs = inputs.batch_graphs(args.batch_graphs, workers=_pool_workers())
    rp, col, w, offs = inputs.concat_csr(graphs)
    gen_s = time.perf_counter() - t0
    G, N, nnz = len(graphs), len(rp) - 1, int(rp[-1])
    sid = stream.cuda_stream
    drp, dcol, dw = (torch.from_numpy(a).cuda() for a in (rp, col, w))
    u = torch.empty(N, dtype=torch.float64, device="cuda")

    def solve_steps(prec, K, shapes=None, replay=None, timing=0):
        kw = dict(seed=1412, precision=prec, timing=timing)
        if replay is not None:
            kw["schedule"] = "replay"
        step_ms, setup_ms, out = [], [], None
        for k in range(K):
            flush.zero_()
            e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _e in range(3))
            e0.record(stream)
            b = cmg.Batch(offs, drp, dcol, dw, stream=sid, **kw)
            if shapes:
                for lvl, sh in enumerate(shapes):
                    b.set_shape(lvl, *sh)
            if replay is not None:
                b.set_replay(replay)
            em.record(stream)
            _u, lam, _res, sts = b.fiedler(u_out=u, stream=sid)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            setup_ms.append(e0.elapsed_time(em))
            out = (b, lam, sts)
            if k + 1 < K:
                b.close()
        return step_ms, setup_ms, out

    def tuned_shapes(prec):
        b = cmg.Batch(offs, drp, dcol, dw, stream=sid, seed=1412, precision=prec)
        b.autotune(stream=sid)
        sh = [b.shape(lvl) for lvl in range(b.union_levels)]
        b.close()
        return sh

    res = {"workload": BATCH_WORKLOAD, "graphs": G, "n_total": N, "nnz_total": nnz,
           "generate_s": round(gen_s, 2),
           "l2": "union CSR (1.7 GB) larger than L2; 256 MB buffer written between steps"}
    for prec, K in (("fp32", args.batch_steps), ("fp64", 1)):
        shapes = tuned_shapes(prec)
        step_ms, setup_ms, (b, lam, sts) = solve_steps(prec, K, shapes)
        st = [b.stats(q) for q in range(G)]
        if prec == "fp64":
            sweeps64 = [s_["sweeps"] for s_ in st]
            lam64, u64 = lam.copy(), u.cpu().numpy()
        else:
            lam32_tol, u32_tol = lam.copy(), u.cpu().numpy()
        b.close()
        tot = sum(step_ms)
        k0 = np.array([s_["sweeps"][0] for s_ in st])
        visits = sum(s_["sweeps"][j] * (s_["n"][j] + s_["nnz"][j]) for s_ in st for j in range(s_["levels"]))
        res[prec] = {"value": G * K / (tot / 1e3), "unit": "solves/s", "steps": K,
                     "ms_per_step": tot / K, "setup_ms": statistics.median(setup_ms),
                     "solve_ms": statistics.median(a - b_ for a, b_ in zip(step_ms, setup_ms)),
                     "warn_maxiter": int((sts != 0).sum()), "shapes": shapes,
                     "level0_sweeps": {"mean": float(k0.mean()), "max": int(k0.max())},
                     "row_and_entry_visits": int(visits)}
        if prec == "fp32":
            # per-level device times (launches issued one by one) and the
            # level-0 launch against HBM bandwidth
            _, _, (bt, _, _) = solve_steps(prec, 1, shapes, timing=1)
            lms = bt.level_ms()
            stt = [bt.stats(q) for q in range(G)]
            by0 = sum(s_["sweeps"][0] * (8 * s_["nnz"][0] + 12 * s_["n"][0]) for s_ in stt)
            bt.close()
            res[prec]["level_ms"] = [round(x, 2) for x in lms]
            res[prec]["level0_launch"] = {"ms": lms[0], "algorithmic_bytes": by0,
                                          "achieved_gbs": by0 / (lms[0] * 1e-3) / 1e9}
    # precision alone: FP32 sweeps with the FP64 run's per-graph sweep counts
    _, _, (b, lam32, _) = solve_steps("fp32", 1, None, replay=sweeps64)
    u32 = u.cpu().numpy()
    b.close()

    def compare(lam_a, u_a):
        rel = np.abs(lam_a - lam64) / np.abs(lam64)
        ang = np.empty(G)
        for q in range(G):
            a_, c_ = u_a[offs[q]:offs[q + 1]], u64[offs[q]:offs[q + 1]]
            cq = abs(float(np.dot(a_, c_))) / (np.linalg.norm(a_) * np.linalg.norm(c_))
            ang[q] = np.arccos(min(1.0, cq))
        return {"lambda2_rel_max": float(rel.max()), "lambda2_rel_p99": float(np.percentile(rel, 99)),
                "angle_max": float(ang.max()), "angle_p99": float(np.percentile(ang, 99)),
                "graphs_within_1e-6_and_1e-4": int(((rel <= 1e-6) & (ang <= 1e-4)).sum())}

    res["fp32_vs_fp64_replay"] = compare(lam32, u32)
    res["fp32_vs_fp64_replay"]["note"] = "FP32 sweeps with the FP64 run's per-graph, per-level sweep counts"
    res["fp32_vs_fp64_tolerance_mode"] = compare(lam32_tol, u32_tol)
    # the plain FP64 form: one graph at a time through cmg_setup / cmg_fiedler
    idx = list(range(0, G, max(1, G // args.batch_plain_sample)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in idx:
        with cmg.Hierarchy(*graphs[q], seed=1412, stream=sid) as h:
            h.fiedler(stream=sid)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res["plain_fp64_single_graph"] = {"value": len(idx) / dt, "unit": "solves/s",
                                      "sample": f"{len(idx)} graphs of the batch, host inputs, one at a time"}
    res["fp32_batched_over_plain_fp64"] = res["fp32"]["value"] / res["plain_fp64_single_graph"]["value"]
    return res


def cl_workload(n):
    return (f"Chung-Lu power-law graph, n {n:,} before the largest component, mean degree 16, "
            "exponent 2.5, degrees capped at sqrt(16 n), lognormal(0,1) weights, seed 1412")


def run_chung_lu(args, stream, flush):
    """Config 3: one large power-law graph through the single-graph path, FP32
    sweeps against the FP64 form (setup + solve per step)."""
    import torch
    from paper_1412_0565_gb300 import cmg, inputs
    t0 = time.perf_counter()
    rp, col, w = inputs.chung_lu(args.cl_n, seed=1412)
    gen_s = time.perf_counter() - t0
    n, nnz = len(rp) - 1, int(rp[-1])
    sid = stream.cuda_stream
    drp, dcol, dw = (torch.from_numpy(a).cuda() for a in (rp, col, w))
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    deg = rp[1:] - rp[:-1]
    out = {"workload": cl_workload(args.cl_n), "n": n, "nnz": nnz, "max_degree": int(deg.max()),
           "generate_s": round(gen_s, 1)}
    res = {}
    for prec in ("fp32", "fp64"):
        opts = cmg.options(seed=1412, precision=prec, timing=1)
        ms, setup = [], []
        for k in range(args.cl_warmup + args.cl_steps):
            flush.zero_()
            e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _e in range(3))
            e0.record(stream)
            h = cmg.Hierarchy(drp, dcol, dw, opts=opts, stream=sid)
            em.record(stream)
            _u, lam, st = h.fiedler(u_out=u, stream=sid)
            e1.record(stream)
            e1.synchronize()
            kinds = h.level_kernels()
            h.close()
            if k >= args.cl_warmup:
                ms.append(e0.elapsed_time(e1))
                setup.append(e0.elapsed_time(em))
        by0 = st["sweeps"][0] * ((8 if prec == "fp32" else 12) * st["nnz"][0] + (12 if prec == "fp32" else 20) * st["n"][0])
        res[prec] = {"u": u.cpu().numpy(), "lam": lam, "sweeps": st["sweeps"]}
        out[prec] = {"value": len(ms) / (sum(ms) / 1e3), "unit": "solves/s", "ms_per_step": statistics.mean(ms),
                     "setup_ms": statistics.mean(setup), "levels": st["levels"], "sweeps": st["sweeps"],
                     "level_n": st["n"], "level_nnz": st["nnz"],
                     "level_kernel": [KERNEL_KIND[k] for k in kinds[0]], "level_staged": kinds[1],
                     "level_ms": [round(x, 3) for x in st["level_ms"]], "lambda2": lam,
                     "residual": st["residual"],
                     "level0_launch": {"ms": st["level_ms"][0], "algorithmic_bytes": by0,
                                       "achieved_gbs": by0 / (st["level_ms"][0] * 1e-3) / 1e9}}
    # precision alone: FP32 sweeps replaying the FP64 sweep counts
    h = cmg.Hierarchy(drp, dcol, dw, seed=1412, precision="fp32", schedule="replay",
                      replay_sweeps=res["fp64"]["sweeps"], stream=sid)
    _u, lam32, _ = h.fiedler(u_out=u, stream=sid)
    h.close()
    u32, u64 = u.cpu().numpy(), res["fp64"]["u"]
    c = abs(float(np.dot(u32, u64))) / (np.linalg.norm(u32) * np.linalg.norm(u64))
    out["fp32_vs_fp64_replay"] = {"lambda2_rel": abs(lam32 - res["fp64"]["lam"]) / abs(res["fp64"]["lam"]),
                                  "angle": float(np.arccos(min(1.0, c)))}
    c2 = abs(float(np.dot(res["fp32"]["u"], u64))) / (np.linalg.norm(res["fp32"]["u"]) * np.linalg.norm(u64))
    out["fp32_vs_fp64_tolerance_mode"] = {
        "lambda2_rel": abs(res["fp32"]["lam"] - res["fp64"]["lam"]) / abs(res["fp64"]["lam"]),
        "angle": float(np.arccos(min(1.0, c2)))}
    return out


KERNEL_KIND = {0: "smem", 1: "slice", 2: "slice+staged", 3: "tiled"}


def run_serving(args):
    """Request loop: closed-loop saturation, then Poisson arrivals at 0.8 of
    it; FP32 server (batching, resident hierarchies) and plain FP64 server
    (no batching) on the same request trace."""
    from paper_1412_0565_gb300 import cmg, inputs
    graphs = inputs.serving_graphs(args.serve_graphs, workers=_pool_workers())
    rng = np.random.default_rng(1412)
    trace = rng.integers(0, len(graphs), size=args.serve_requests)
    out = {"workload": SERVE_WORKLOAD.format(P=len(graphs)), "requests": int(len(trace)),
           "distinct_graphs": len(graphs), "n_max": int(max(len(g[0]) - 1 for g in graphs)),
           "n_median": int(np.median([len(g[0]) - 1 for g in graphs]))}
    lam_by = {}
    for name, cfg, prec in (("fp32", dict(workers=4, max_batch=256, batch_max_n=50000), "fp32"),
                            ("fp64_plain", dict(workers=4, max_batch=1), "fp64")):
        def run(rate):
            with cmg.Server(seed=1412, precision=prec, **cfg) as srv:
                ids = [srv.add_graph(*g) for g in graphs]
                t0 = time.perf_counter()
                tickets = []
                if rate is None:
                    tickets = [srv.submit(ids[k], want_vector=False) for k in trace]
                else:
                    arr = np.cumsum(np.random.default_rng(7).exponential(1.0 / rate, size=len(trace)))
                    for k, ta in zip(trace, arr):
                        d = t0 + ta - time.perf_counter()
                        if d > 0:
                            time.sleep(d)
                        tickets.append(srv.submit(ids[k], want_vector=False))
                rs = [srv.wait(t)[1] for t in tickets]
                dt = time.perf_counter() - t0
                return rs, dt, srv.stats()

        rs, dt, st = run(None)
        sat = len(trace) / dt
        rs2, dt2, st2 = run(0.8 * sat)
        lat = np.array([r["latency_ms"] for r in rs2])
        lam_by[name] = np.array([r["lambda2"] for r in rs2])
        out[name] = {"saturation_solves_s": sat, "rho": 0.8, "offered_rate": 0.8 * sat,
                     "achieved_solves_s": len(trace) / dt2,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "warm_fraction": float(np.mean([r["warm"] for r in rs2])),
                     "batched_fraction": float(np.mean([r["batch_size"] > 1 for r in rs2])),
                     "jobs": {k: st2[k] for k in ("single_jobs", "batch_jobs", "warm_jobs", "evictions")},
                     "peak_device_bytes": st2["peak_bytes"]}
    rel = np.abs(lam_by["fp32"] - lam_by["fp64_plain"]) / np.abs(lam_by["fp64_plain"])
    out["fp32_vs_fp64_lambda2_rel"] = {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)),
                                       "note": "tolerance mode (sweep counts may differ)"}
    # precision alone on the serving graphs: FP32 sweeps replaying the FP64
    # solve's per-level sweep counts
    lam_rel, ang = [], []
    for g in graphs[:args.serve_replay_sample]:
        u64, l64, st64 = cmg.fiedler(*g, seed=1412, precision="fp64")
        u32, l32, _ = cmg.fiedler(*g, seed=1412, precision="fp32", schedule="replay",
                                  replay_sweeps=st64["sweeps"])
        lam_rel.append(abs(l32 - l64) / abs(l64))
        c = abs(float(np.dot(u32, u64))) / (np.linalg.norm(u32) * np.linalg.norm(u64))
        ang.append(float(np.arccos(min(1.0, c))))
    out["fp32_vs_fp64_replay"] = {"graphs": len(lam_rel), "lambda2_rel_max": max(lam_rel),
                                  "angle_max": max(ang),
                                  "within_1e-6_and_1e-4": int(sum((r <= 1e-6) and (a <= 1e-4)
                                                                  for r, a in zip(lam_rel, ang)))}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-plain-sample", type=int, default=32)
    ap.add_argument("--serve-graphs", type=int, default=48)
    ap.add_argument("--serve-requests", type=int, default=160)
    ap.add_argument("--serve-replay-sample", type=int, default=16)
    ap.add_argument("--no-chung-lu", action="store_true")
    ap.add_argument("--cl-steps", type=int, default=3)
    ap.add_argument("--cl-warmup", type=int, default=1)
    ap.add_argument("--cl-n", type=int, default=4_194_304,
                    help="Chung-Lu vertices before the largest component (smaller: profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
