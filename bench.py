"""Benchmark: CMG Fiedler solves/s on the 100^3 7-point grid (1M vertices).

A step is one pass of the whole method (Alg. 1): cmg_setup (heavy edge
coarsening + Galerkin products on every level) and cmg_fiedler (coarsest
solve, prolongation and power iteration on every level, final vector,
Rayleigh quotient and residual) on the synthetic 100x100x100 grid with
U[0.5, 1.5] edge weights (seed 1412), inputs resident in device memory.  The
headline is the FP64 form, the paper's arithmetic; the FP32-sweep form, the
64x64 grid, the 4,096-graph batch, the request loop and the Chung-Lu graph
are reported under their own keys, each result's accuracy against the CPU
oracle.

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
L2_NOTE = "inputs 71 MB < L2: a 256 MB buffer is written between timed steps (flush)"
METRIC = "Fiedler solves/s (CMG setup + solve, 3D grid 1M vertices)"
UNIT = "solves/s"


def config(world: int) -> dict:
    """The workload of both arms (identical dicts: the reference arm times the
    oracle on exactly this configuration)."""
    return dict(WORKLOAD, l2=L2_NOTE, parallelism=f"replicas{world}")


def make_graph():
    from paper_1412_0565_gb300 import inputs
    return inputs.grid3d(100, 100, 100, "uniform", seed=1412)


def sweep_bytes(n, nnz, fp32=False):
    """Algorithmic bytes of one power-iteration sweep: the CSR stream
    (col int32 + weight), the row pointers, one read of x and one write of y."""
    if fp32:
        return 8 * nnz + 12 * n
    return 12 * nnz + 20 * n


def sweep_flops_fp64(n, nnz):
    """Algorithmic FP64 flops of one FP64 sweep: an FMA per stored entry, and
    per row the diagonal FMA (g - d_i) x_i, the shift and scale (2), and the
    sums y, y^2, y x_prev of the stop test (5)."""
    return 2 * nnz + 9 * n


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


PROFILES = {"fp64": os.path.join(ROOT, "profiles", "k_power_sell_f64_grid3d_100_level0.md"),
            "fp32": os.path.join(ROOT, "profiles", "k_power_sell_f32_grid3d_100_level0.md")}
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)
# FP64 pipe: 2 FMA per SM per clock (the nominal 1.25 TFLOP/s of a 152-SM GB300 at 2.07 GHz)
FP64_FMA_PER_SM_CLK = 2
SMS = 152
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


def profiled_traffic(prec):
    """DRAM bytes per level-0 launch from the committed ncu summary, or None
    when the kernel code changed since that capture."""
    try:
        text = open(PROFILES[prec]).read()
        h = kernel_fingerprint()
        fields = dict(line.strip("- ").split(": ", 1) for line in text.splitlines()
                      if line.startswith("- ") and ": " in line)
        if fields.get("kernel_code_sha256_16") != h:
            return None, "kernel changed since the ncu capture"
        return int(fields["traffic_bytes_per_launch"]), "dram read+write per launch, ncu (profiles/)"
    except Exception as e:  # missing or malformed summary
        return None, f"no ncu summary ({type(e).__name__})"


def cpu_info():
    """CPU model and core count of this host (lscpu, then /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        f = dict(l.split(":", 1) for l in out.splitlines() if ":" in l)
        f = {k.strip(): v.strip() for k, v in f.items()}
        model = f.get("Model name", "")
        if f.get("Vendor ID"):
            model = f"{f['Vendor ID']} {model}".strip()
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for l in fh:
                    if l.lower().startswith(("model name", "cpu model", "cpu part")):
                        model = l.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"model": model or os.uname().machine, "nproc": os.cpu_count(), "arch": os.uname().machine}


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
    ci = cpu_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cpu_model": ci["model"], "nproc": ci["nproc"],
                         "sample": f"{args.steps} full CMG solves (setup+solve, FP64) of the 1M-vertex "
                                   f"grid, single-threaded C oracle on one of {ci['nproc']} cores "
                                   f"({ci['model']})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _angle(a, b):
    c = abs(float(np.dot(a, b))) / (np.linalg.norm(a) * np.linalg.norm(b))
    return float(np.arccos(min(1.0, c)))


def _vec_err(u, ref):
    if np.dot(u, ref) < 0:
        u = -u
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))


# ---------------------------------------------------------------- oracle jobs (spawned pool)
def _oracle_job(job):
    """One oracle solve in a worker process: ("batch", i) graph i of the
    4,096-graph batch; ("graph", name, rp, col, w) an explicit graph.
    Returns (key, sweeps, u, lambda, residual, seconds)."""
    import oracle
    from paper_1412_0565_gb300 import inputs
    t0 = time.perf_counter()
    if job[0] == "batch":
        g = inputs.batch_graph(job[1])
        key = job[1]
    elif job[0] == "chung_lu":
        g = inputs.chung_lu(job[1], seed=1412)
        key = "chung_lu"
    else:
        g = job[2:]
        key = job[1]
    r = oracle.Hierarchy(*g, seed=1412).solve()
    return key, r["sweeps"], r["u"], r["lam"], r["res"], time.perf_counter() - t0


def run_oracle_jobs(jobs, workers):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    out = {}
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for key, sw, u, lam, res, dt in ex.map(_oracle_job, jobs, chunksize=4):
            out[key] = {"sweeps": sw, "u": u, "lam": lam, "res": res, "s": dt}
    return out


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
        info = {}

        def step(mid=None):
            h = cmg.Hierarchy(drp, dcol, dw, opts=opts, stream=sid)
            if mid is not None:
                mid.record(stream)
            _, lam, st = h.fiedler(u_out=u, stream=sid)
            if not info:
                info["kinds"] = h.level_kernels()
                info["prec"] = h.level_precision()
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
                "kinds": info["kinds"], "prec": info["prec"]}

    with ClockSampler(local) as clk:
        r64 = measure("fp64", args.steps, args.warmup)
        r32 = measure("fp32", args.steps, args.warmup) if not args.no_fp32 else None
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0

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

    def level0(r, fp32):
        st0 = r["stats"][-1]
        ns, nnzs, sweeps = st0["n"], st0["nnz"], st0["sweeps"]
        L = len(ns)
        ms0 = statistics.median(s["level_ms"][0] for s in r["stats"])
        by0 = level_launch_bytes(ns[0], nnzs[0], sweeps[0], ns[1] if L > 1 else 0, fp32)
        tot_b = sum(level_launch_bytes(ns[j], nnzs[j], sweeps[j], ns[j + 1] if j + 1 < L else 0,
                                       r["prec"][j] == "fp32") for j in range(L))
        tot_ms = statistics.median(sum(s["level_ms"]) for s in r["stats"])
        return ms0, by0, tot_b, tot_ms, st0

    def roofline(r, fp32):
        """The dominant kernel: the level-0 power-iteration launch.  FP64
        sweeps are bound by the FP64 pipe on this GPU (at its peak a sweep's
        FP64 work takes longer than its bytes at the HBM copy peak); FP32
        sweeps by memory."""
        ms0, by0, tot_b, tot_ms, st0 = level0(r, fp32)
        n0, nnz0, k0 = st0["n"][0], st0["nnz"][0], st0["sweeps"][0]
        gbs = by0 / (ms0 * 1e-3) / 1e9
        traffic, tnote = profiled_traffic("fp32" if fp32 else "fp64")
        hbm = {"achieved": gbs, "peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
               "frac": gbs / hbm_peak, "frac_of_nominal": gbs / NOMINAL_HBM_GBS}
        common = {"bytes_per_launch": by0, "launch_ms": ms0, "sweeps_per_launch": k0,
                  "traffic": traffic, "traffic_note": tnote,
                  "l2_resident": by0 / max(k0, 1) < 126e6,
                  "note": ("the level's sweep stream fits in L2 (129 MB): after the first sweep it "
                           "is served from L2, so the GB/s is an effective streaming rate, not DRAM "
                           "traffic (traffic = ncu DRAM bytes)"),
                  "all_levels": {"bytes": tot_b, "ms": tot_ms,
                                 "achieved_gbs": tot_b / (tot_ms * 1e-3) / 1e9}}
        if fp32:
            return dict({"bound": "hbm", "kernel": "k_power_sell<float, int>, level-0 launch"}, **hbm,
                        **common)
        flops = k0 * sweep_flops_fp64(n0, nnz0)
        peak_tf = FP64_FMA_PER_SM_CLK * 2 * SMS * sm_mhz * 1e6 / 1e12
        tf = flops / (ms0 * 1e-3) / 1e12
        return dict({"bound": "alu", "kernel": "k_power_sell<double, int>, level-0 launch",
                     "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                     "peak_source": "derived: 2 FP64 FMA per SM per clock x 152 SMs x the median SM "
                                    "clock of the run (nominal 1.25 TFLOP/s)",
                     "flops_per_launch": flops,
                     "hbm": hbm}, **common)

    def e2e(precision):
        """The public API with host buffers: host->device copy of the CSR and
        device->host copy of the vector inside the timed region."""
        ms = []
        try:
            rp_h, col_h, w_h, hu = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
                                    for a in (rp, col, w, np.empty(n, dtype=np.float64)))
            pinned = True
        except Exception:
            rp_h, col_h, w_h, hu = (np.ascontiguousarray(a) for a in (rp, col, w, np.empty(n, dtype=np.float64)))
            pinned = False
        for _ in range(max(3, min(args.steps, 8))):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = cmg.Hierarchy(rp_h, col_h, w_h, seed=1412, precision=precision, stream=sid)
            h.fiedler(u_out=hu, stream=sid)
            h.close()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return {"value": whole_job_rate(len(ms), sum(ms), world), "unit": UNIT,
                "h2d_bytes_per_step": 8 * (n + 1) + 12 * nnz, "d2h_bytes_per_step": 8 * n,
                "host_memory": "pinned" if pinned else "pageable", "steps": len(ms)}

    roof64 = roofline(r64, False)
    e2e64 = e2e("fp64") if not args.no_e2e else None
    fp32 = None
    if r32 is not None:
        ms0, by0, tot_b, tot_ms, st32 = level0(r32, True)
        fp32 = {"value": r32["value"], "unit": UNIT, "ms_per_step": r32["ms_per_step"],
                "dtype": "f32 sweeps on levels of at least 2^20 stored entries, f64 sweeps below; "
                         "float-float stop/mean/norm sums; f64 last level-0 sweep and Rayleigh quotient",
                "latency_ms": {"p50": r32["p50_ms"], "p99": r32["p99_ms"]},
                "split_ms": {"setup": r32["setup_ms"], "solve": r32["solve_ms"]},
                "levels": {"sweeps": st32["sweeps"], "precision": r32["prec"],
                           "kernel": [KERNEL_KIND[k] for k in r32["kinds"][0]],
                           "level_ms": [round(x, 4) for x in st32["level_ms"]]},
                "lambda2": st32["lambda2"], "residual": st32["residual"],
                "roofline": roofline(r32, True),
                "e2e": e2e("fp32") if not args.no_e2e else None,
                "gpu_launches": r32["launches"]}

    c1 = run_c1(args, stream, flush) if (not args.no_c1 and world == 1) else None
    batch = run_batch(args, stream, flush) if (not args.no_batch and world == 1) else None
    serving = run_serving(args) if (not args.no_serving and world == 1) else None
    chung_lu = run_chung_lu(args, stream, flush) if (not args.no_chung_lu and world == 1) else None
    gcmg = run_gcmg(args, stream) if (not args.no_gcmg and world == 1) else None
    study = run_schedule_study(args, stream) if (not args.no_study and world == 1) else None

    if rank == 0:
        cpu = None
        ci = cpu_info()
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            reps, t0 = 0, time.perf_counter()
            while reps < 3 or (time.perf_counter() - t0 < 10 and reps < 8):
                oracle_solve(rp, col, w)
                reps += 1
            dt = time.perf_counter() - t0
            cpu = {"value": reps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "cpu_model": ci["model"], "nproc": ci["nproc"],
                   "sample": f"{reps} full CMG solves (setup+solve, FP64) of the same 1M-vertex grid, "
                             f"single-threaded C oracle on one of {ci['nproc']} cores ({ci['model']})"}
        # ---- accuracy against the CPU oracle (spawned worker processes, after
        # every timed region)
        accuracy = None
        if world == 1 and not args.no_oracle_checks:
            accuracy = oracle_checks(args, (rp, col, w), r64, r32, batch, chung_lu, stream)
        st64 = r64["stats"][-1]
        if batch:
            for k in [k for k in batch if k.startswith("_")]:
                batch.pop(k)
        line = {
            "metric": METRIC, "value": r64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": r64["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64",
            "dtype_note": "f64 sweeps, f64 Rayleigh quotient and residual; the stop cosine, mean and norm "
                          "sums in float-float (about 48 bits: the 1 - 1e-8 cosine test is resolved to "
                          "about 1e-14)",
            "data": "synthetic",
            "config": config(world),
            "latency_ms": {"p50": r64["p50_ms"], "p99": r64["p99_ms"]},
            "split_ms": {"setup": r64["setup_ms"], "solve": r64["solve_ms"]},
            "levels": {"n": st64["n"], "nnz": st64["nnz"], "sweeps": st64["sweeps"],
                       "kernel": [KERNEL_KIND[k] for k in r64["kinds"][0]],
                       "level_ms": [round(x, 4) for x in st64["level_ms"]]},
            "lambda2": st64["lambda2"], "residual": st64["residual"],
            "roofline": roof64, "cpu_baseline": cpu,
            "e2e": e2e64,
            "gpu_launches": r64["launches"],
            "clocks": clocks,
            "host": ci,
            "fp32": fp32,
            "accuracy_vs_oracle": accuracy,
            "c1": c1,
            "batch": batch,
            "serving": serving,
            "chung_lu": chung_lu,
            "gcmg": gcmg,
            "schedule_study": study,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def oracle_checks(args, c2_graph, r64, r32, batch, chung_lu, stream):
    """Every accuracy statement of the line, against the FP64 CPU oracle run
    in spawned processes: the C2 vectors, all (or a seeded sample of) the
    4,096 batch graphs, and a Chung-Lu graph of the same recipe small enough
    for the oracle.  FP32 results are compared in replay mode (the oracle's
    own per-level sweep counts replayed on the GPU: precision alone); FP64
    results in tolerance mode (same counts expected)."""
    import torch
    from paper_1412_0565_gb300 import cmg, inputs
    t0 = time.perf_counter()
    G = args.batch_graphs if batch is not None else 0
    if G and args.batch_oracle_sample and args.batch_oracle_sample < G:
        idx = sorted(np.random.default_rng(1412).choice(G, args.batch_oracle_sample, replace=False).tolist())
    else:
        idx = list(range(G))
    jobs = [("graph", "c2", *c2_graph)]
    if args.cl_oracle_n:
        jobs.append(("chung_lu", args.cl_oracle_n))
    jobs += [("batch", i) for i in idx]
    res = run_oracle_jobs(jobs, workers=max(1, min(16, (os.cpu_count() or 2) - 1)))
    out = {"oracle_s": round(time.perf_counter() - t0, 1)}
    # ---- C2: FP64 form in tolerance mode; FP32 form with the oracle's counts
    o = res["c2"]
    out["c2_fp64"] = {"vec_rel_err": _vec_err(r64["u"], o["u"]),
                      "lambda2_rel_err": abs(r64["lam"] - o["lam"]) / abs(o["lam"]),
                      "same_sweeps": r64["stats"][-1]["sweeps"] == o["sweeps"].tolist(),
                      "gate": "vector <= 1e-10, lambda2 <= 1e-12"}
    if r32 is not None:
        rp, col, w = c2_graph
        u32, lam32, _ = cmg.fiedler(rp, col, w, seed=1412, precision="fp32", schedule="replay",
                                    replay_sweeps=o["sweeps"].tolist())
        out["c2_fp32_replay"] = {"lambda2_rel_err": abs(lam32 - o["lam"]) / abs(o["lam"]),
                                 "angle_rad": _angle(u32, o["u"]), "gate": "lambda2 <= 1e-6, angle <= 1e-4"}
    # ---- batch: every sampled graph, FP64 batch (tolerance) and FP32 batch (replay)
    if idx:
        graphs = batch["_graphs"]
        rp, col, w, offs = batch["_union"]
        drp, dcol, dw = (torch.from_numpy(a).cuda() for a in (rp, col, w))
        sid = stream.cuda_stream
        u64, lam64 = batch["_u64"], batch["_lam64"]
        sw64 = batch["_sweeps64"]
        # FP32 batch with the oracle's counts (graphs outside the sample keep
        # the GPU FP64 counts; only the sample is compared)
        reps = [list(s) for s in sw64]
        for i in idx:
            reps[i] = res[i]["sweeps"].tolist()
        u_t = torch.empty(len(rp) - 1, dtype=torch.float64, device="cuda")
        with cmg.Batch(offs, drp, dcol, dw, seed=1412, precision="fp32", schedule="replay", stream=sid) as b:
            b.set_replay(reps)
            _, lam32, _, _ = b.fiedler(u_out=u_t, stream=sid)
        u32 = u_t.cpu().numpy()
        with cmg.Batch(offs, drp, dcol, dw, seed=1412, precision="fp64", schedule="replay", stream=sid) as b:
            b.set_replay(reps)
            _, lam64r, _, _ = b.fiedler(u_out=u_t, stream=sid)
        u64r = u_t.cpu().numpy()
        rel64, vec64, rel32, ang32, same = [], [], [], [], 0
        rel64r, vec64r, apart = [], [], []
        for i in idx:
            ref = res[i]
            a, b_ = offs[i], offs[i + 1]
            rel64r.append(abs(lam64r[i] - ref["lam"]) / abs(ref["lam"]))
            vec64r.append(_vec_err(u64r[a:b_], ref["u"]))
            if list(sw64[i]) != ref["sweeps"].tolist():
                apart.append({"graph": int(i), "gpu_sweeps": list(sw64[i]), "oracle_sweeps": ref["sweeps"].tolist()})
            rel64.append(abs(lam64[i] - ref["lam"]) / abs(ref["lam"]))
            vec64.append(_vec_err(u64[a:b_], ref["u"]))
            same += int(list(sw64[i]) == ref["sweeps"].tolist())
            rel32.append(abs(lam32[i] - ref["lam"]) / abs(ref["lam"]))
            ang32.append(_angle(u32[a:b_], ref["u"]))
        rel32, ang32 = np.array(rel32), np.array(ang32)
        out["batch_graphs_compared"] = len(idx)
        out["batch_sample"] = "all graphs" if len(idx) == G else f"seeded sample of {len(idx)} of {G}"
        out["batch_fp64_tolerance"] = {"vec_rel_err_max": max(vec64), "lambda2_rel_err_max": max(rel64),
                                       "same_sweeps": same, "gate": "vector <= 1e-10, lambda2 <= 1e-12",
                                       "within_gate": int(sum((v <= 1e-10) and (r <= 1e-12)
                                                              for v, r in zip(vec64, rel64))),
                                       "sweeps_apart": apart[:8],
                                       "note": "a graph whose stop cosine lies within rounding of 1 - tol "
                                               "on some level can stop one sweep apart from the oracle "
                                               "(float-float vs sequential FP64 sums); the replay "
                                               "comparison below takes the oracle's counts"}
        out["batch_fp64_replay"] = {"vec_rel_err_max": max(vec64r), "lambda2_rel_err_max": max(rel64r),
                                    "gate": "vector <= 1e-10, lambda2 <= 1e-12",
                                    "within_gate": int(sum((v <= 1e-10) and (r <= 1e-12)
                                                           for v, r in zip(vec64r, rel64r)))}
        out["batch_fp32_replay"] = {"lambda2_rel_err_max": float(rel32.max()),
                                    "lambda2_rel_err_p99": float(np.percentile(rel32, 99)),
                                    "angle_max": float(ang32.max()), "gate": "lambda2 <= 1e-6, angle <= 1e-4",
                                    "within_gate": int(((rel32 <= 1e-6) & (ang32 <= 1e-4)).sum())}
        tol32 = batch.get("_lam32_tol")
        if tol32 is not None:
            rt = np.array([abs(tol32[i] - res[i]["lam"]) / abs(res[i]["lam"]) for i in idx])
            at = np.array([_angle(batch["_u32_tol"][offs[i]:offs[i + 1]], res[i]["u"]) for i in idx])
            out["batch_fp32_tolerance_mode"] = {
                "lambda2_rel_err_max": float(rt.max()), "angle_max": float(at.max()),
                "within_1e-6_and_1e-4": int(((rt <= 1e-6) & (at <= 1e-4)).sum()),
                "note": "each form stops on its own cosine test: a stop one sweep earlier or later "
                        "moves the vector by up to arccos(1 - tol) = 1.4e-4 rad (the stop rule's "
                        "resolution), not by FP32 rounding; the replay comparison above isolates "
                        "precision"}
    # ---- Chung-Lu of the same recipe, small enough for the oracle
    if args.cl_oracle_n:
        o = res["chung_lu"]
        g = inputs.chung_lu(args.cl_oracle_n, seed=1412)
        nn = len(g[0]) - 1
        with cmg.Hierarchy(*g, seed=1412, precision="fp64") as h:
            u64c, l64c, st64c = h.fiedler()
        with cmg.Hierarchy(*g, seed=1412, precision="fp32", schedule="replay",
                           replay_sweeps=o["sweeps"].tolist()) as h:
            u32c, l32c, _ = h.fiedler()
            prec = h.level_precision()
        d = np.add.reduceat(g[2], g[0][:-1])
        bound = nn / (nn - 1) * float(d.min())
        from oracle import gershgorin
        gg = gershgorin(*g)
        out["chung_lu_small"] = {
            "workload": cl_workload(args.cl_oracle_n), "n": nn, "nnz": int(g[0][-1]),
            "fp64_vs_oracle": {"vec_rel_err": _vec_err(u64c, o["u"]),
                               "lambda2_rel_err": abs(l64c - o["lam"]) / abs(o["lam"]),
                               "same_sweeps": st64c["sweeps"] == o["sweeps"].tolist()},
            "fp32_replay_vs_oracle": {"lambda2_rel_err": abs(l32c - o["lam"]) / abs(o["lam"]),
                                      "angle_rad": _angle(u32c, o["u"]), "level_precision": prec},
            "oracle_lambda": o["lam"], "oracle_residual": o["res"], "g": gg,
            "lambda2_upper_bound": bound,
            "per_sweep_change_bound": bound / gg,
            "fp32_unit_roundoff": 2.0 ** -24,
            "note": ("lambda2 <= n/(n-1) min_i d_i (Fiedler's bound) is far below the returned "
                     "Rayleigh quotient: the cosine stop ends the power iteration as soon as a sweep "
                     "turns the vector by less than arccos(1 - tol), i.e. once the Rayleigh quotient "
                     "is below about g sqrt(2 tol); with g / lambda2 of order 1e5 and more, the "
                     "oracle and both GPU forms stop there alike (the method's behaviour, not a "
                     "precision effect); per sweep the Fiedler component changes by at most "
                     "lambda2 / g relative, a few FP32 ulps")}
    return out


KERNEL_KIND = {0: "smem", 1: "slice", 2: "slice+staged", 3: "tiled", 4: "two-phase", 5: "cluster"}

TABLE4 = os.path.join(ROOT, "tests", "golden", "table4_gcmg.txt")


def run_gcmg(args, stream):
    """Alg. 4 (geometric CMG): the Table 4 setting (2D, N 1025, beta 4, k0 1,
    coarsest 33 x 33) against the paper's printed errors and the oracle, and a
    3D grid in the regime the paper calls optimal (4 < beta < 2^3)."""
    import torch
    import oracle
    from paper_1412_0565_gb300 import cmg
    sid = stream.cuda_stream
    out = {}
    for name, (dim, N, J, beta, k0, steps) in (("table4_2d", (2, 1025, 5, 4.0, 1, 20)),
                                               ("grid3d", (3, 257, 5, 6.0, 1, 5))):
        u = torch.empty(N ** dim, dtype=torch.float64, device="cuda")
        ms = []
        for k in range(2 + steps):
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record(stream)
            _, r0, rk, ks = cmg.gcmg_grid(dim, N, J, beta=beta, k0=k0, u_out=u, stream=sid)
            e1.record(stream)
            e1.synchronize()
            if k >= 2:
                ms.append(e0.elapsed_time(e1))
        lam = [2 - 2 * np.cos(np.pi / ((N - 1) // 2 ** j + 1)) for j in range(J + 1)]
        n_j = [((N - 1) // 2 ** j + 1) ** dim for j in range(J + 1)]
        rec = {"workload": f"unit grid graph {N}^{dim}, {J} geometric coarsenings, beta {beta}, k0 {k0}",
               "value": len(ms) / (sum(ms) / 1e3), "unit": "solves/s", "ms": statistics.median(ms),
               "k": ks.tolist(), "vertex_sweeps": int(sum(k_ * m for k_, m in zip(ks.tolist(), n_j))),
               "err_r0": [abs(l - r) for l, r in zip(lam, r0)], "err_rk": [abs(l - r) for l, r in zip(lam, rk)]}
        if dim * N ** dim <= 2_200_000 and not args.no_oracle_checks:
            ref = oracle.gcmg_grid(dim, N, J, beta=beta, k0=k0)
            uh = u.cpu().numpy()
            rec["vs_oracle"] = {"rq_rel_err_max": float(max(np.max(np.abs(r0 - ref["r0"]) / ref["r0"]),
                                                            np.max(np.abs(rk - ref["rk"]) / ref["rk"]))),
                                "vec_rel_err": _vec_err(uh, ref["u"])}
        if name == "table4_2d":
            with open(TABLE4) as f:
                rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
            rec["table4"] = {"paper_err_r0": [float(r[1]) for r in rows],
                             "paper_err_rk": [float(r[2]) for r in rows],
                             "max_rel_diff": max(max(abs(rec["err_r0"][int(r[0])] - float(r[1])) / float(r[1]),
                                                     abs(rec["err_rk"][int(r[0])] - float(r[2])) / float(r[2]))
                                                 for r in rows)}
        out[name] = rec
    return out


def run_schedule_study(args, stream):
    """The fixed schedule k_j = ceil(k0 beta^j) of Sec. 3 (Theorem 3.10 and
    its cost corollary) with the algebraic hierarchy, on unit-weight grids
    whose lambda_2 is known in closed form: accuracy (relative error of the
    returned Rayleigh quotient, residual) against cost (sum_j k_j n_j and
    k_j nnz_j, device time) for a range of beta and k0, beside the paper's
    tolerance rule.  With geometric coarsening (n_j / n_{j+1} = 2^d, h_{j+1}
    / h_j = 2) the theory's window is 4 < beta < 2^d; heavy edge coarsening
    shrinks a level about 3x, so the analogous window is
    (n_j/n_{j+1})^(2/d) < beta < n_j/n_{j+1}, and the schedules tried stop
    where the coarse levels' sweep counts explode (a configuration whose
    predicted total exceeds the caps below is reported as skipped)."""
    import torch
    from paper_1412_0565_gb300 import cmg, inputs
    sid = stream.cuda_stream
    out = {}
    for name, (graph, N) in (("grid2d_1024", (lambda: inputs.grid2d(1024, 1024, "unit"), 1024)),
                              ("grid3d_100", (lambda: inputs.grid3d(100, 100, 100, "unit"), 100))):
        rp, col, w = graph()
        lam_exact = 2 - 2 * np.cos(np.pi / N)
        drp, dcol, dw = (torch.from_numpy(a).cuda() for a in (rp, col, w))
        u = torch.empty(len(rp) - 1, dtype=torch.float64, device="cuda")
        rows = []
        with cmg.Hierarchy(drp, dcol, dw, stream=sid, seed=1412) as h:
            ns0 = h.sizes()[0]
        ratio = float(np.exp(np.mean(np.log(np.array(ns0[:-2], float) / np.array(ns0[1:-1], float)))))
        runs = [("tol", None, None)] + [("fixed", b, k0) for b in args.study_betas for k0 in args.study_k0s]
        for sched, beta, k0 in runs:
            if sched == "fixed":
                kp = [int(np.ceil(k0 * beta ** j)) for j in range(len(ns0))]
                if sum(kp) > 200_000 or sum(a * b for a, b in zip(kp, ns0)) > 300 * ns0[0]:
                    rows.append({"schedule": sched, "beta": beta, "k0": k0, "skipped": True,
                                 "predicted_sweeps": kp})
                    continue
            kw = dict(seed=1412, precision="fp64", timing=1)
            if sched == "fixed":
                kw.update(schedule="fixed", beta=float(beta), k0=int(k0))
            with cmg.Hierarchy(drp, dcol, dw, stream=sid, **kw) as h:
                ms = []
                for rep in range(3):
                    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                    e0.record(stream)
                    _, lam, st = h.fiedler(u_out=u, stream=sid)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
            ks, ns, nz = st["sweeps"], st["n"], st["nnz"]
            rows.append({"schedule": sched, "beta": beta, "k0": k0, "sweeps": ks,
                         "lambda2_rel_err": (lam - lam_exact) / lam_exact, "residual": st["residual"],
                         "cost_kn": int(sum(a * b for a, b in zip(ks, ns))),
                         "cost_knnz": int(sum(a * b for a, b in zip(ks, nz))),
                         "solve_ms": min(ms)})
        out[name] = {"n": len(rp) - 1, "lambda2_exact": lam_exact, "levels_n": ns0,
                     "mean_coarsening_ratio": ratio,
                     "window_beta": [ratio ** (2.0 / (2 if "2d" in name else 3)), ratio], "runs": rows}
    return out


def run_c1(args, stream, flush):
    """Config 1: the 64 x 64 unit grid (FP64): solves/s, latency, and the
    result against the closed form (lambda2 = 2 - 2 cos(pi/64), double) and
    the oracle."""
    import torch
    import oracle
    from paper_1412_0565_gb300 import cmg, inputs
    rp, col, w = inputs.grid2d(64, 64, "unit")
    n = len(rp) - 1
    sid = stream.cuda_stream
    drp, dcol, dw = (torch.from_numpy(a).cuda() for a in (rp, col, w))
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    opts = cmg.options(seed=1412, precision="fp64")
    ms = []
    for k in range(5 + args.c1_steps):
        flush.zero_()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        with cmg.Hierarchy(drp, dcol, dw, opts=opts, stream=sid) as h:
            _, lam, st = h.fiedler(u_out=u, stream=sid)
        e1.record(stream)
        e1.synchronize()
        if k >= 5:
            ms.append(e0.elapsed_time(e1))
    uh = u.cpu().numpy()
    ref_u, ref_lam, _, _, ref = oracle.fiedler(rp, col, w, seed=1412)
    lam_exact = 2 - 2 * np.cos(np.pi / 64)
    x = np.tile(np.arange(64), 64)
    y = np.repeat(np.arange(64), 64)
    Q = np.stack([np.cos(np.pi * (x + 0.5) / 64), np.cos(np.pi * (y + 0.5) / 64)], axis=1)
    Q, _ = np.linalg.qr(Q)
    srt = sorted(ms)
    return {"workload": "grid2d_64x64_unit (n 4,096, nnz 16,128), FP64", "steps": len(ms),
            "value": len(ms) / (sum(ms) / 1e3), "unit": UNIT,
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
            "sweeps": st["sweeps"], "lambda2": lam, "residual": st["residual"],
            "vs_oracle": {"vec_rel_err": _vec_err(uh, ref_u), "lambda2_rel_err": abs(lam - ref_lam) / ref_lam,
                          "same_sweeps": st["sweeps"] == ref["sweeps"].tolist()},
            "vs_closed_form": {"lambda2_exact": lam_exact, "lambda2_rel_err": (lam - lam_exact) / lam_exact,
                               "fiedler_space_residual": float(np.linalg.norm(uh - Q @ (Q.T @ uh))),
                               "note": "default (tolerance) mode is an approximation: lambda~ >= lambda2"}}


BATCH_WORKLOAD = ("4096 graphs, n log-uniform [500, 20000], random geometric (mean degree 8) / "
                  "near-square 2D grid / Barabasi-Albert m=4 round-robin, U[0.5,1.5] weights, seed 1412")
SERVE_WORKLOAD = ("requests drawn uniformly from {P} graphs with log n ~ Normal truncated to "
                  "[ln 1e3, ln 2e6] (families and weights as the batch), Poisson arrivals at rho x the "
                  "closed-loop saturation rate")


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

    res["fp32_vs_gpu_fp64_replay"] = compare(lam32, u32)
    res["fp32_vs_gpu_fp64_replay"]["note"] = ("FP32 sweeps with the GPU FP64 run's per-graph, per-level "
                                              "sweep counts, every graph (accuracy_vs_oracle compares "
                                              "with the CPU oracle)")
    res["fp32_vs_gpu_fp64_tolerance_mode"] = compare(lam32_tol, u32_tol)
    # arrays for the oracle comparison (removed before printing)
    res["_graphs"], res["_union"] = graphs, (rp, col, w, offs)
    res["_u64"], res["_lam64"], res["_sweeps64"] = u64, lam64, sweeps64
    res["_u32_tol"], res["_lam32_tol"] = u32_tol, lam32_tol
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
    d = np.add.reduceat(w, rp[:-1])
    bound = n / (n - 1) * float(d.min())
    out = {"workload": cl_workload(args.cl_n), "n": n, "nnz": nnz, "max_degree": int(deg.max()),
           "generate_s": round(gen_s, 1), "lambda2_upper_bound": bound,
           "lambda2_upper_bound_note": "Fiedler: lambda2 <= n/(n-1) min_i d_i (weighted degree)"}
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
            h_prec = h.level_precision()
            h.close()
            if k >= args.cl_warmup:
                ms.append(e0.elapsed_time(e1))
                setup.append(e0.elapsed_time(em))
        by0 = st["sweeps"][0] * ((8 if prec == "fp32" else 12) * st["nnz"][0] + (12 if prec == "fp32" else 20) * st["n"][0])
        res[prec] = {"u": u.cpu().numpy(), "lam": lam, "sweeps": st["sweeps"]}
        out[prec] = {"value": len(ms) / (sum(ms) / 1e3), "unit": "solves/s", "ms_per_step": statistics.mean(ms),
                     "level_precision": h_prec,
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
    lam = res["fp64"]["lam"]
    out["meets_lambda2_target"] = bool(lam <= bound * (1 + 1e-6))
    out["accuracy_note"] = (
        f"the returned Rayleigh quotient ({lam:.4g}) is {lam / bound:.0f} times Fiedler's upper bound "
        f"on lambda2 ({bound:.4g}): with the paper's stop rule (cos >= 1 - 1e-8) the power iteration "
        "ends once a sweep turns the vector by less than 1.4e-4 rad, which on this graph happens long "
        "before the vector approaches the Fiedler vector (g / lambda2 >= 1e6); these solves/s are not "
        "at the lambda2 <= 1e-6 target.  The same stop happens in the oracle (accuracy_vs_oracle."
        "chung_lu_small)")
    c2 = abs(float(np.dot(res["fp32"]["u"], u64))) / (np.linalg.norm(res["fp32"]["u"]) * np.linalg.norm(u64))
    out["fp32_vs_fp64_tolerance_mode"] = {
        "lambda2_rel": abs(res["fp32"]["lam"] - res["fp64"]["lam"]) / abs(res["fp64"]["lam"]),
        "angle": float(np.arccos(min(1.0, c2)))}
    return out


KERNEL_KIND = {0: "smem", 1: "slice", 2: "slice+staged", 3: "tiled", 4: "two-phase", 5: "cluster"}


def run_serving(args):
    """Config 5, the request loop: Poisson arrivals at rho x the closed-loop
    saturation rate for each rho, on a trace of requests drawn from a pool of
    graphs whose sizes are lognormal over 1e3 .. 2e6 vertices; FP32 server
    (batching of cold small graphs, resident hierarchies) against a plain
    FP64 server (no batching) at the same loads; p50/p99 latency, job mix,
    device memory measured against the budget, and the FP32 results against
    the CPU oracle on the served graphs small enough for it."""
    from paper_1412_0565_gb300 import cmg, inputs
    graphs = inputs.serving_graphs(args.serve_graphs, workers=_pool_workers())
    rng = np.random.default_rng(1412)
    trace = rng.integers(0, len(graphs), size=args.serve_requests)
    sizes = [len(g[0]) - 1 for g in graphs]
    out = {"workload": SERVE_WORKLOAD.format(P=len(graphs)), "requests_per_load": int(len(trace)),
           "distinct_graphs": len(graphs), "distinct_in_trace": int(len(set(trace.tolist()))),
           "n_max": int(max(sizes)), "n_median": int(np.median(sizes)),
           "cut": (f"{len(trace)} requests per load from a pool of {len(graphs)} graphs (the configured "
                   "10,000-request trace would take tens of minutes per load)"),
           "min_batch": args.serve_min_batch}
    servers = (("fp32", dict(workers=4, max_batch=256, batch_max_n=8192, min_batch=args.serve_min_batch),
                "fp32", args.serve_rhos),
               ("fp64_plain", dict(workers=4, max_batch=1), "fp64", [0.8]))
    lam_served = {}
    for name, cfg, prec, rhos in servers:
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
        rec = {"saturation_solves_s": sat, "saturation_jobs": {k: st[k] for k in
                                                              ("single_jobs", "batch_jobs", "warm_jobs")},
               "loads": {}}
        for rho in rhos:
            rs2, dt2, st2 = run(rho * sat)
            lat = np.array([r["latency_ms"] for r in rs2])
            rec["loads"][str(rho)] = {
                "offered_rate": rho * sat, "achieved_solves_s": len(trace) / dt2,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "warm_fraction": float(np.mean([r["warm"] for r in rs2])),
                "batched_fraction": float(np.mean([r["batch_size"] > 1 for r in rs2])),
                "jobs": {k: st2[k] for k in ("single_jobs", "batch_jobs", "warm_jobs", "evictions")},
                "reserved_peak_bytes": st2["peak_bytes"], "measured_peak_bytes": st2["measured_peak_bytes"],
                "budget_bytes": st2["budget_bytes"],
                "within_budget": bool(st2["measured_peak_bytes"] <= st2["budget_bytes"])}
            if rho == 0.8:
                lam_served[name] = {int(k): r["lambda2"] for k, r in zip(trace, rs2)}
        out[name] = rec
    common = sorted(set(lam_served["fp32"]) & set(lam_served["fp64_plain"]))
    rel = np.array([abs(lam_served["fp32"][k] - lam_served["fp64_plain"][k]) / abs(lam_served["fp64_plain"][k])
                    for k in common])
    out["fp32_vs_fp64_lambda2_rel_tolerance_mode"] = {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)),
                                                      "note": "each form stops on its own cosine test"}
    # ---- a burst of small-graph requests (the batch's families and sizes,
    # up to 8,192 vertices): Poisson arrivals far above one graph's solve
    # rate, so cold requests pile up and the FP32 server batches them
    idx = [i for i, nv in enumerate(inputs.batch_sizes(4096)) if nv <= 8192][:args.serve_burst_graphs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=_pool_workers(), mp_context=mp.get_context("spawn")) as ex:
        small_g = list(ex.map(inputs.batch_graph, idx, chunksize=16))
    burst = {"workload": (f"{len(small_g)} distinct graphs of the 4,096-graph batch's families with at "
                          f"most 8,192 vertices, each requested once, Poisson arrivals at "
                          f"{args.serve_burst_rate:.0f}/s")}
    for name, cfg, prec in (("fp32_batched", dict(workers=4, max_batch=256, batch_max_n=8192, min_batch=32), "fp32"),
                            ("fp64_plain", dict(workers=4, max_batch=1), "fp64")):
        with cmg.Server(seed=1412, precision=prec, **cfg) as srv:
            ids = [srv.add_graph(*g) for g in small_g]
            arr = np.cumsum(np.random.default_rng(11).exponential(1.0 / args.serve_burst_rate, size=len(ids)))
            t0 = time.perf_counter()
            tickets = []
            for gid, ta in zip(ids, arr):
                d = t0 + ta - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets.append(srv.submit(gid, want_vector=False))
            rs = [srv.wait(t)[1] for t in tickets]
            dt = time.perf_counter() - t0
            st = srv.stats()
        lat = np.array([r["latency_ms"] for r in rs])
        burst[name] = {"solves_s": len(rs) / dt, "p50_ms": float(np.percentile(lat, 50)),
                       "p99_ms": float(np.percentile(lat, 99)),
                       "batched_fraction": float(np.mean([r["batch_size"] > 1 for r in rs])),
                       "jobs": {k: st[k] for k in ("single_jobs", "batch_jobs", "warm_jobs")},
                       "measured_peak_bytes": st["measured_peak_bytes"]}
    burst["fp32_batched_over_fp64_plain"] = burst["fp32_batched"]["solves_s"] / burst["fp64_plain"]["solves_s"]
    out["small_graph_burst"] = burst
    # precision alone against the oracle: the served graphs up to 50,000
    # vertices, FP32 sweeps replaying the oracle's per-level sweep counts
    import oracle
    small = [i for i in sorted(set(trace.tolist())) if sizes[i] <= 50_000][:args.serve_oracle_sample]
    lam_rel, ang = [], []
    for i in small:
        g = graphs[i]
        ref = oracle.Hierarchy(*g, seed=1412).solve()
        u32, l32, _ = cmg.fiedler(*g, seed=1412, precision="fp32", schedule="replay",
                                  replay_sweeps=ref["sweeps"].tolist())
        lam_rel.append(abs(l32 - ref["lam"]) / abs(ref["lam"]))
        ang.append(_angle(u32, ref["u"]))
    out["fp32_replay_vs_oracle"] = {"graphs": len(lam_rel), "lambda2_rel_err_max": max(lam_rel),
                                    "angle_max": max(ang), "gate": "lambda2 <= 1e-6, angle <= 1e-4",
                                    "within_gate": int(sum((r <= 1e-6) and (a <= 1e-4)
                                                           for r, a in zip(lam_rel, ang)))}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--no-gcmg", action="store_true")
    ap.add_argument("--no-study", action="store_true")
    ap.add_argument("--study-betas", type=float, nargs="+", default=[1.5, 2.0, 2.5, 3.0, 3.5, 4.0])
    ap.add_argument("--study-k0s", type=int, nargs="+", default=[1, 4, 16])
    ap.add_argument("--c1-steps", type=int, default=50)
    ap.add_argument("--no-oracle-checks", action="store_true")
    ap.add_argument("--batch-oracle-sample", type=int, default=0,
                    help="compare a seeded sample of this many batch graphs with the oracle (0: all)")
    ap.add_argument("--cl-oracle-n", type=int, default=250_000,
                    help="Chung-Lu vertices (before the largest component) of the oracle comparison (0: skip)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-plain-sample", type=int, default=32)
    ap.add_argument("--serve-graphs", type=int, default=96)
    ap.add_argument("--serve-requests", type=int, default=240)
    ap.add_argument("--serve-rhos", type=float, nargs="+", default=[0.5, 0.8, 0.95])
    ap.add_argument("--serve-min-batch", type=int, default=8)
    ap.add_argument("--serve-oracle-sample", type=int, default=24)
    ap.add_argument("--serve-burst-graphs", type=int, default=1024)
    ap.add_argument("--serve-burst-rate", type=float, default=4000.0)
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
