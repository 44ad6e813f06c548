"""Thin ctypes binding of libcmg (the C-ABI in include/cmg.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Host buffers are numpy arrays; device buffers are torch CUDA tensors (torch is
used for device memory and streams, nothing else).  There is no CPU fallback:
if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

CMG_MAX_LEVELS = 64
MEM_HOST, MEM_DEVICE = 0, 1
FP64, FP32_SWEEP = 0, 1
SCHEDULES = {"tol": 0, "fixed": 1, "replay": 2}

STATUS = {
    0: "OK", 1: "WARN_MAXITER", -1: "ERR_INVALID_ARG", -2: "ERR_NOT_SYMMETRIC",
    -3: "ERR_SELF_LOOP", -4: "ERR_BAD_WEIGHT", -5: "ERR_ISOLATED_VERTEX", -6: "ERR_TOO_SMALL",
    -7: "ERR_OOM", -8: "ERR_CUDA", -9: "ERR_DEVICE_TIMEOUT", -10: "ERR_BAD_CSR",
    -11: "ERR_TOO_LARGE", -12: "ERR_TIMEOUT",
}

# every symbol include/cmg.h declares
EXPORTS = [
    "cmg_options_default", "cmg_status_string", "cmg_version", "cmg_setup", "cmg_fiedler",
    "cmg_hierarchy_info", "cmg_level_kernels", "cmg_level_precision", "cmg_hierarchy_device_bytes", "cmg_estimate_device_bytes",
    "cmg_get_aggregates", "cmg_get_level_csr", "cmg_free", "cmg_heaviest_neighbour",
    "cmg_visit_ranks", "cmg_hec_aggregate", "cmg_power_sweeps", "cmg_rayleigh_residual",
    "cmg_power_sweeps_noalloc", "cmg_kernel_launches", "cmg_debug_fail_alloc_after", "cmg_debug_stall_barrier",
    "cmg_setup_batch", "cmg_fiedler_batch", "cmg_batch_info", "cmg_batch_stats",
    "cmg_batch_get_aggregates", "cmg_batch_get_level_csr", "cmg_batch_set_replay",
    "cmg_batch_config", "cmg_batch_autotune", "cmg_batch_level_ms", "cmg_batch_device_bytes",
    "cmg_batch_free", "cmg_server_config_default", "cmg_server_create", "cmg_server_add_graph",
    "cmg_server_submit", "cmg_server_submit_ex", "cmg_solve_options_default", "cmg_fiedler_ex",
    "cmg_server_wait", "cmg_gcmg_grid", "cmg_eigenpairs", "cmg_server_wait_for", "cmg_server_get_stats",
    "cmg_server_destroy",
]

NOALLOC_MAX_N = 262144
NOALLOC_MAX_NNZ = 4194304


class CmgError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{what}: {self.name} ({status})" if what else f"{self.name} ({status})")


class Options(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("beta", C.c_double), ("seed", C.c_uint64),
        ("coarse_size", C.c_int32), ("max_levels", C.c_int32), ("precision", C.c_int32),
        ("schedule", C.c_int32), ("k0", C.c_int32), ("max_sweeps", C.c_int32),
        ("max_sweeps_coarsest", C.c_int32), ("validate", C.c_int32), ("timing", C.c_int32),
        ("reserved", C.c_int32), ("replay_sweeps", C.c_int32 * CMG_MAX_LEVELS),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("lambda2", C.c_double), ("residual", C.c_double), ("levels", C.c_int32),
        ("status", C.c_int32), ("n", C.c_int64 * CMG_MAX_LEVELS),
        ("nnz", C.c_int64 * CMG_MAX_LEVELS), ("sweeps", C.c_int32 * CMG_MAX_LEVELS),
        ("cos_final", C.c_double * CMG_MAX_LEVELS), ("level_ms", C.c_double * CMG_MAX_LEVELS),
        ("finalize_ms", C.c_double),
    ]

    def as_dict(self):
        L = self.levels
        return {"lambda2": self.lambda2, "residual": self.residual, "levels": L,
                "status": STATUS.get(self.status, self.status),
                "n": list(self.n[:L]), "nnz": list(self.nnz[:L]),
                "sweeps": list(self.sweeps[:L]), "cos_final": list(self.cos_final[:L]),
                "level_ms": list(self.level_ms[:L]), "finalize_ms": self.finalize_ms}


class SolveOptions(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("x0", C.c_void_p), ("x0_mem", C.c_int32),
                ("x0_level", C.c_int32), ("reserved", C.c_int32 * 4)]


class BatchShape(C.Structure):
    _fields_ = [("threads_per_graph", C.c_int32), ("lanes_per_row", C.c_int32),
                ("graphs_per_cta", C.c_int32), ("stage_csr", C.c_int32)]

    def as_tuple(self):
        return (self.threads_per_graph, self.lanes_per_row, self.graphs_per_cta, self.stage_csr)


class ServerConfig(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_batch", C.c_int32), ("batch_max_n", C.c_int64),
                ("mem_budget", C.c_uint64), ("keep_resident", C.c_int32), ("min_batch", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("warm", C.c_int32),
                ("pad", C.c_int32), ("lambda2", C.c_double), ("residual", C.c_double),
                ("submit_ns", C.c_uint64), ("admit_ns", C.c_uint64), ("done_ns", C.c_uint64)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, self.status), "batch_size": self.batch_size,
                "warm": bool(self.warm), "lambda2": self.lambda2, "residual": self.residual,
                "latency_ms": (self.done_ns - self.submit_ns) / 1e6,
                "queue_ms": (self.admit_ns - self.submit_ns) / 1e6}


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("single_jobs", C.c_int64), ("batch_jobs", C.c_int64),
                ("warm_jobs", C.c_int64), ("evictions", C.c_int64), ("resident", C.c_int64),
                ("peak_bytes", C.c_uint64), ("used_bytes", C.c_uint64), ("budget_bytes", C.c_uint64),
                ("measured_peak_bytes", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Loads libcmg.so (building it in-tree first when its sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_stale else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libcmg.so not found at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        V = C.c_void_p
        I32, I64, F64 = C.c_int32, C.c_int64, C.c_double
        P = C.POINTER
        sig = {
            "cmg_options_default": (I32, [P(Options)]),
            "cmg_status_string": (C.c_char_p, [I32]),
            "cmg_version": (C.c_char_p, []),
            "cmg_setup": (I32, [I64, V, V, V, I32, P(Options), V, P(V)]),
            "cmg_fiedler": (I32, [V, V, I32, P(F64), P(Stats), V]),
            "cmg_hierarchy_info": (I32, [V, P(I32), V, V]),
            "cmg_level_kernels": (I32, [V, V, V]),
            "cmg_hierarchy_device_bytes": (I32, [V, P(C.c_size_t)]),
            "cmg_estimate_device_bytes": (I32, [I64, I64, I32, P(C.c_size_t)]),
            "cmg_get_aggregates": (I32, [V, I32, V]),
            "cmg_get_level_csr": (I32, [V, I32, V, V, V, P(F64)]),
            "cmg_free": (I32, [V]),
            "cmg_heaviest_neighbour": (I32, [I32, V, V, V, V, V]),
            "cmg_visit_ranks": (I32, [I32, C.c_uint64, I32, V, V]),
            "cmg_hec_aggregate": (I32, [I32, V, V, V, V, V, P(I64), V]),
            "cmg_power_sweeps": (I32, [I32, V, V, V, F64, V, I32, V, P(F64), V]),
            "cmg_rayleigh_residual": (I32, [I32, V, V, V, V, P(F64), P(F64), V]),
            "cmg_power_sweeps_noalloc": (I32, [I32, V, V, V, F64, V, I32, V, P(F64), V]),
            "cmg_kernel_launches": (I32, [P(C.c_uint64)]),
            "cmg_debug_fail_alloc_after": (I32, [I64]),
            "cmg_debug_stall_barrier": (I32, [I64, I32]),
            "cmg_setup_batch": (I32, [I32, V, V, V, V, I32, P(Options), V, P(V)]),
            "cmg_fiedler_batch": (I32, [V, V, I32, V, V, V, V]),
            "cmg_batch_info": (I32, [V, P(I32), P(I32), I32, P(I64), P(I64)]),
            "cmg_batch_stats": (I32, [V, I32, P(Stats)]),
            "cmg_batch_get_aggregates": (I32, [V, I32, I32, V]),
            "cmg_batch_get_level_csr": (I32, [V, I32, I32, V, V, V, P(F64)]),
            "cmg_batch_set_replay": (I32, [V, V]),
            "cmg_batch_config": (I32, [V, I32, I32, P(BatchShape)]),
            "cmg_batch_autotune": (I32, [V, V]),
            "cmg_batch_level_ms": (I32, [V, I32, P(F64)]),
            "cmg_batch_device_bytes": (I32, [V, P(C.c_size_t)]),
            "cmg_batch_free": (I32, [V]),
            "cmg_server_config_default": (I32, [P(ServerConfig)]),
            "cmg_server_create": (I32, [P(ServerConfig), P(Options), P(V)]),
            "cmg_server_add_graph": (I32, [V, I64, V, V, V, P(I64)]),
            "cmg_server_submit": (I32, [V, I64, V, P(I64)]),
            "cmg_level_precision": (I32, [V, V]),
            "cmg_gcmg_grid": (I32, [I32, I32, I32, F64, I32, V, I32, V, V, V, V]),
            "cmg_eigenpairs": (I32, [V, I32, V, V, I32, V, V, P(Stats), V]),
            "cmg_server_submit_ex": (I32, [V, I64, P(SolveOptions), V, P(I64)]),
            "cmg_solve_options_default": (I32, [V, P(SolveOptions)]),
            "cmg_fiedler_ex": (I32, [V, P(SolveOptions), V, I32, P(F64), P(Stats), V]),
            "cmg_server_wait": (I32, [V, I64, P(Request)]),
            "cmg_server_wait_for": (I32, [V, I64, I64, P(Request)]),
            "cmg_server_get_stats": (I32, [V, P(ServerStats)]),
            "cmg_server_destroy": (I32, [V]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(st: int, what: str, allow_warn: bool = True):
    if st == 0 or (allow_warn and st == 1):
        return st
    raise CmgError(st, what)


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def _ptr(x):
    """(pointer, mem) of a numpy array or torch tensor (contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return C.c_void_p(x.ctypes.data), MEM_HOST
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return C.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST)
    raise TypeError(type(x))


def options(**kw) -> Options:
    o = Options()
    _check(load().cmg_options_default(C.byref(o)), "cmg_options_default")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "fp32": FP32_SWEEP}[v]
        if k == "schedule" and isinstance(v, str):
            v = SCHEDULES[v]
        if k == "replay_sweeps":
            arr = (C.c_int32 * CMG_MAX_LEVELS)()
            for i, x in enumerate(v):
                arr[i] = int(x)
            o.replay_sweeps = arr
            continue
        setattr(o, k, v)
    return o


def status_string(st: int) -> str:
    return load().cmg_status_string(st).decode()


def version() -> str:
    return load().cmg_version().decode()


def estimate_device_bytes(n: int, nnz: int, precision=FP64) -> int:
    out = C.c_size_t()
    _check(load().cmg_estimate_device_bytes(n, nnz, precision, C.byref(out)), "estimate")
    return out.value


def _as_inputs(row_ptr, col, w):
    if isinstance(row_ptr, np.ndarray):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
    return row_ptr, col, w


class Hierarchy:
    """Alg. 1 Step 1 (setup) resident on the GPU; `fiedler()` runs Steps 2-3."""

    def __init__(self, row_ptr, col, w, *, opts: Options | None = None, stream=None, **kw):
        lib = load()
        if opts is None:
            opts = options(**kw)
        self.opts = opts
        row_ptr, col, w = _as_inputs(row_ptr, col, w)
        self._keep = (row_ptr, col, w)
        p_rp, mem = _ptr(row_ptr)
        p_col, mem2 = _ptr(col)
        p_w, mem3 = _ptr(w)
        if not (mem == mem2 == mem3):
            raise ValueError("row_ptr, col and w must all be host or all be device buffers")
        n = (row_ptr.shape[0] if hasattr(row_ptr, "shape") else len(row_ptr)) - 1
        h = C.c_void_p()
        self._h = None
        st = lib.cmg_setup(n, p_rp, p_col, p_w, mem, C.byref(opts), _stream(stream), C.byref(h))
        _check(st, "cmg_setup", allow_warn=False)
        self._h = h
        self._keep = None
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            load().cmg_free(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def levels(self) -> int:
        L = C.c_int32()
        _check(load().cmg_hierarchy_info(self._h, C.byref(L), None, None), "info")
        return L.value

    def sizes(self):
        L = self.levels
        n = np.zeros(L, dtype=np.int64)
        nnz = np.zeros(L, dtype=np.int64)
        _check(load().cmg_hierarchy_info(self._h, None, C.c_void_p(n.ctypes.data),
                                         C.c_void_p(nnz.ctypes.data)), "info")
        return n.tolist(), nnz.tolist()

    def level_kernels(self):
        """Per level: (kind, staged) -- kind 0 shared-memory kernel, 1 slice
        kernel, 2 slice kernel with `staged` iterate entries staged in shared
        memory, 3 row-tile kernel, 4 two-phase kernel, 5 cluster kernel."""
        L = self.levels
        kind = np.zeros(L, dtype=np.int32)
        staged = np.zeros(L, dtype=np.int32)
        _check(load().cmg_level_kernels(self._h, C.c_void_p(kind.ctypes.data),
                                        C.c_void_p(staged.ctypes.data)), "level_kernels")
        return kind.tolist(), staged.tolist()

    def eigenpairs(self, k: int, *, seed=None, U_out=None, stream=None):
        """cmg_eigenpairs: k approximate eigenpairs by the cascade with block
        power iteration.  Returns (U [k, n] numpy or the given torch CUDA
        tensor of k*n float64, lambda[k], residual[k], stats dict)."""
        if U_out is None:
            U_out = np.empty((k, self.n), dtype=np.float64)
        p_u, mem = _ptr(U_out)
        lam = np.zeros(k)
        res = np.zeros(k)
        stats = Stats()
        so = None
        if seed is not None:
            so = SolveOptions()
            _check(load().cmg_solve_options_default(self._h, C.byref(so)), "solve_options")
            so.seed = int(seed)
        _check(load().cmg_eigenpairs(self._h, int(k), C.byref(so) if so is not None else None, p_u, mem,
                                     C.c_void_p(lam.ctypes.data), C.c_void_p(res.ctypes.data),
                                     C.byref(stats), _stream(stream)), "cmg_eigenpairs")
        return U_out, lam, res, stats.as_dict()

    def level_precision(self):
        """Per level: "fp32" or "fp64" sweeps."""
        p = np.zeros(self.levels, dtype=np.int32)
        _check(load().cmg_level_precision(self._h, C.c_void_p(p.ctypes.data)), "level_precision")
        return ["fp32" if x == 1 else "fp64" for x in p.tolist()]

    def device_bytes(self) -> int:
        b = C.c_size_t()
        _check(load().cmg_hierarchy_device_bytes(self._h, C.byref(b)), "bytes")
        return b.value

    def aggregates(self, level: int) -> np.ndarray:
        n = self.sizes()[0][level]
        a = np.empty(n, dtype=np.int32)
        _check(load().cmg_get_aggregates(self._h, level, C.c_void_p(a.ctypes.data)), "aggregates")
        return a

    def level_csr(self, level: int):
        ns, nnzs = self.sizes()
        rp = np.empty(ns[level] + 1, dtype=np.int64)
        col = np.empty(nnzs[level], dtype=np.int32)
        w = np.empty(nnzs[level], dtype=np.float64)
        g = C.c_double()
        _check(load().cmg_get_level_csr(self._h, level, C.c_void_p(rp.ctypes.data),
                                        C.c_void_p(col.ctypes.data), C.c_void_p(w.ctypes.data),
                                        C.byref(g)), "level_csr")
        return rp, col, w, g.value

    def fiedler(self, u_out=None, stream=None, *, seed=None, x0=None, x0_level=0):
        """Returns (u, lambda2, stats dict).  u_out: numpy (host) or torch CUDA
        tensor (device) of n float64; allocated on the host when None.
        seed / x0 / x0_level: a re-solve with another Gaussian start, or from
        a start vector on level x0_level (cmg_fiedler_ex); x0 is numpy (host)
        or a torch CUDA float64 tensor."""
        if u_out is None:
            u_out = np.empty(self.n, dtype=np.float64)
        p_u, mem = _ptr(u_out)
        lam = C.c_double()
        stats = Stats()
        if seed is None and x0 is None:
            st = load().cmg_fiedler(self._h, p_u, mem, C.byref(lam), C.byref(stats), _stream(stream))
        else:
            so = SolveOptions()
            _check(load().cmg_solve_options_default(self._h, C.byref(so)), "solve_options")
            if seed is not None:
                so.seed = int(seed)
            keep = None
            if x0 is not None:
                if isinstance(x0, np.ndarray):
                    x0 = keep = np.ascontiguousarray(x0, dtype=np.float64)
                p_x, xmem = _ptr(x0)
                so.x0, so.x0_mem, so.x0_level = p_x, xmem, int(x0_level)
            st = load().cmg_fiedler_ex(self._h, C.byref(so), p_u, mem, C.byref(lam), C.byref(stats),
                                       _stream(stream))
            del keep
        _check(st, "cmg_fiedler")
        return u_out, lam.value, stats.as_dict()


def fiedler(row_ptr, col, w, *, stream=None, **kw):
    """Alg. 1 end to end: setup + solve.  Returns (u, lambda2, stats)."""
    with Hierarchy(row_ptr, col, w, stream=stream, **kw) as h:
        return h.fiedler(stream=stream)


class Batch:
    """Batched Alg. 1 for many graphs: the union CSR (union column indices)
    with vertex offsets `graph_offsets` (int64[G+1]).  `fiedler()` solves
    every graph; results use the union layout."""

    def __init__(self, graph_offsets, row_ptr, col, w, *, opts: Options | None = None,
                 stream=None, **kw):
        lib = load()
        if opts is None:
            opts = options(**kw)
        self.opts = opts
        offs = np.ascontiguousarray(graph_offsets, dtype=np.int64)
        row_ptr, col, w = _as_inputs(row_ptr, col, w)
        p_rp, mem = _ptr(row_ptr)
        p_col, mem2 = _ptr(col)
        p_w, mem3 = _ptr(w)
        if not (mem == mem2 == mem3):
            raise ValueError("row_ptr, col and w must all be host or all be device buffers")
        self.G = len(offs) - 1
        self.offsets = offs
        self.N = int(offs[-1])
        b = C.c_void_p()
        self._b = None
        st = lib.cmg_setup_batch(self.G, C.c_void_p(offs.ctypes.data), p_rp, p_col, p_w, mem,
                                 C.byref(opts), _stream(stream), C.byref(b))
        _check(st, "cmg_setup_batch", allow_warn=False)
        self._b = b

    def close(self):
        if getattr(self, "_b", None):
            load().cmg_batch_free(self._b)
            self._b = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def union_levels(self) -> int:
        L = C.c_int32()
        _check(load().cmg_batch_info(self._b, None, C.byref(L), -1, None, None), "batch_info")
        return L.value

    def union_size(self, level: int):
        n, nnz = C.c_int64(), C.c_int64()
        _check(load().cmg_batch_info(self._b, None, None, level, C.byref(n), C.byref(nnz)), "info")
        return n.value, nnz.value

    def stats(self, graph: int) -> dict:
        s = Stats()
        _check(load().cmg_batch_stats(self._b, graph, C.byref(s)), "batch_stats")
        return s.as_dict()

    def aggregates(self, graph: int, level: int) -> np.ndarray:
        n = self.stats(graph)["n"][level]
        a = np.empty(n, dtype=np.int32)
        _check(load().cmg_batch_get_aggregates(self._b, graph, level, C.c_void_p(a.ctypes.data)),
               "batch_aggregates")
        return a

    def level_csr(self, graph: int, level: int):
        st = self.stats(graph)
        n, m = st["n"][level], st["nnz"][level]
        rp = np.empty(n + 1, dtype=np.int64)
        col = np.empty(m, dtype=np.int32)
        w = np.empty(m, dtype=np.float64)
        g = C.c_double()
        _check(load().cmg_batch_get_level_csr(self._b, graph, level, C.c_void_p(rp.ctypes.data),
                                              C.c_void_p(col.ctypes.data), C.c_void_p(w.ctypes.data),
                                              C.byref(g)), "batch_level_csr")
        return rp, col, w, g.value

    def set_replay(self, sweeps):
        """sweeps: int array [G][64] (or None to return to opts.replay_sweeps)."""
        if sweeps is None:
            _check(load().cmg_batch_set_replay(self._b, None), "set_replay")
            return
        arr = np.zeros((self.G, CMG_MAX_LEVELS), dtype=np.int32)
        for q, row in enumerate(sweeps):
            arr[q, :len(row)] = row
        _check(load().cmg_batch_set_replay(self._b, C.c_void_p(arr.ctypes.data)), "set_replay")

    def shape(self, level: int):
        sh = BatchShape()
        _check(load().cmg_batch_config(self._b, level, 0, C.byref(sh)), "batch_config")
        return sh.as_tuple()

    def set_shape(self, level: int, threads_per_graph: int, lanes_per_row: int,
                  graphs_per_cta: int, stage_csr: int = 1):
        sh = BatchShape(threads_per_graph, lanes_per_row, graphs_per_cta, stage_csr)
        _check(load().cmg_batch_config(self._b, level, 1, C.byref(sh)), "batch_config",
               allow_warn=False)

    def autotune(self, stream=None):
        _check(load().cmg_batch_autotune(self._b, _stream(stream)), "batch_autotune", allow_warn=False)

    def level_ms(self):
        """Per-union-level device times of the last solve (options timing=1)."""
        out = []
        for lvl in range(self.union_levels):
            ms = C.c_double()
            _check(load().cmg_batch_level_ms(self._b, lvl, C.byref(ms)), "batch_level_ms")
            out.append(ms.value)
        return out

    def device_bytes(self) -> int:
        b = C.c_size_t()
        _check(load().cmg_batch_device_bytes(self._b, C.byref(b)), "batch_bytes")
        return b.value

    def fiedler(self, u_out=None, stream=None):
        """Returns (u, lambda2[G], residual[G], status[G]); u is the union vector
        (numpy on the host unless a torch CUDA tensor is passed)."""
        if u_out is None:
            u_out = np.empty(self.N, dtype=np.float64)
        p_u, mem = _ptr(u_out)
        lam = np.empty(self.G, dtype=np.float64)
        res = np.empty(self.G, dtype=np.float64)
        sts = np.empty(self.G, dtype=np.int32)
        st = load().cmg_fiedler_batch(self._b, p_u, mem, C.c_void_p(lam.ctypes.data),
                                      C.c_void_p(res.ctypes.data), C.c_void_p(sts.ctypes.data),
                                      _stream(stream))
        _check(st, "cmg_fiedler_batch")
        return u_out, lam, res, sts


class Server:
    """Request loop for Fiedler solves (cmg_server_*): register host graphs,
    submit requests, wait for results.  Graph arrays are kept alive here."""

    def __init__(self, *, workers=4, max_batch=256, batch_max_n=8192, mem_budget=0,
                 keep_resident=1, min_batch=32, opts: Options | None = None, **kw):
        lib = load()
        cfg = ServerConfig()
        _check(lib.cmg_server_config_default(C.byref(cfg)), "server_config")
        cfg.workers, cfg.max_batch, cfg.batch_max_n = workers, max_batch, batch_max_n
        cfg.mem_budget, cfg.keep_resident, cfg.min_batch = mem_budget, keep_resident, min_batch
        self.opts = opts if opts is not None else options(**kw)
        s = C.c_void_p()
        self._s = None
        _check(lib.cmg_server_create(C.byref(cfg), C.byref(self.opts), C.byref(s)), "server_create",
               allow_warn=False)
        self._s = s
        self._graphs = []
        self._outs = {}

    def add_graph(self, row_ptr, col, w) -> int:
        row_ptr, col, w = _as_inputs(np.asarray(row_ptr), np.asarray(col), np.asarray(w))
        gid = C.c_int64()
        _check(load().cmg_server_add_graph(self._s, len(row_ptr) - 1, C.c_void_p(row_ptr.ctypes.data),
                                           C.c_void_p(col.ctypes.data), C.c_void_p(w.ctypes.data),
                                           C.byref(gid)), "server_add_graph", allow_warn=False)
        self._graphs.append((row_ptr, col, w))
        return gid.value

    def submit(self, graph_id: int, want_vector: bool = True, *, seed=None, x0=None,
               x0_level=0) -> int:
        """Queues a solve; seed / x0 / x0_level make it a re-solve with its own
        options (cmg_server_submit_ex; x0 is a host array, kept alive here
        until the request is waited for)."""
        n = len(self._graphs[graph_id][0]) - 1
        u = np.empty(n, dtype=np.float64) if want_vector else None
        t = C.c_int64()
        pu = C.c_void_p(u.ctypes.data) if u is not None else None
        keep = None
        if seed is None and x0 is None:
            _check(load().cmg_server_submit(self._s, graph_id, pu, C.byref(t)), "server_submit",
                   allow_warn=False)
        else:
            so = SolveOptions()
            _check(load().cmg_solve_options_default(None, C.byref(so)), "solve_options")
            so.seed = int(self.opts.seed if seed is None else seed)
            if x0 is not None:
                keep = np.ascontiguousarray(x0, dtype=np.float64)
                so.x0, so.x0_mem, so.x0_level = keep.ctypes.data, 0, int(x0_level)
            _check(load().cmg_server_submit_ex(self._s, graph_id, C.byref(so), pu, C.byref(t)),
                   "server_submit", allow_warn=False)
        self._outs[t.value] = (u, keep)
        return t.value

    def wait(self, ticket: int, timeout_s: float | None = None):
        """Returns (u or None, request dict); raises on a failed request (and
        with ERR_TIMEOUT when timeout_s passes first)."""
        r = Request()
        if timeout_s is None:
            st = load().cmg_server_wait(self._s, ticket, C.byref(r))
        else:
            st = load().cmg_server_wait_for(self._s, ticket, int(timeout_s * 1000), C.byref(r))
            if st == -12:
                raise CmgError(st, "server_wait")
        u, _ = self._outs.pop(ticket, (None, None))
        _check(st, "server_wait")
        return u, r.as_dict()

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().cmg_server_get_stats(self._s, C.byref(s)), "server_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "_s", None):
            load().cmg_server_destroy(self._s)
            self._s = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ step entry points
def heaviest_neighbour(rp32, col, w, stream=None):
    torch = _torch()
    n = rp32.numel() - 1
    m = torch.empty(n, dtype=torch.int32, device=rp32.device)
    _check(load().cmg_heaviest_neighbour(n, _ptr(rp32)[0], _ptr(col)[0], _ptr(w)[0], _ptr(m)[0],
                                         _stream(stream)), "heaviest_neighbour")
    return m


def visit_ranks(n: int, seed: int, level: int, device="cuda", stream=None):
    torch = _torch()
    r = torch.empty(n, dtype=torch.int32, device=device)
    _check(load().cmg_visit_ranks(n, C.c_uint64(seed), level, _ptr(r)[0], _stream(stream)),
           "visit_ranks")
    return r


def hec_aggregate(rp32, col, w, rank, stream=None):
    torch = _torch()
    n = rp32.numel() - 1
    agg = torch.empty(n, dtype=torch.int32, device=rp32.device)
    c = C.c_int64()
    _check(load().cmg_hec_aggregate(n, _ptr(rp32)[0], _ptr(col)[0], _ptr(w)[0], _ptr(rank)[0],
                                    _ptr(agg)[0], C.byref(c), _stream(stream)), "hec_aggregate")
    return agg, c.value


def power_sweeps(rp32, col, w, x_in, k: int, g: float = 0.0, stream=None):
    torch = _torch()
    n = rp32.numel() - 1
    u = torch.empty(n, dtype=torch.float64, device=rp32.device)
    cs = C.c_double()
    _check(load().cmg_power_sweeps(n, _ptr(rp32)[0], _ptr(col)[0], _ptr(w)[0], float(g),
                                   _ptr(x_in)[0], int(k), _ptr(u)[0], C.byref(cs), _stream(stream)),
           "power_sweeps")
    return u, cs.value


def power_sweeps_noalloc(rp32, col, w, x_in, k: int, g: float = 0.0, u_out=None, stream=None):
    """cmg_power_sweeps_noalloc: same as power_sweeps, scratch in a fixed device
    array (no allocation by the library).  u_out: torch CUDA float64 tensor."""
    torch = _torch()
    n = rp32.numel() - 1
    if u_out is None:
        u_out = torch.empty(n, dtype=torch.float64, device=rp32.device)
    cs = C.c_double()
    _check(load().cmg_power_sweeps_noalloc(n, _ptr(rp32)[0], _ptr(col)[0], _ptr(w)[0], float(g),
                                           _ptr(x_in)[0], int(k), _ptr(u_out)[0], C.byref(cs),
                                           _stream(stream)), "power_sweeps_noalloc")
    return u_out, cs.value


def rayleigh_residual(rp32, col, w, u, stream=None):
    lam = C.c_double()
    res = C.c_double()
    n = rp32.numel() - 1
    _check(load().cmg_rayleigh_residual(n, _ptr(rp32)[0], _ptr(col)[0], _ptr(w)[0], _ptr(u)[0],
                                        C.byref(lam), C.byref(res), _stream(stream)), "rayleigh")
    return lam.value, res.value


def kernel_launches() -> int:
    c = C.c_uint64()
    _check(load().cmg_kernel_launches(C.byref(c)), "kernel_launches")
    return c.value


def debug_fail_alloc_after(k: int):
    load().cmg_debug_fail_alloc_after(int(k))


def debug_stall_barrier(launch: int, barrier: int = 0):
    """Test hook: the launch-th next multi-CTA cooperative launch holds its grid
    barrier number `barrier`, so its bounded waits run out (launch < 0: off)."""
    _check(load().cmg_debug_stall_barrier(int(launch), int(barrier)), "debug_stall_barrier")


def gcmg_grid(dim: int, N: int, J: int, *, beta: float = 4.0, k0: int = 1, u_out=None, stream=None):
    """cmg_gcmg_grid: Alg. 4 on the unit N^dim grid graph with J geometric
    coarsenings.  Returns (u, r0[J+1], rk[J+1], k[J+1]); u is numpy (host) or
    the given torch CUDA float64 tensor."""
    if u_out is None:
        u_out = np.empty(N ** dim, dtype=np.float64)
    p_u, mem = _ptr(u_out)
    r0 = np.zeros(J + 1)
    rk = np.zeros(J + 1)
    ks = np.zeros(J + 1, dtype=np.int32)
    _check(load().cmg_gcmg_grid(int(dim), int(N), int(J), float(beta), int(k0), p_u, mem,
                                C.c_void_p(r0.ctypes.data), C.c_void_p(rk.ctypes.data),
                                C.c_void_p(ks.ctypes.data), _stream(stream)), "gcmg_grid")
    return u_out, r0, rk, ks
