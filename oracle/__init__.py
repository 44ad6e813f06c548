"""CPU oracle for the cascadic multigrid (CMG) Fiedler-vector method.

TEST INFRASTRUCTURE ONLY.  A plain, sequential, FP64 restatement of
arXiv 1412.0565 (Alg. 1, Alg. 2, Alg. 3; Definition 2.1; Proposition 2.7),
written in C (``cmg_oracle.c``) and loaded here through ctypes.  Only the
test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import this package.  It shares no code with the CUDA
library in ``paper_1412_0565_gb300``; neither imports the other.

Every function below is a marshalling wrapper around one C routine; the
arithmetic lives in C.  The C file's header lists the readings (R1..R11) taken
where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcmg_oracle.so")
_lock = threading.Lock()
_lib = None

I64P = C.POINTER(C.c_int64)
I32P = C.POINTER(C.c_int32)
F64P = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.orc_splitmix64.restype = C.c_uint64
        lib.orc_splitmix64.argtypes = [C.c_uint64]
        lib.orc_visit_rank.restype = C.c_int64
        lib.orc_visit_rank.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int64]
        lib.orc_visit_ranks.restype = None
        lib.orc_visit_ranks.argtypes = [C.c_uint64, C.c_int32, C.c_int64, I64P]
        lib.orc_gaussian_start.restype = None
        lib.orc_gaussian_start.argtypes = [C.c_uint64, C.c_int64, F64P]
        lib.orc_gershgorin.restype = C.c_double
        lib.orc_gershgorin.argtypes = [C.c_int64, I64P, F64P]
        lib.orc_heaviest_neighbour.restype = None
        lib.orc_heaviest_neighbour.argtypes = [C.c_int64, I64P, I32P, F64P, I32P]
        lib.orc_hec.restype = C.c_int64
        lib.orc_hec.argtypes = [C.c_int64, I64P, I32P, F64P, I64P, I32P]
        lib.orc_rayleigh_residual.restype = None
        lib.orc_rayleigh_residual.argtypes = [C.c_int64, I64P, I32P, F64P, F64P, F64P, F64P]
        lib.orc_power_iteration.restype = C.c_int64
        lib.orc_power_iteration.argtypes = [C.c_int64, I64P, I32P, F64P, C.c_double, F64P,
                                            C.c_double, C.c_int32, C.c_int64, C.c_int64, F64P,
                                            F64P, I32P]
        lib.orc_setup.restype = C.c_void_p
        lib.orc_setup.argtypes = [C.c_int64, I64P, I32P, F64P, C.c_uint64, C.c_int32, C.c_int32]
        lib.orc_levels.restype = C.c_int32
        lib.orc_levels.argtypes = [C.c_void_p]
        lib.orc_level_info.restype = None
        lib.orc_level_info.argtypes = [C.c_void_p, C.c_int32, I64P, I64P, F64P]
        lib.orc_level_csr.restype = None
        lib.orc_level_csr.argtypes = [C.c_void_p, C.c_int32, I64P, I32P, F64P]
        lib.orc_level_agg.restype = C.c_int32
        lib.orc_level_agg.argtypes = [C.c_void_p, C.c_int32, I32P]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [C.c_void_p]
        lib.orc_solve.restype = C.c_int32
        lib.orc_solve.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_int32, C.c_double,
                                  C.c_int32, I64P, C.c_int64, C.c_int64, C.c_int32, C.c_double,
                                  F64P, F64P, F64P, I64P, F64P]
        lib.orc_solve_ex.restype = C.c_int32
        lib.orc_solve_ex.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_int32, C.c_double,
                                     C.c_int32, I64P, C.c_int64, C.c_int64, C.c_int32,
                                     C.c_double, C.c_int32, F64P, F64P, F64P, F64P, I64P, F64P,
                                     F64P, F64P]
        lib.orc_solve_block.restype = C.c_int32
        lib.orc_solve_block.argtypes = [C.c_void_p, C.c_int32, C.c_uint64, C.c_double, C.c_int32,
                                        I64P, C.c_int64, C.c_int64, C.c_int32, C.c_double, F64P,
                                        F64P, F64P, I64P]
        lib.orc_gcmg_grid.restype = C.c_int32
        lib.orc_gcmg_grid.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_double, C.c_int32, F64P,
                                      F64P, I64P, F64P]
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _csr(rp, col, w):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    return rp, col, w


# ---------------------------------------------------------------- generators
def splitmix64(x: int) -> int:
    """One SplitMix64 output from state x (Steele, Lea, Flood 2014)."""
    return int(_load().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def visit_ranks(seed: int, level: int, n: int) -> np.ndarray:
    """Alg. 2's randperm, as ranks r(v) (vertex v is visited at step r(v))."""
    r = np.empty(n, dtype=np.int64)
    _load().orc_visit_ranks(C.c_uint64(seed), level, n, _p(r, C.c_int64))
    return r


def gaussian_start(seed: int, n: int) -> np.ndarray:
    """Alg. 1 Step 2's randn(n_J) (Box-Muller on splitmix64 uniforms)."""
    x = np.empty(n, dtype=np.float64)
    _load().orc_gaussian_start(C.c_uint64(seed), n, _p(x, C.c_double))
    return x


# ---------------------------------------------------------------- method steps
def gershgorin(rp, col, w) -> float:
    """Alg. 3's g = max_i sum_j |l_ij|."""
    rp, col, w = _csr(rp, col, w)
    return float(_load().orc_gershgorin(len(rp) - 1, _p(rp, C.c_int64), _p(w, C.c_double)))


def heaviest_neighbour(rp, col, w) -> np.ndarray:
    """Alg. 2's argmin(L(:, v)) for every v (ties -> lowest index)."""
    rp, col, w = _csr(rp, col, w)
    n = len(rp) - 1
    m = np.empty(n, dtype=np.int32)
    _load().orc_heaviest_neighbour(n, _p(rp, C.c_int64), _p(col, C.c_int32), _p(w, C.c_double),
                                   _p(m, C.c_int32))
    return m


def hec(rp, col, w, rank) -> tuple[np.ndarray, int]:
    """Alg. 2 executed literally with visit ranks `rank`; returns (agg, c)."""
    rp, col, w = _csr(rp, col, w)
    n = len(rp) - 1
    rank = np.ascontiguousarray(rank, dtype=np.int64)
    agg = np.empty(n, dtype=np.int32)
    c = _load().orc_hec(n, _p(rp, C.c_int64), _p(col, C.c_int32), _p(w, C.c_double),
                        _p(rank, C.c_int64), _p(agg, C.c_int32))
    return agg, int(c)


def rayleigh_residual(rp, col, w, u) -> tuple[float, float]:
    """lambda = u^T L u / u^T u (edge-difference form) and ||(L - lambda I)u|| / ||u||."""
    rp, col, w = _csr(rp, col, w)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lam = C.c_double()
    res = C.c_double()
    _load().orc_rayleigh_residual(len(rp) - 1, _p(rp, C.c_int64), _p(col, C.c_int32),
                                  _p(w, C.c_double), _p(u, C.c_double), C.byref(lam), C.byref(res))
    return lam.value, res.value


def power_iteration(rp, col, w, y0, *, tol=1e-8, fixed=None, max_sweeps=20000, g=None):
    """Alg. 3.  fixed=k runs exactly k sweeps; otherwise the tolerance rule.

    Returns (u, sweeps, final_cos, capped)."""
    rp, col, w = _csr(rp, col, w)
    n = len(rp) - 1
    if g is None:
        g = gershgorin(rp, col, w)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    u = np.empty(n, dtype=np.float64)
    cs = C.c_double()
    cap = C.c_int32()
    k = _load().orc_power_iteration(n, _p(rp, C.c_int64), _p(col, C.c_int32), _p(w, C.c_double),
                                    float(g), _p(y0, C.c_double), float(tol),
                                    1 if fixed is not None else 0, int(fixed or 0), int(max_sweeps),
                                    _p(u, C.c_double), C.byref(cs), C.byref(cap))
    return u, int(k), cs.value, bool(cap.value)


class Hierarchy:
    """Alg. 1 Step 1 (setup phase) on the CPU; levels are read back as numpy arrays."""

    def __init__(self, rp, col, w, *, seed=1412, coarse_size=25, max_levels=64):
        rp, col, w = _csr(rp, col, w)
        self._keep = (rp, col, w)
        lib = _load()
        self._h = lib.orc_setup(len(rp) - 1, _p(rp, C.c_int64), _p(col, C.c_int32),
                                _p(w, C.c_double), C.c_uint64(seed), coarse_size, max_levels)
        if not self._h:
            raise ValueError("graph too small (n < 2)")
        self.seed = seed

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_free(h)
            self._h = None

    @property
    def levels(self) -> int:
        return int(_load().orc_levels(self._h))

    def info(self, level):
        n = C.c_int64()
        nnz = C.c_int64()
        g = C.c_double()
        _load().orc_level_info(self._h, level, C.byref(n), C.byref(nnz), C.byref(g))
        return n.value, nnz.value, g.value

    def csr(self, level):
        n, nnz, _ = self.info(level)
        rp = np.empty(n + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        w = np.empty(nnz, dtype=np.float64)
        _load().orc_level_csr(self._h, level, _p(rp, C.c_int64), _p(col, C.c_int32),
                              _p(w, C.c_double))
        return rp, col, w

    def agg(self, level):
        n, _, _ = self.info(level)
        a = np.empty(n, dtype=np.int32)
        ok = _load().orc_level_agg(self._h, level, _p(a, C.c_int32))
        return a if ok else None

    def sizes(self):
        return [self.info(l)[0] for l in range(self.levels)]

    def solve(self, *, tol=1e-8, schedule="tol", beta=4.0, k0=1, replay=None,
              max_sweeps=20000, max_sweeps_coarsest=100000, converged=False, conv_rtol=1e-11,
              seed=None, start_level=None, x0=None, trace=False):
        """Alg. 1 Steps 2-3.  Returns dict(u, lam, res, sweeps, cos, capped).

        start_level / x0: start the cascade on that level from x0 (in the
        level's numbering) instead of the Gaussian start on the coarsest level.
        trace: also return "start" and "end", lists (one entry per level,
        None for levels not visited) of the vector each level's power
        iteration starts from (before Gram-Schmidt) and the one it returns."""
        J = self.levels - 1
        sizes = self.sizes()
        n0 = sizes[0]
        sched = {"tol": 0, "fixed": 1, "replay": 2}[schedule]
        rep = np.zeros(J + 1, dtype=np.int64)
        if replay is not None:
            rep[:] = np.asarray(replay, dtype=np.int64)[: J + 1]
        sl = -1
        xp = None
        if start_level is not None:
            sl = int(start_level)
            if not 0 <= sl <= J:
                raise ValueError("start_level out of range")
            xp = np.ascontiguousarray(x0, dtype=np.float64)
            if xp.shape != (sizes[sl],):
                raise ValueError("x0 must have the start level's size")
        u = np.empty(n0, dtype=np.float64)
        lam = C.c_double()
        res = C.c_double()
        sweeps = np.zeros(J + 1, dtype=np.int64)
        cos = np.zeros(J + 1, dtype=np.float64)
        tot = int(sum(sizes))
        ts = np.full(tot, np.nan) if trace else None
        te = np.full(tot, np.nan) if trace else None
        nul = C.cast(None, F64P)
        warn = _load().orc_solve_ex(
            self._h, C.c_uint64(self.seed if seed is None else seed), float(tol), sched,
            float(beta), int(k0), _p(rep, C.c_int64), int(max_sweeps), int(max_sweeps_coarsest),
            1 if converged else 0, float(conv_rtol), sl,
            _p(xp, C.c_double) if xp is not None else nul, _p(u, C.c_double), C.byref(lam),
            C.byref(res), _p(sweeps, C.c_int64), _p(cos, C.c_double),
            _p(ts, C.c_double) if trace else nul, _p(te, C.c_double) if trace else nul)
        out = {"u": u, "lam": lam.value, "res": res.value, "sweeps": sweeps, "cos": cos,
               "capped": bool(warn)}
        if trace:
            off = np.concatenate([[0], np.cumsum(sizes)])
            top = J if sl < 0 else sl
            out["start"] = [ts[off[j]:off[j + 1]].copy() if j <= top else None for j in range(J + 1)]
            out["end"] = [te[off[j]:off[j + 1]].copy() if j <= top else None for j in range(J + 1)]
        return out


def eigenpairs(h: "Hierarchy", k: int, *, seed=None, tol=1e-8, replay=None, max_sweeps=20000,
               max_sweeps_coarsest=100000, converged=False, conv_rtol=1e-11):
    """k eigenpairs by the cascade with block power iteration (the Remark
    after Alg. 4) on hierarchy h.  Returns dict(U [k, n0], lam[k], res[k],
    sweeps, capped)."""
    J = h.levels - 1
    n0 = h.sizes()[0]
    rep = np.zeros(J + 1, dtype=np.int64)
    if replay is not None:
        rep[:] = np.asarray(replay, dtype=np.int64)[: J + 1]
    U = np.empty((k, n0))
    lam = np.empty(k)
    res = np.empty(k)
    sweeps = np.zeros(J + 1, dtype=np.int64)
    st = _load().orc_solve_block(h._h, int(k), C.c_uint64(h.seed if seed is None else seed),
                                 float(tol), 2 if replay is not None else 0, _p(rep, C.c_int64),
                                 int(max_sweeps), int(max_sweeps_coarsest), 1 if converged else 0,
                                 float(conv_rtol), _p(U, C.c_double), _p(lam, C.c_double),
                                 _p(res, C.c_double), _p(sweeps, C.c_int64))
    if st < 0:
        raise ValueError("k must be between 1 and n_J - 1")
    return {"U": U, "lam": lam, "res": res, "sweeps": sweeps, "capped": bool(st)}


def fiedler(rp, col, w, *, seed=1412, tol=1e-8, coarse_size=25, **kw):
    """Whole CMG (Alg. 1): returns (u, lambda2, residual, hierarchy, result dict)."""
    h = Hierarchy(rp, col, w, seed=seed, coarse_size=coarse_size)
    r = h.solve(tol=tol, **kw)
    return r["u"], r["lam"], r["res"], h, r


def gcmg_grid(dim: int, N: int, J: int, *, beta=4.0, k0=1):
    """Alg. 4 (geometric CMG) on the unit N^dim grid graph with J coarsenings
    (the Table 4 setting is dim 2, N 1025, J 5, beta 4, k0 1).  Returns dict
    (u, r0, rk, k): per level the Rayleigh quotient of the prolonged start and
    after the k_j smoothing steps, and k_j."""
    n = N ** dim
    r0 = np.zeros(J + 1)
    rk = np.zeros(J + 1)
    ks = np.zeros(J + 1, dtype=np.int64)
    u = np.empty(n)
    st = _load().orc_gcmg_grid(dim, N, J, float(beta), int(k0), _p(r0, C.c_double),
                               _p(rk, C.c_double), _p(ks, C.c_int64), _p(u, C.c_double))
    if st != 0:
        raise ValueError("invalid grid sizes for geometric coarsening")
    return {"u": u, "r0": r0, "rk": rk, "k": ks}
