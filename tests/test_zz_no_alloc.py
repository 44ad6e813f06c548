"""cmg_power_sweeps_noalloc: the allocation-free variant of cmg_power_sweeps.

For callers that must not allocate device memory (their device memory is
already reserved by their own allocator, or allocation calls are not allowed
where they run).  The variant keeps its scratch in one fixed device array; the
checks below call it through the C-ABI and compare it with cmg_power_sweeps,
twice in a row (the array keeps the previous call's contents), with the
library's own allocator armed to fail so any allocation would show.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(rp, col, w):
    return (torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(col).cuda(),
            torch.from_numpy(w).cuda())


def call_noalloc(lib, drp, dcol, dw, x, k, u):
    n = drp.numel() - 1
    cs = C.c_double()
    st = lib.cmg_power_sweeps_noalloc(n, C.c_void_p(drp.data_ptr()), C.c_void_p(dcol.data_ptr()),
                                      C.c_void_p(dw.data_ptr()), 0.0, C.c_void_p(x.data_ptr()),
                                      int(k), C.c_void_p(u.data_ptr()), C.byref(cs),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, cs.value


@pytest.mark.parametrize("name,k", [("grid", 25), ("random", 40)])
def test_noalloc_matches_allocating_entry_point_twice(name, k):
    lib = cmg.load()
    if name == "grid":
        rp, col, w = inputs.grid2d(300, 200, "uniform", seed=21)   # large enough for the tiled kernel
    else:
        rp, col, w = inputs.random_connected(1500, 4000, seed=22)  # small-level kernel
    n = len(rp) - 1
    drp, dcol, dw = dev(rp, col, w)
    ref, ref_cos = cmg.power_sweeps(drp, dcol, dw, torch.from_numpy(oracle.gaussian_start(9, n)).cuda(), k)
    ref = ref.cpu().numpy()
    tol = 1e-14 * k * np.sqrt(n)
    for call in range(2):
        x = torch.from_numpy(oracle.gaussian_start(9, n)).cuda()
        u = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        cmg.debug_fail_alloc_after(0)        # any allocation by the library would now fail
        try:
            st, cs = call_noalloc(lib, drp, dcol, dw, x, k, u)
        finally:
            cmg.debug_fail_alloc_after(-1)
        assert cmg.STATUS[st] == "OK", (call, st)
        got = u.cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol, (call, np.linalg.norm(got - ref))
        assert abs(cs - ref_cos) <= 1e-13


def test_noalloc_rejects_sizes_beyond_the_limit():
    lib = cmg.load()
    rp, col, w = inputs.path(8)
    drp, dcol, dw = dev(rp, col, w)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    cs = C.c_double()
    # n is checked before any device access, so the small buffers are never read
    st = lib.cmg_power_sweeps_noalloc(cmg.NOALLOC_MAX_N + 1, C.c_void_p(drp.data_ptr()),
                                      C.c_void_p(dcol.data_ptr()), C.c_void_p(dw.data_ptr()), 0.0,
                                      C.c_void_p(x.data_ptr()), 3, C.c_void_p(u.data_ptr()),
                                      C.byref(cs), None)
    assert cmg.STATUS[st] == "ERR_TOO_LARGE"
