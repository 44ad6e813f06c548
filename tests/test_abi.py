"""The C-ABI library builds, loads and exports every symbol include/cmg.h
declares; host-only entry points behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1412_0565_gb300 import cmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(cmg_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = cmg.load()
    names = declared_functions()
    assert len(names) >= 17
    assert sorted(names) == sorted(cmg.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_build_targets_sm_103a_only():
    from paper_1412_0565_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_options_default_matches_paper_settings():
    o = cmg.options()
    assert o.tol == 1e-8 and o.coarse_size == 25 and o.max_levels == 64
    assert o.precision == cmg.FP64 and o.schedule == 0 and o.validate == 1
    assert C.sizeof(cmg.Options) == 320
    assert C.sizeof(cmg.Stats) == 8 + 8 + 4 + 4 + 64 * (8 + 8 + 4 + 8 + 8) + 8


def test_status_strings_and_version():
    for code in cmg.STATUS:
        assert cmg.status_string(code)
    assert "sm_103a" in cmg.version()


def test_host_side_argument_errors_need_no_gpu():
    lib = cmg.load()
    h = C.c_void_p()
    rp = np.array([0, 0], dtype=np.int64)
    col = np.zeros(1, dtype=np.int32)
    w = np.ones(1)
    st = lib.cmg_setup(1, C.c_void_p(rp.ctypes.data), C.c_void_p(col.ctypes.data),
                       C.c_void_p(w.ctypes.data), 0, None, None, C.byref(h))
    assert cmg.STATUS[st] == "ERR_TOO_SMALL"
    st = lib.cmg_setup(5, None, None, None, 0, None, None, C.byref(h))
    assert cmg.STATUS[st] == "ERR_INVALID_ARG"
    st = lib.cmg_setup(5, C.c_void_p(rp.ctypes.data), C.c_void_p(col.ctypes.data),
                       C.c_void_p(w.ctypes.data), 7, None, None, C.byref(h))
    assert cmg.STATUS[st] == "ERR_INVALID_ARG"
    bad = cmg.options(tol=2.0)
    st = lib.cmg_setup(5, C.c_void_p(rp.ctypes.data), C.c_void_p(col.ctypes.data),
                       C.c_void_p(w.ctypes.data), 0, C.byref(bad), None, C.byref(h))
    assert cmg.STATUS[st] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_fiedler(None, None, 0, None, None, None)] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_free(None)] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_level_kernels(None, None, None)] == "ERR_INVALID_ARG"


def test_estimate_device_bytes_monotone():
    a = cmg.estimate_device_bytes(1000, 6000)
    b = cmg.estimate_device_bytes(1_000_000, 6_000_000)
    assert 0 < a < b
    assert cmg.estimate_device_bytes(10**6, 6 * 10**6, cmg.FP32_SWEEP) > 0


def test_batch_host_side_argument_errors_need_no_gpu():
    lib = cmg.load()
    b = C.c_void_p()
    rp = np.array([0, 0], dtype=np.int64)
    col = np.zeros(1, dtype=np.int32)
    w = np.ones(1)
    P = lambda a: C.c_void_p(a.ctypes.data)

    def setup(offs, mem=0, opts=None, G=None):
        offs = np.asarray(offs, dtype=np.int64)
        return cmg.STATUS[lib.cmg_setup_batch(len(offs) - 1 if G is None else G, P(offs), P(rp),
                                              P(col), P(w), mem, opts, None, C.byref(b))]

    assert setup([0, 4, 5]) == "ERR_TOO_SMALL"          # graph 1 has one vertex
    assert setup([0, 4, 3, 8]) == "ERR_INVALID_ARG"     # decreasing offsets
    assert setup([1, 4, 8]) == "ERR_INVALID_ARG"        # does not start at 0
    assert setup([0, 4, 8], G=0) == "ERR_INVALID_ARG"
    assert setup([0, 4, 8], mem=3) == "ERR_INVALID_ARG"
    bad = cmg.options(coarse_size=0)
    assert setup([0, 4, 8], opts=C.byref(bad)) == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_fiedler_batch(None, None, 0, None, None, None, None)] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_batch_free(None)] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_batch_stats(None, 0, None)] == "ERR_INVALID_ARG"
    assert not b.value


def test_server_argument_errors_need_no_gpu():
    lib = cmg.load()
    s = C.c_void_p()
    cfg = cmg.ServerConfig()
    assert lib.cmg_server_config_default(C.byref(cfg)) == 0
    assert cfg.workers == 4 and cfg.max_batch == 256 and cfg.keep_resident == 1 and cfg.min_batch == 32
    for field, bad in (("workers", 0), ("workers", 65), ("max_batch", 0), ("min_batch", -1)):
        c2 = cmg.ServerConfig.from_buffer_copy(cfg)
        setattr(c2, field, bad)
        assert cmg.STATUS[lib.cmg_server_create(C.byref(c2), None, C.byref(s))] == "ERR_INVALID_ARG"
    o = cmg.options(timing=1)
    assert cmg.STATUS[lib.cmg_server_create(C.byref(cfg), C.byref(o), C.byref(s))] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_server_destroy(None)] == "ERR_INVALID_ARG"
    assert cmg.STATUS[lib.cmg_server_wait(None, 1, None)] == "ERR_INVALID_ARG"
    assert not s.value


def test_public_structs_match_header_sizes():
    assert C.sizeof(cmg.BatchShape) == 16
    assert C.sizeof(cmg.ServerConfig) == 4 + 4 + 8 + 8 + 4 + 4
    assert C.sizeof(cmg.Request) == 16 + 16 + 24
    assert C.sizeof(cmg.ServerStats) == 6 * 8 + 4 * 8
    assert C.sizeof(cmg.SolveOptions) == 8 + 8 + 4 + 4 + 4 * 4
