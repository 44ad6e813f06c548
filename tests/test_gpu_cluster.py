"""The cluster kernel (k_power_cluster: FP64 sweeps of one level spread over a
thread-block cluster of 2..8 CTAs) against the CPU oracle.

CMG_CLUSTER=128 plans every FP64 level from 128 rows on that a cluster can
hold, so that graphs of several families and sizes run it on one or more
levels (with 2 to 8 CTAs).  Bar: identical per-level sweep counts, vector
within 1e-10, lambda2 within 1e-12; repeated solves bit-identical (every CTA
sums the CTAs' stop sums in rank order)."""
import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KIND_CLUSTER = 5

CASES = {
    "grid_ragged": lambda: inputs.grid2d(145, 171, "uniform", seed=2),
    "grid3d": lambda: inputs.grid3d(30, 30, 30, "uniform", seed=1412),
    "random": lambda: inputs.random_connected(6000, 24000, seed=3),
    "rgg": lambda: inputs.rgg(8000, 8.0, seed=5),
    # power-law graphs small enough that their hub slices fit: clusters on
    # levels of 3,000, 861 and 224 rows (BA) and 2,999, 855 and 220 rows
    # (Chung-Lu; slot order, rows by decreasing degree, makes the slices fit)
    "ba": lambda: inputs.barabasi_albert(3000, 4, seed=6),
    "chung_lu": lambda: inputs.chung_lu(3000, seed=7),
}


def aligned_err(u, ref):
    if np.dot(u, ref) < 0:
        u = -u
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("name", sorted(CASES))
def test_cluster_kernel_matches_oracle(monkeypatch, name):
    monkeypatch.setenv("CMG_CLUSTER", "128")
    rp, col, w = CASES[name]()
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    kind, _ = h.level_kernels()
    assert KIND_CLUSTER in kind
    u, lam, st = h.fiedler()
    u2, lam2, _ = h.fiedler()
    h.close()
    assert np.array_equal(u, u2) and lam == lam2
    ref_u, ref_lam, _, oh, ref = oracle.fiedler(rp, col, w, seed=1412)
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref_u) <= 1e-10
    assert abs(lam - ref_lam) <= 1e-12 * abs(ref_lam)


def test_cluster_kernel_in_the_fp32_form_and_on_resolves(monkeypatch):
    """FP32 sweep form (its coarse levels sweep in FP64, some in a cluster)
    within the FP32 gate, and a re-solve from a start vector on a cluster
    level against orc_solve_ex."""
    monkeypatch.setenv("CMG_CLUSTER", "128")
    rp, col, w = CASES["grid3d"]()
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    ref = oh.solve()
    h = cmg.Hierarchy(rp, col, w, seed=1412, precision="fp32", schedule="replay",
                      replay_sweeps=ref["sweeps"].tolist())
    kind, _ = h.level_kernels()
    assert KIND_CLUSTER in kind
    u, lam, st = h.fiedler()
    h.close()
    assert abs(lam - ref["lam"]) <= 1e-6 * abs(ref["lam"])
    c = abs(np.dot(u, ref["u"])) / (np.linalg.norm(u) * np.linalg.norm(ref["u"]))
    assert np.arccos(min(1.0, c)) <= 1e-4
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    kind, _ = h.level_kernels()
    lvl = kind.index(KIND_CLUSTER)
    x0 = np.random.default_rng(4).standard_normal(h.sizes()[0][lvl])
    u, lam, st = h.fiedler(x0=x0, x0_level=lvl)
    h.close()
    r = oh.solve(start_level=lvl, x0=x0)
    assert st["sweeps"] == r["sweeps"].tolist()
    assert aligned_err(u, r["u"]) <= 1e-10
    assert abs(lam - r["lam"]) <= 1e-12 * abs(r["lam"])


def test_cluster_plan_on_the_benchmark_grid():
    """Default rule: the 100^3 grid's 3,000- and 847-row levels run in a
    cluster; the 245-row level and smaller stay on one CTA."""
    rp, col, w = inputs.grid3d(100, 100, 100, "uniform", seed=1412)
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    kind, _ = h.level_kernels()
    n = h.sizes()[0]
    h.close()
    for k, rows in zip(kind, n):
        if rows in (3000, 847):
            assert k == KIND_CLUSTER
        if rows < 512:
            assert k == 0
