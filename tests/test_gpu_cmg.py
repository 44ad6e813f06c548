"""Whole-method parity (Alg. 1) of the CUDA path against the CPU oracle.

FP64: identical hierarchy and per-level sweep counts, vector within 1e-10
relative 2-norm after sign alignment, lambda2 within 1e-12 relative.
FP32 sweep form: lambda2 relative error <= 1e-6 and angle <= 1e-4 rad against
the FP64 oracle run with the same per-level sweep counts (replay schedule).
"""
import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VEC_TOL = 1e-10
LAM_TOL = 1e-12


def aligned_err(u, ref):
    if np.dot(u, ref) < 0:
        u = -u
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def angle(u, ref):
    c = abs(np.dot(u, ref)) / (np.linalg.norm(u) * np.linalg.norm(ref))
    return float(np.arccos(min(1.0, c)))


CASES = {
    "grid64_unit": lambda: inputs.grid2d(64, 64, "unit"),
    "grid_ragged": lambda: inputs.grid2d(45, 71, "uniform", seed=2),
    "grid3d_small": lambda: inputs.grid3d(20, 20, 20, "uniform", seed=1412),
    "random": lambda: inputs.random_connected(4000, 12000, seed=3),
    "random_ties": lambda: inputs.random_connected(2500, 5000, seed=4, ties=True),
    "rgg": lambda: inputs.rgg(6000, 8.0, seed=5),
    "ba": lambda: inputs.barabasi_albert(5000, 4, seed=6),
    "chung_lu": lambda: inputs.chung_lu(30000, seed=7),
    "path": lambda: inputs.path(300),
    "cycle": lambda: inputs.cycle(250),
    "complete": lambda: inputs.complete(40),
    "tiny": lambda: inputs.path(5, [1.0, 2.0, 3.0, 4.0]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fiedler_fp64_matches_oracle(name):
    rp, col, w = CASES[name]()
    seed = 1412
    h = cmg.Hierarchy(rp, col, w, seed=seed)
    u, lam, st = h.fiedler()
    ref_u, ref_lam, ref_res, oh, ref = oracle.fiedler(rp, col, w, seed=seed)
    assert h.sizes()[0] == oh.sizes()
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref_u) <= VEC_TOL
    assert abs(lam - ref_lam) <= LAM_TOL * abs(ref_lam)
    assert st["residual"] == pytest.approx(ref_res, rel=1e-6, abs=1e-13)
    # output contract: unit norm, orthogonal to 1, canonical sign
    assert abs(np.linalg.norm(u) - 1.0) <= 1e-13
    assert abs(u.sum()) <= 1e-12 * np.sqrt(len(u))
    i = int(np.argmax(np.abs(u)))
    assert u[i] > 0
    h.close()


def test_degenerate_graphs():
    # n = 2: B_g annihilates the only vector orthogonal to 1 (R10)
    rp, col, w = inputs.path(2, [0.75])
    u, lam, st = cmg.fiedler(rp, col, w)
    assert np.allclose(np.abs(u), 1 / np.sqrt(2), atol=1e-15) and u[0] * u[1] < 0
    assert lam == pytest.approx(1.5, rel=1e-14)
    # a star collapses into one aggregate: the input is the coarsest level
    rp, col, w = inputs.star(200)
    h = cmg.Hierarchy(rp, col, w)
    assert h.levels == 1
    u, lam, st = h.fiedler()
    ref_u, ref_lam, _, _, _ = oracle.fiedler(rp, col, w)
    assert aligned_err(u, ref_u) <= VEC_TOL and lam == pytest.approx(ref_lam, rel=LAM_TOL)


def test_device_buffers_and_stream():
    rp, col, w = inputs.grid2d(50, 40, "uniform", seed=9)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        drp = torch.from_numpy(rp).cuda()
        dcol = torch.from_numpy(col).cuda()
        dw = torch.from_numpy(w).cuda()
        h = cmg.Hierarchy(drp, dcol, dw, stream=s.cuda_stream)
        u = torch.empty(len(rp) - 1, dtype=torch.float64, device="cuda")
        _, lam, st = h.fiedler(u_out=u, stream=s.cuda_stream)
    s.synchronize()
    ref_u, ref_lam, _, _, _ = oracle.fiedler(rp, col, w)
    assert aligned_err(u.cpu().numpy(), ref_u) <= VEC_TOL
    assert lam == pytest.approx(ref_lam, rel=LAM_TOL)


@pytest.mark.parametrize("name", ["grid3d_small", "chung_lu"])
def test_repeat_solves_are_bitwise_reproducible(name):
    """Fixed-order reductions: repeated solves give identical bits (this also
    covers the sign flip of the final vector, where CTAs must agree)."""
    rp, col, w = CASES[name]()
    h = cmg.Hierarchy(rp, col, w)
    u1, l1, _ = h.fiedler()
    for _ in range(4):
        u2, l2, _ = h.fiedler()
        assert np.array_equal(u1, u2) and l1 == l2
    h2 = cmg.Hierarchy(rp, col, w)
    u3, l3, _ = h2.fiedler()
    assert np.array_equal(u1, u3) and l1 == l3


@pytest.mark.parametrize("schedule", ["fixed", "replay"])
def test_schedules_match_oracle(schedule):
    rp, col, w = inputs.grid2d(90, 70, "uniform", seed=12)
    oh = oracle.Hierarchy(rp, col, w, seed=3)
    if schedule == "fixed":
        ref = oh.solve(schedule="fixed", beta=2.0, k0=2)
        h = cmg.Hierarchy(rp, col, w, seed=3, schedule="fixed", beta=2.0, k0=2)
    else:
        base = oh.solve()
        reps = [max(1, k // 2) for k in base["sweeps"]]
        ref = oh.solve(schedule="replay", replay=reps)
        h = cmg.Hierarchy(rp, col, w, seed=3, schedule="replay", replay_sweeps=reps)
    u, lam, st = h.fiedler()
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref["u"]) <= VEC_TOL
    assert lam == pytest.approx(ref["lam"], rel=LAM_TOL)


# Graphs of the 4,096-graph mixed batch (preferential-attachment graphs with
# about 12,000 sweeps on some coarse level, and a random geometric graph) on
# which FP32 sweeps on every level missed lambda2 within 1e-6 of the oracle:
# the rounding accumulated along the coarse levels' long sweep chains.
FP32_HARD = {f"batch4096_{i}": (lambda i=i: inputs.batch_graph(i)) for i in (671, 1814, 2267, 2933, 2889)}


@pytest.mark.parametrize("name", ["grid64_unit", "grid3d_small", "random", "rgg", "ba", "chung_lu"]
                         + sorted(FP32_HARD))
def test_fp32_sweep_form_accuracy(name):
    """FP32 sweeps (on the levels that carry the bytes) with float-float
    reductions and a final FP64 recompute, against the FP64 oracle run with
    the same per-level sweep counts (the oracle's own tolerance-mode counts,
    replayed), so the comparison measures precision alone: lambda2 within
    1e-6 relative, vector within 1e-4 rad."""
    rp, col, w = (CASES.get(name) or FP32_HARD[name])()
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    ref = oh.solve()
    h = cmg.Hierarchy(rp, col, w, seed=1412, precision="fp32", schedule="replay",
                      replay_sweeps=ref["sweeps"].tolist())
    u32, lam32, st32 = h.fiedler()
    prec = h.level_precision()
    h.close()
    assert st32["sweeps"] == ref["sweeps"].tolist()
    assert all((p == "fp32") == (m >= 2**20) for p, m in zip(prec, st32["nnz"]))
    assert abs(lam32 - ref["lam"]) <= 1e-6 * abs(ref["lam"])
    assert angle(u32, ref["u"]) <= 1e-4


def test_capped_sweeps_warn_but_return_a_vector():
    rp, col, w = inputs.grid2d(60, 60, "uniform", seed=4)
    h = cmg.Hierarchy(rp, col, w, max_sweeps=3, max_sweeps_coarsest=3)
    u, lam, st = h.fiedler()
    assert st["status"] == "WARN_MAXITER"
    assert all(k <= 3 for k in st["sweeps"])
    oh = oracle.Hierarchy(rp, col, w)
    ref = oh.solve(max_sweeps=3, max_sweeps_coarsest=3)
    assert ref["capped"] and aligned_err(u, ref["u"]) <= VEC_TOL


def test_full_size_3d_grid_matches_oracle():
    """The benchmark workload: 100^3 7-point grid, U[0.5, 1.5] weights, seed 1412."""
    rp, col, w = inputs.grid3d(100, 100, 100, "uniform", seed=1412)
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    u, lam, st = h.fiedler()
    ref_u, ref_lam, _, oh, ref = oracle.fiedler(rp, col, w, seed=1412)
    assert h.sizes()[0] == oh.sizes()
    for lvl in range(oh.levels - 1):
        assert np.array_equal(h.aggregates(lvl), oh.agg(lvl))
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref_u) <= VEC_TOL
    assert abs(lam - ref_lam) <= LAM_TOL * abs(ref_lam)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_staged_iterate_kernel_matches_oracle(monkeypatch, precision):
    """The slice kernel that stages the iterate's highest-degree prefix in
    shared memory, forced on every slice level, against the oracle; also the
    same solve with staging off.  (The two launch different CTA counts, so
    their float-float partial sums group differently: they agree within the
    parity tolerances, not bit for bit.)  70,000 vertices: the staged prefix
    (about 57,000 FP32 or 28,500 FP64 entries) is shorter than level 0, so
    both gather paths run."""
    rp, col, w = inputs.chung_lu(70000, seed=11)
    assert len(rp) - 1 > 57344
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    ref64 = oh.solve()
    for mode in ("1", "0"):
        monkeypatch.setenv("CMG_STAGE", mode)
        h = cmg.Hierarchy(rp, col, w, seed=1412, precision=precision)
        kind, staged = h.level_kernels()
        if mode == "0":
            assert 2 not in kind and not any(staged)
        else:
            assert kind[0] == 2 and 0 < staged[0] < len(rp) - 1
            assert all((k == 2) == (s > 0) for k, s in zip(kind, staged))
            assert 1 not in kind
        u, lam, st = h.fiedler()
        for _ in range(2):
            u2, lam2, _ = h.fiedler()
            assert np.array_equal(u, u2) and lam == lam2
        h.close()
        if precision == "fp64":
            assert st["sweeps"] == ref64["sweeps"].tolist()
            assert aligned_err(u, ref64["u"]) <= VEC_TOL
            assert abs(lam - ref64["lam"]) <= LAM_TOL * abs(ref64["lam"])
        else:
            ref = oh.solve(schedule="replay", replay=st["sweeps"])
            assert abs(lam - ref["lam"]) <= 1e-6 * abs(ref["lam"])
            assert angle(u, ref["u"]) <= 1e-4
    monkeypatch.delenv("CMG_STAGE")


def test_stage_rule_picks_dense_power_law_levels():
    """Without the override, staging is chosen where gathers are many per
    staged entry: the dense coarse levels of a power-law graph, not the
    levels of a 3-D grid.  A level whose iterate is far longer than shared
    memory stages a 32,768-entry prefix in the FP32 form when that prefix
    serves at least 3 times its share of the rows (the hub columns: 42 % of
    level 0's gathers for 8.2 % of its rows here)."""
    # levels of this graph: 399,708 / 105,389 / 25,604 / 6,072 / 1,088 rows
    # with 6.4M / 5.7M / 5.3M / 3.8M / 0.65M stored entries
    h = cmg.Hierarchy(*inputs.chung_lu(400000, seed=12), seed=1412, precision="fp32")
    kind, staged = h.level_kernels()
    assert kind[0] == 2 and staged[0] == 32768   # a short prefix of a long iterate
    assert kind[2] == 2 and staged[2] == 25604   # the whole iterate, 5.3M gathers a sweep
    h.close()
    h = cmg.Hierarchy(*inputs.grid3d(60, 60, 60, "uniform", seed=1), seed=1412, precision="fp32")
    kind, staged = h.level_kernels()
    assert 2 not in kind and 1 in kind
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hub_row_split_into_many_chunks_matches_oracle(precision):
    """A heavy row longer than 2,048 entries is cut into chunks that several
    warps sum, and the warp of its last chunk waits for the others and adds
    their partials in chunk order.  A hub of 12,000 entries (6 chunks) on a
    22,501-vertex graph runs that path on level 0 (and its aggregate's row
    on the next levels) at a size the oracle solves in seconds.  The hub's
    weights are scaled by 1e-3 so that its degree does not set the shift
    g far above the grid's degrees (which would stop every level after one
    sweep)."""
    rp, col, w = inputs.hub_grid(150, 150, 12000, seed=31, hub_scale=1e-3)
    assert int(np.diff(rp).max()) == 12000
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    h = cmg.Hierarchy(rp, col, w, seed=1412, precision=precision)
    kind, _ = h.level_kernels()
    assert kind[0] in (1, 2)                 # level 0 runs the slice kernel
    u, lam, st = h.fiedler()
    u2, lam2, _ = h.fiedler()
    assert np.array_equal(u, u2) and lam == lam2
    h.close()
    if precision == "fp64":
        ref = oh.solve()
        assert st["sweeps"] == ref["sweeps"].tolist()
        assert aligned_err(u, ref["u"]) <= VEC_TOL
        assert abs(lam - ref["lam"]) <= LAM_TOL * abs(ref["lam"])
    else:
        ref = oh.solve(schedule="replay", replay=st["sweeps"])
        assert abs(lam - ref["lam"]) <= 1e-6 * abs(ref["lam"])
        assert angle(u, ref["u"]) <= 1e-4
