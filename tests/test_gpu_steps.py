"""Per-step parity of the CUDA path against the CPU oracle (through the C-ABI).

Integer and structural steps (heaviest neighbour, visit ranks, aggregates,
coarse sparsity and coarse weights) must match bit for bit; FP64 power
sweeps and the Rayleigh quotient within a few ulps times the sweep count.
"""
import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(rp, col, w):
    return (torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(col).cuda(),
            torch.from_numpy(w).cuda())


GRAPHS = {
    "grid64": lambda: inputs.grid2d(64, 64, "unit"),
    "grid_ragged": lambda: inputs.grid2d(37, 53, "uniform", seed=3),
    "grid3d": lambda: inputs.grid3d(21, 17, 13, "uniform", seed=5),
    "random_ties": lambda: inputs.random_connected(3000, 6000, seed=7, ties=True),
    "random_real": lambda: inputs.random_connected(5000, 20000, seed=8),
    "rgg": lambda: inputs.rgg(4000, 8.0, seed=9),
    "ba": lambda: inputs.barabasi_albert(3000, 4, seed=10),
    "chung_lu": lambda: inputs.chung_lu(20000, seed=11),
    "star": lambda: inputs.star(300),
    "path2": lambda: inputs.path(2, [0.5]),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_heaviest_neighbour_bit_exact(name):
    rp, col, w = GRAPHS[name]()
    m = cmg.heaviest_neighbour(*dev(rp, col, w)).cpu().numpy()
    assert np.array_equal(m, oracle.heaviest_neighbour(rp, col, w))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 1000, 4097, 65536, 100003, 1 << 20])
def test_visit_ranks_bit_exact(n):
    for level in (0, 3):
        r = cmg.visit_ranks(n, 1412, level).cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        assert np.array_equal(r, oracle.visit_ranks(1412, level, n))


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_hec_aggregates_bit_exact(name):
    rp, col, w = GRAPHS[name]()
    n = len(rp) - 1
    for seed in (0, 1):
        rank = oracle.visit_ranks(seed, 0, n)
        agg_ref, c_ref = oracle.hec(rp, col, w, rank)
        drp, dcol, dw = dev(rp, col, w)
        agg, c = cmg.hec_aggregate(drp, dcol, dw, torch.from_numpy(rank.astype(np.int32)).cuda())
        assert c == c_ref
        assert np.array_equal(agg.cpu().numpy(), agg_ref)


def test_hec_exhaustive_small_graphs_all_orders():
    """Every visit order of many small connected graphs (weights with ties).
    The graphs run as one block-diagonal graph: Alg. 2 on a disjoint union
    equals Alg. 2 on each component with the induced order, so order t of
    every component is checked in one call (t over all 6! orders; smaller
    graphs cycle through theirs).  Random interleaved global orders follow."""
    import itertools
    rng = np.random.default_rng(0)
    graphs = []
    for n in range(2, 7):
        for s in range(10):
            graphs.append(inputs.random_connected(n, int(rng.integers(0, 2 * n)),
                                                  seed=1000 * n + s, ties=True))
    rp, col, w, offs = inputs.concat_csr(graphs)
    N = len(rp) - 1
    drp, dcol, dw = dev(rp, col, w)
    perms = {n: list(itertools.permutations(range(n))) for n in range(2, 7)}

    def check(rank):
        agg_ref, c_ref = oracle.hec(rp, col, w, rank)
        agg, c = cmg.hec_aggregate(drp, dcol, dw, torch.from_numpy(rank.astype(np.int32)).cuda())
        assert c == c_ref
        assert np.array_equal(agg.cpu().numpy(), agg_ref)

    for t in range(720):
        rank = np.empty(N, dtype=np.int64)
        for g in range(len(graphs)):
            n = int(offs[g + 1] - offs[g])
            rank[offs[g]:offs[g + 1]] = offs[g] + np.array(perms[n][t % len(perms[n])])
        check(rank)
    for t in range(50):
        check(rng.permutation(N))


@pytest.mark.parametrize("name", ["grid64", "grid3d", "random_real", "chung_lu", "rgg", "ba"])
def test_hierarchy_levels_bit_exact(name):
    """Every level: aggregates, coarse sparsity and coarse FP64 weights."""
    rp, col, w = GRAPHS[name]()
    h = cmg.Hierarchy(rp, col, w, seed=77)
    ref = oracle.Hierarchy(rp, col, w, seed=77)
    assert h.sizes()[0] == ref.sizes()
    for lvl in range(ref.levels):
        grp, gcol, gw, gg = h.level_csr(lvl)
        rrp, rcol, rw = ref.csr(lvl)
        assert np.array_equal(grp, rrp) and np.array_equal(gcol, rcol)
        assert np.array_equal(gw.view(np.int64), rw.view(np.int64)), lvl
        assert gg == ref.info(lvl)[2]
        if lvl < ref.levels - 1:
            assert np.array_equal(h.aggregates(lvl), ref.agg(lvl))
    h.close()


@pytest.mark.parametrize("name", ["grid_ragged", "random_real", "chung_lu"])
@pytest.mark.parametrize("k", [0, 1, 7, 60])
def test_power_sweeps_match_oracle(name, k):
    rp, col, w = GRAPHS[name]()
    n = len(rp) - 1
    x0 = oracle.gaussian_start(3, n)
    u_ref, _, cos_ref, _ = oracle.power_iteration(rp, col, w, x0, fixed=k)
    drp, dcol, dw = dev(rp, col, w)
    u, cs = cmg.power_sweeps(drp, dcol, dw, torch.from_numpy(x0).cuda(), k)
    u = u.cpu().numpy()
    err = np.linalg.norm(u - u_ref)
    assert err <= 1e-14 * max(1, k) * np.sqrt(n), err
    if k > 0:
        assert abs(cs - cos_ref) <= 1e-13


@pytest.mark.parametrize("name", ["grid64", "random_real", "chung_lu", "ba"])
def test_rayleigh_residual_match_oracle(name):
    rp, col, w = GRAPHS[name]()
    n = len(rp) - 1
    u = oracle.gaussian_start(5, n)
    lam_ref, res_ref = oracle.rayleigh_residual(rp, col, w, u)
    drp, dcol, dw = dev(rp, col, w)
    lam, res = cmg.rayleigh_residual(drp, dcol, dw, torch.from_numpy(u).cuda())
    assert lam == pytest.approx(lam_ref, rel=1e-13)
    assert res == pytest.approx(res_ref, rel=1e-12)
