"""The seeded synthetic inputs match their stated recipes (no GPU).

Every graph the tests and the bench use comes from inputs.py; these checks
pin the structure those recipes promise: a valid symmetric CSR without
self-loops, the stated sizes, weight distributions and mean degrees, one
connected component where the recipe keeps the largest, a power-law degree
tail for Chung-Lu, and identical output for identical seeds.
"""
import numpy as np
import pytest

from paper_1412_0565_gb300 import inputs

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import connected_components  # noqa: E402


def check_csr(rp, col, w):
    n = len(rp) - 1
    assert rp.dtype == np.int64 and col.dtype == np.int32 and w.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == len(col) == len(w)
    assert np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.all((col >= 0) & (col < n))
    assert not np.any(rows == col), "self-loop"
    # columns strictly ascending within each row (no duplicate entries)
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    assert np.all(w > 0) and np.all(np.isfinite(w))
    A = scipy_sparse.csr_matrix((w, col, rp), shape=(n, n))
    D = (A - A.T).tocoo()
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0, "not symmetric"
    return n, A


def n_components(A):
    return connected_components(A, directed=False)[0]


def test_grid_sizes_match_the_recipes():
    rp, col, w = inputs.grid2d(64, 64, "unit")
    n, _ = check_csr(rp, col, w)
    assert (n, len(col)) == (4096, 16128)          # 64x64 5-point grid
    assert np.all(w == 1.0)
    rp, col, w = inputs.grid3d(10, 11, 12, "uniform", seed=3)
    n, A = check_csr(rp, col, w)
    edges = 9 * 11 * 12 + 10 * 10 * 12 + 10 * 11 * 11
    assert (n, len(col)) == (10 * 11 * 12, 2 * edges)
    # the 100^3 grid of the benchmark: 2 * 3 * 99 * 100^2 entries
    assert 2 * 3 * 99 * 100 ** 2 == 5_940_000
    assert w.min() >= 0.5 and w.max() <= 1.5
    assert n_components(A) == 1
    # vertex (x, y, z) has id (z b + y) a + x: the x-neighbour of 0 is 1
    assert col[rp[0]] == 1


def test_uniform_weights_are_uniform():
    rp, col, w = inputs.grid3d(30, 30, 30, "uniform", seed=5)
    check_csr(rp, col, w)
    assert w.min() >= 0.5 and w.max() <= 1.5
    assert abs(w.mean() - 1.0) < 0.01
    assert abs(w.var() - 1.0 / 12.0) < 0.003


def test_same_seed_same_graph_other_seed_other_graph():
    for make in (lambda s: inputs.grid2d(20, 30, "uniform", seed=s),
                 lambda s: inputs.rgg(3000, 8.0, seed=s),
                 lambda s: inputs.barabasi_albert(3000, 4, seed=s),
                 lambda s: inputs.chung_lu(5000, seed=s),
                 lambda s: inputs.random_connected(2000, 4000, seed=s)):
        a, b, c = make(11), make(11), make(12)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
        assert not (len(a[1]) == len(c[1]) and np.array_equal(a[1], c[1]) and np.array_equal(a[2], c[2]))


def test_random_geometric_graph_mean_degree_and_connectivity():
    rp, col, w = inputs.rgg(20000, 8.0, seed=21)
    n, A = check_csr(rp, col, w)
    assert n_components(A) == 1                  # largest component kept
    assert n > 0.97 * 20000                       # at mean degree 8 nearly all of it
    assert 7.2 < len(col) / n < 8.4               # mean degree about 8 (boundary effects lower it)
    assert w.min() >= 0.5 and w.max() <= 1.5


def test_barabasi_albert_edges_hubs_and_connectivity():
    n, m = 20000, 4
    rp, col, w = inputs.barabasi_albert(n, m, seed=22)
    n2, A = check_csr(rp, col, w)
    assert n2 == n and n_components(A) == 1
    full = (m + 1) * m // 2 + (n - m - 1) * m    # edges before merging repeated targets
    assert 0.97 * full <= len(col) // 2 <= full
    deg = np.diff(rp)
    assert deg.min() >= 1
    assert deg.max() > 20 * (len(col) / n)        # preferential attachment makes hubs


def test_chung_lu_mean_degree_cap_tail_and_weights():
    n0 = 60000
    rp, col, w = inputs.chung_lu(n0, seed=23)
    n, A = check_csr(rp, col, w)
    assert n_components(A) == 1
    assert 0.9 * n0 < n <= n0
    deg = np.diff(rp)
    assert 15.0 < deg.mean() < 17.0              # mean degree 16 (the largest component)
    assert deg.max() <= 1.5 * np.sqrt(16 * n0)   # expected degrees capped at sqrt(16 n)
    # degree tail: P(deg >= k) ~ k^-(gamma - 1) = k^-1.5 between 32 and 256
    ks = np.array([32, 64, 128, 256])
    ccdf = np.array([(deg >= k).mean() for k in ks])
    slope = np.polyfit(np.log(ks), np.log(ccdf), 1)[0]
    assert -1.9 < slope < -1.1
    lw = np.log(w)
    assert abs(lw.mean()) < 0.02 and abs(lw.std() - 1.0) < 0.02   # lognormal(0, 1)


def test_random_connected_is_connected_and_ties_are_small_integers():
    rp, col, w = inputs.random_connected(3000, 6000, seed=24, ties=True)
    n, A = check_csr(rp, col, w)
    assert n == 3000 and n_components(A) == 1
    assert set(np.unique(w).tolist()) <= {1.0, 2.0, 3.0}


def test_batch_and_serving_sizes():
    s = inputs.batch_sizes(4096, 500, 20000, seed=1412)
    assert len(s) == 4096 and s.min() >= 499 and s.max() <= 20000
    # log-uniform: log n has mean (ln 500 + ln 20000) / 2 and uniform spread
    ls = np.log(s + 0.5)
    assert abs(ls.mean() - 0.5 * (np.log(500) + np.log(20000))) < 0.06
    assert abs(ls.std() - (np.log(20000) - np.log(500)) / np.sqrt(12)) < 0.05
    r = inputs.serving_sizes(2000, 1e3, 2e6, seed=1412)
    assert len(r) == 2000 and r.min() >= 999 and r.max() <= 2_000_000
    lr = np.log(r + 0.5)
    a, b = np.log(1e3), np.log(2e6)
    assert abs(lr.mean() - 0.5 * (a + b)) < 0.1


def test_batch_families_and_union():
    gs = inputs.batch_graphs(6, 500, 2000, seed=5)
    sizes = inputs.batch_sizes(6, 500, 2000, seed=5)
    for i, g in enumerate(gs):
        n, A = check_csr(*g)
        assert n_components(A) == 1
        if i % 3 == 1:        # near-square grid with at least the requested vertices
            assert n >= sizes[i]
        else:                 # RGG (largest component) and BA: at most the requested count
            assert n <= sizes[i]
    rp, col, w, offs = inputs.concat_csr(gs)
    n, A = check_csr(rp, col, w)
    assert n == offs[-1] and n_components(A) == len(gs)
    for q in range(len(gs)):
        lo, hi = offs[q], offs[q + 1]
        blk = col[rp[lo]:rp[hi]]
        assert blk.min() >= lo and blk.max() < hi   # block diagonal
