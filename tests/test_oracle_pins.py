"""Pins of the CPU oracle against what the paper and the mathematics fix.

The oracle (oracle/cmg_oracle.c) is the definition the CUDA path is compared
with, so it is itself checked here against things other than itself:
published generator outputs, closed-form spectra, invariants the paper proves
(Lemma 2.6, Proposition 2.7, Theorem 2.8), hand-worked examples of Alg. 2,
Table 3's level sizes, brute-force dense eigensolvers and library routines.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1412_0565_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_laplacian(rp, col, w):
    n = len(rp) - 1
    W = np.zeros((n, n))
    for i in range(n):
        W[i, col[rp[i]:rp[i + 1]]] = w[rp[i]:rp[i + 1]]
    return np.diag(W.sum(axis=1)) - W


def align(u, ref):
    return u if np.dot(u, ref) >= 0 else -u


def subspace_residual(u, Q):
    Q, _ = np.linalg.qr(Q)
    return np.linalg.norm(u - Q @ (Q.T @ u)) / np.linalg.norm(u)


# ------------------------------------------------------------------ generators
def test_splitmix64_published_outputs():
    """SplitMix64 (Steele, Lea, Flood 2014): published reference outputs."""
    G = 0x9E3779B97F4A7C15
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for row in rows:
        state = int(row[0], 0)
        for k, out in enumerate(row[1:]):
            assert oracle.splitmix64((state + k * G) & 0xFFFFFFFFFFFFFFFF) == int(out, 0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 16, 17, 63, 64, 65, 100, 255, 256, 1000, 4097])
def test_visit_ranks_are_a_permutation(n):
    """Alg. 2's randperm: the ranks must be a bijection onto [0, n)."""
    for level in (0, 1, 5):
        r = oracle.visit_ranks(1412, level, n)
        assert sorted(r.tolist()) == list(range(n))


def test_visit_ranks_depend_on_seed_and_level_and_look_random():
    n = 20000
    r0 = oracle.visit_ranks(1412, 0, n)
    r1 = oracle.visit_ranks(1412, 1, n)
    r2 = oracle.visit_ranks(7, 0, n)
    assert (r0 != r1).mean() > 0.99 and (r0 != r2).mean() > 0.99
    # rank correlation with the identity is O(1/sqrt(n)) for a random permutation
    for r in (r0, r1, r2):
        rho = np.corrcoef(np.arange(n), r)[0, 1]
        assert abs(rho) < 5.0 / np.sqrt(n)


def test_gaussian_start_is_standard_normal():
    """Alg. 1 Step 2's randn: Box-Muller must give N(0, 1) samples."""
    import scipy.stats as st
    x = oracle.gaussian_start(1412, 200000)
    assert abs(x.mean()) < 5.0 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 5.0 * np.sqrt(2.0 / x.size)
    assert st.kstest(x, "norm").pvalue > 1e-4
    y = oracle.gaussian_start(1413, 50)
    assert not np.array_equal(y, x[:50])


# ------------------------------------------------------------------ S1: argmax
@pytest.mark.parametrize("seed", range(5))
def test_heaviest_neighbour_brute_force(seed):
    rp, col, w = inputs.random_connected(300, 600, seed=seed, ties=(seed % 2 == 0))
    m = oracle.heaviest_neighbour(rp, col, w)
    L = dense_laplacian(rp, col, w)
    for v in range(len(rp) - 1):
        colv = L[:, v].copy()
        # argmin of the column of L; numpy returns the first (lowest) index
        assert m[v] == int(np.argmin(colv))


def test_heaviest_neighbour_pointer_graph_has_only_two_cycles():
    """With lowest-index ties, following v -> m(v) never closes a cycle longer than 2."""
    for seed in range(6):
        rp, col, w = inputs.random_connected(400, 900, seed=seed, ties=True)
        m = oracle.heaviest_neighbour(rp, col, w)
        n = len(m)
        for v in range(n):
            x, seen = v, []
            for _ in range(n + 1):
                seen.append(x)
                x = int(m[x])
                if x in seen:
                    cyc = seen[seen.index(x):]
                    assert len(cyc) == 2
                    break


# ------------------------------------------------------------------ S2-S4: HEC
def test_hec_hand_worked_path():
    """Path 0-1-2-3 with weights 1, 3, 2: m = (1, 2, 1, 2).
    Visit order 3, 0, 1, 2: vertex 3 creates {3, 2} as aggregate 0, vertex 0
    creates {0, 1} as aggregate 1, vertices 1 and 2 are already mapped.
    Visit order 1, 0, 3, 2: vertex 1 creates {1, 2}; 0 and 3 join it (c = 1)."""
    rp, col, w = inputs.path(4, [1.0, 3.0, 2.0])
    assert oracle.heaviest_neighbour(rp, col, w).tolist() == [1, 2, 1, 2]
    agg, c = oracle.hec(rp, col, w, rank=[1, 2, 3, 0])
    assert c == 2 and agg.tolist() == [1, 1, 0, 0]
    agg, c = oracle.hec(rp, col, w, rank=[1, 0, 3, 2])
    assert c == 1 and agg.tolist() == [0, 0, 0, 0]


def test_hec_heavy_matching_is_order_independent():
    """If the heaviest edges form a perfect matching, every visit order yields
    exactly the matched pairs (Alg. 2 then coincides with heavy edge matching)."""
    n = 40
    wts = np.where(np.arange(n - 1) % 2 == 0, 3.0, 1.0)
    rp, col, w = inputs.path(n, wts)
    for s in range(10):
        agg, c = oracle.hec(rp, col, w, oracle.visit_ranks(s, 0, n))
        assert c == n // 2
        for i in range(0, n, 2):
            assert agg[i] == agg[i + 1]
        assert len(set(agg.tolist())) == n // 2


def test_hec_star_collapses_to_one_aggregate():
    rp, col, w = inputs.star(30)
    for s in range(8):
        agg, c = oracle.hec(rp, col, w, oracle.visit_ranks(s, 0, 30))
        assert c == 1 and (agg == 0).all()


def _check_hec_invariants(rp, col, w, rank, agg, c):
    n = len(rp) - 1
    # labels are a surjection onto 0..c-1 (I^T 1 = 1: one aggregate per vertex)
    assert agg.min() == 0 and agg.max() == c - 1
    sizes = np.bincount(agg, minlength=c)
    # Lemma 2.6: every aggregate has >= 2 vertices, so c <= n/2
    assert sizes.min() >= 2 and c <= n // 2
    # aggregates are numbered in the order their creators are visited
    order = np.argsort(rank)
    first_seen = []
    seen = set()
    for v in order:
        a = int(agg[v])
        if a not in seen:
            seen.add(a)
            first_seen.append(a)
    assert first_seen == list(range(c))
    # each aggregate is connected in the fine graph
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    rows = np.repeat(np.arange(n), np.diff(rp))
    same = agg[rows] == agg[col]
    A = sp.coo_matrix((np.ones(same.sum()), (rows[same], col[same])), shape=(n, n))
    ncomp, _ = connected_components(A, directed=False)
    assert ncomp == c


@pytest.mark.parametrize("seed", range(4))
def test_hec_invariants_random_graphs(seed):
    rp, col, w = inputs.random_connected(500, 800, seed=seed, ties=(seed % 2 == 1))
    rank = oracle.visit_ranks(seed, 0, 500)
    agg, c = oracle.hec(rp, col, w, rank)
    _check_hec_invariants(rp, col, w, rank, agg, c)


def test_hec_invariants_grids():
    for (a, b, wt) in [(30, 20, "unit"), (17, 23, "uniform")]:
        rp, col, w = inputs.grid2d(a, b, wt, seed=3)
        rank = oracle.visit_ranks(11, 0, a * b)
        agg, c = oracle.hec(rp, col, w, rank)
        _check_hec_invariants(rp, col, w, rank, agg, c)


def test_level_sizes_match_table3():
    """Table 3: the unit 100x100 grid coarsens as 10000, 3653, 1195, 384, 137,
    46, 14.  The visit order is random, so the mean over seeds is compared
    (within 10%, or 3 vertices on the two smallest levels where one vertex is
    already 2-7%) on the levels the paper lists."""
    with open(os.path.join(GOLDEN, "table3_level_sizes.txt")) as f:
        paper = [int(x) for l in f if l.strip() and not l.startswith("#") for x in l.split()]
    rp, col, w = inputs.grid2d(100, 100, "unit")
    runs = [oracle.Hierarchy(rp, col, w, seed=s).sizes() for s in range(8)]
    depth = min(len(r) for r in runs)
    assert depth >= 6
    for lvl in range(1, min(depth, len(paper))):
        mean = np.mean([r[lvl] for r in runs])
        assert abs(mean - paper[lvl]) <= max(0.10 * paper[lvl], 3.0), (lvl, mean, paper[lvl])
    # the coarsest level is the first with <= 25 vertices (Alg. 1's while loop)
    for r in runs:
        assert r[-1] <= 25 and all(x > 25 for x in r[:-1])


# ------------------------------------------------------------------ S5: Galerkin
def _galerkin_check(rp, col, w, seed, exact):
    h = oracle.Hierarchy(rp, col, w, seed=seed, coarse_size=2, max_levels=2)
    assert h.levels == 2
    agg = h.agg(0)
    n, c = len(rp) - 1, h.info(1)[0]
    rpc, colc, wc = h.csr(1)
    L = dense_laplacian(rp, col, w)
    P = np.zeros((c, n))
    P[agg, np.arange(n)] = 1.0
    Lc = P @ L @ P.T                      # explicit I L I^T
    Wc = np.zeros((c, c))
    for a in range(c):
        Wc[a, colc[rpc[a]:rpc[a + 1]]] = wc[rpc[a]:rpc[a + 1]]
        assert np.all(np.diff(colc[rpc[a]:rpc[a + 1]]) > 0)        # sorted, unique
        assert a not in colc[rpc[a]:rpc[a + 1]]                     # no diagonal stored
    assert np.array_equal(Wc, Wc.T)                                 # bitwise symmetric
    assert np.all(wc > 0)                                           # off-diagonals of L_c < 0
    off = -Lc.copy()
    np.fill_diagonal(off, 0.0)
    if exact:
        assert np.array_equal(off, Wc)
    else:
        assert np.allclose(off, Wc, rtol=64 * np.finfo(float).eps, atol=0)
    # Proposition 2.7(2): L_c 1 = 0, i.e. diag(L_c) = coarse row sums
    assert np.allclose(np.diag(Lc), Wc.sum(axis=1), rtol=1e-13)
    # Proposition 2.7(3): restriction keeps 1-perp
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(n)
    u -= u.mean()
    assert abs((P @ u).sum()) <= 1e-12 * np.abs(u).sum()
    # coarse graph is connected
    from scipy.sparse.csgraph import connected_components
    import scipy.sparse as sp
    ncomp, _ = connected_components(sp.csr_matrix(Wc), directed=False)
    assert ncomp == 1


@pytest.mark.parametrize("seed", range(3))
def test_galerkin_equals_triple_product_integer_weights(seed):
    rp, col, w = inputs.random_connected(300, 700, seed=seed, ties=True)
    _galerkin_check(rp, col, w, seed, exact=True)


@pytest.mark.parametrize("seed", range(3))
def test_galerkin_equals_triple_product_real_weights(seed):
    rp, col, w = inputs.random_connected(300, 700, seed=seed + 10)
    _galerkin_check(rp, col, w, seed, exact=False)


def test_galerkin_canonical_summation_order():
    """R5: w_ab is the left-to-right sum over fine pairs in (i, j) order.  Weights
    1, 2^-53, 2^-53 summed in that order give 1 (each tiny term rounds away); the
    other orders would give 1 + 2^-52.  Fine graph: vertices 0,1 (aggregate A) and
    2,3 (aggregate B) with heavy internal edges 0-1 and 2-3 and cross edges
    0-2 (1), 0-3 (2^-53), 1-3 (2^-53)."""
    t = 2.0 ** -53
    u = [0, 2, 0, 0, 1]
    v = [1, 3, 2, 3, 3]
    ww = [10.0, 10.0, 1.0, t, t]
    rp, col, w = inputs.csr_from_edges(4, u, v, ww)
    h = oracle.Hierarchy(rp, col, w, seed=0, coarse_size=1, max_levels=2)
    assert h.levels == 2 and h.info(1)[0] == 2
    rpc, colc, wc = h.csr(1)
    assert wc.tolist() == [1.0, 1.0]


# ------------------------------------------------------------------ S9/S10: PI, RQ
def test_rayleigh_residual_exact_eigenpair():
    n = 30
    rp, col, w = inputs.path(n)
    i = np.arange(n)
    phi = np.cos(np.pi * (i + 0.5) / n)
    lam, res = oracle.rayleigh_residual(rp, col, w, phi)
    assert abs(lam - (2 - 2 * np.cos(np.pi / n))) <= 1e-14
    assert res <= 1e-14


def test_gershgorin_shift():
    rp, col, w = inputs.random_connected(100, 200, seed=1)
    L = dense_laplacian(rp, col, w)
    assert oracle.gershgorin(rp, col, w) == pytest.approx(np.abs(L).sum(axis=1).max(), rel=1e-15)


def test_power_iteration_contraction_rate():
    """Theorem 2.8 on B_g: the tangent of the angle to the Fiedler vector
    contracts by (g - lambda3)/(g - lambda2) per sweep (path P_n)."""
    n = 24
    rp, col, w = inputs.path(n)
    g = oracle.gershgorin(rp, col, w)
    lam = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    phi2 = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    phi2 /= np.linalg.norm(phi2)
    y0 = oracle.gaussian_start(5, n)
    tans = []
    for k in (200, 260):
        u, kk, _, _ = oracle.power_iteration(rp, col, w, y0, fixed=k)
        c = abs(np.dot(u, phi2))
        tans.append(np.sqrt(1 - c * c) / c)
    rate = (tans[1] / tans[0]) ** (1.0 / 60)
    assert rate == pytest.approx((g - lam[2]) / (g - lam[1]), rel=1e-2)


def test_power_iteration_stops_on_cosine_rule():
    rp, col, w = inputs.grid2d(12, 9, "uniform", seed=2)
    y0 = oracle.gaussian_start(3, 108)
    u, k, c, capped = oracle.power_iteration(rp, col, w, y0, tol=1e-8)
    assert k >= 1 and c >= 1 - 1e-8 and not capped
    # one sweep fewer would not have met the rule
    u1, _, c1, _ = oracle.power_iteration(rp, col, w, y0, fixed=k - 1)
    if k > 1:
        assert c1 < 1 - 1e-8
    # each iterate is orthogonal to 1 and normalised
    assert abs(u.sum()) <= 1e-14 * np.sqrt(108)
    assert abs(np.linalg.norm(u) - 1) <= 1e-14


def test_two_vertex_graph():
    """n = 2: the only vector orthogonal to 1 is (1, -1)/sqrt(2), lambda2 = 2w
    (B_g annihilates it; the iteration stops on the eigenvector)."""
    rp, col, w = inputs.path(2, [0.75])
    u, lam, res, h, r = oracle.fiedler(rp, col, w)
    assert h.levels == 1
    # +-(1, -1)/sqrt(2); the sign rule sees a tie up to rounding
    assert np.allclose(align(u, np.array([1.0, -1.0])), [1 / np.sqrt(2), -1 / np.sqrt(2)], atol=1e-15)
    assert lam == pytest.approx(1.5, rel=1e-15) and res <= 1e-15


# ------------------------------------------------------------------ closed forms (converged mode)
def _converged(rp, col, w, seed=1412):
    # vector error ~ residual / (lambda3 - lambda2): drive the residual to 1e-14 g
    u, lam, res, h, r = oracle.fiedler(rp, col, w, seed=seed, converged=True, conv_rtol=1e-14)
    assert res <= 1e-14 * oracle.gershgorin(rp, col, w)
    return u, lam, res


def test_closed_form_path():
    n = 40
    rp, col, w = inputs.path(n)
    u, lam, res = _converged(rp, col, w)
    phi = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    phi /= np.linalg.norm(phi)
    assert lam == pytest.approx(2 - 2 * np.cos(np.pi / n), rel=1e-12)
    assert np.linalg.norm(align(u, phi) - phi) <= 1e-9


def test_closed_form_cycle_double_eigenvalue():
    n = 30
    rp, col, w = inputs.cycle(n)
    u, lam, res = _converged(rp, col, w)
    i = np.arange(n)
    Q = np.stack([np.cos(2 * np.pi * i / n), np.sin(2 * np.pi * i / n)], axis=1)
    assert lam == pytest.approx(2 - 2 * np.cos(2 * np.pi / n), rel=1e-12)
    assert subspace_residual(u, Q) <= 1e-9


def test_closed_form_rectangular_grid():
    a, b = 14, 9
    rp, col, w = inputs.grid2d(a, b, "unit")
    u, lam, res = _converged(rp, col, w)
    x = np.tile(np.arange(a), b)
    phi = np.cos(np.pi * (x + 0.5) / a)
    phi /= np.linalg.norm(phi)
    assert lam == pytest.approx(2 - 2 * np.cos(np.pi / a), rel=1e-12)
    assert np.linalg.norm(align(u, phi) - phi) <= 1e-9


def test_closed_form_square_grid_double_eigenvalue():
    a = 12
    rp, col, w = inputs.grid2d(a, a, "unit")
    u, lam, res = _converged(rp, col, w)
    x = np.tile(np.arange(a), a)
    y = np.repeat(np.arange(a), a)
    Q = np.stack([np.cos(np.pi * (x + 0.5) / a), np.cos(np.pi * (y + 0.5) / a)], axis=1)
    assert lam == pytest.approx(2 - 2 * np.cos(np.pi / a), rel=1e-12)
    assert subspace_residual(u, Q) <= 1e-9


def test_closed_form_complete_and_star():
    rp, col, w = inputs.complete(12)
    u, lam, res = _converged(rp, col, w)
    assert lam == pytest.approx(12.0, rel=1e-12) and abs(u.sum()) < 1e-13
    rp, col, w = inputs.star(15)
    u, lam, res = _converged(rp, col, w)
    assert lam == pytest.approx(1.0, rel=1e-12)
    assert abs(u[0]) < 1e-9 and abs(u.sum()) < 1e-13   # the centre is a node of every lambda=1 vector


def test_weighted_path_against_tridiagonal_solver():
    rng = np.random.default_rng(7)
    n = 60
    wts = rng.uniform(0.5, 1.5, n - 1)
    rp, col, w = inputs.path(n, wts)
    d = np.zeros(n)
    d[:-1] += wts
    d[1:] += wts
    ev, V = sla.eigh_tridiagonal(d, -wts)
    u, lam, res = _converged(rp, col, w)
    assert lam == pytest.approx(ev[1], rel=1e-12)
    assert np.linalg.norm(align(u, V[:, 1]) - V[:, 1]) <= 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs_against_dense_eigensolver(seed):
    n = [40, 90, 150, 200][seed]
    rp, col, w = inputs.random_connected(n, 2 * n, seed=100 + seed)
    ev, V = np.linalg.eigh(dense_laplacian(rp, col, w))
    u, lam, res = _converged(rp, col, w, seed=seed)
    assert lam == pytest.approx(ev[1], rel=1e-12)
    if (ev[2] - ev[1]) > 1e-3 * ev[1]:
        assert np.linalg.norm(align(u, V[:, 1]) - V[:, 1]) <= 1e-8


@pytest.mark.parametrize("seed", range(3))
def test_cmg_default_mode_courant_fischer(seed):
    """Default (tolerance) mode is approximate; it must still satisfy
    lambda~ >= lambda2 (Courant-Fischer, u orthogonal to 1), be normalised,
    orthogonal to 1, and carry the canonical sign."""
    rp, col, w = inputs.random_connected(180, 400, seed=200 + seed)
    ev = np.linalg.eigvalsh(dense_laplacian(rp, col, w))
    g = oracle.gershgorin(rp, col, w)
    u, lam, res, h, r = oracle.fiedler(rp, col, w, seed=seed)
    assert lam >= ev[1] - 1e-14 * g
    assert abs(np.linalg.norm(u) - 1) <= 1e-14
    assert abs(u.sum()) <= 1e-14 * np.sqrt(len(u)) * 10
    i = int(np.argmax(np.abs(u)))
    assert u[i] > 0
    assert (r["sweeps"] >= 1).all()


def test_fixed_and_replay_schedules():
    rp, col, w = inputs.grid2d(40, 30, "uniform", seed=5)
    h = oracle.Hierarchy(rp, col, w, seed=9)
    J = h.levels - 1
    r = h.solve(schedule="fixed", beta=2.0, k0=3)
    for j in range(J):
        assert r["sweeps"][j] == int(np.ceil(3 * 2.0 ** j))
    t = h.solve()
    rr = h.solve(schedule="replay", replay=t["sweeps"])
    assert np.array_equal(rr["sweeps"], t["sweeps"])
    assert np.array_equal(rr["u"], t["u"])


# ------------------------------------------------------------------ Alg. 1 Step 3: the cascade
def _prolongation_matrix(agg, n_coarse):
    """(I_j^{j+1})^T of Sec. 2 Step 1 as an explicit 0/1 matrix: row i has its
    one 1 in the column of vertex i's aggregate."""
    import scipy.sparse as sp
    n = len(agg)
    return sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, n_coarse))


def _fiedler_space(L, rel=1e-6):
    """Eigenvectors of L whose eigenvalue is lambda2 within `rel` (dense)."""
    ev, V = np.linalg.eigh(L)
    keep = [i for i in range(1, len(ev)) if ev[i] <= ev[1] * (1 + rel) + 1e-14]
    return V[:, keep]


def _subspace_cosine(x, Q):
    x = x - x.mean()
    x = x / np.linalg.norm(x)
    Q, _ = np.linalg.qr(Q)
    return float(np.linalg.norm(Q.T @ x))


_CASCADE_GRAPHS = {
    "grid_64x64_unit": lambda: inputs.grid2d(64, 64, "unit"),
    "grid_14x9_unit": lambda: inputs.grid2d(14, 9, "unit"),
    "grid_40x30_uniform": lambda: inputs.grid2d(40, 30, "uniform", seed=5),
    "rgg_1500": lambda: inputs.rgg(1500, seed=3),
    "path_300": lambda: inputs.path(300),
}


@pytest.mark.parametrize("name", ["grid_14x9_unit", "grid_40x30_uniform", "rgg_1500", "random_200"])
def test_cascade_prolongs_with_the_explicit_transposed_restriction(name):
    """Alg. 1 Step 3: the start of level j is (I_j^{j+1})^T applied to the
    coarse result, with the restriction I_j^{j+1} of that same level j (Sec. 2
    Step 1: (I)_pq = 1 iff q is in aggregate p), entry for entry; the coarsest
    level starts from randn (Step 2).  Checked against an explicitly assembled
    sparse matrix product on every level of each hierarchy."""
    if name == "random_200":
        rp, col, w = inputs.random_connected(200, 400, seed=103)
    else:
        rp, col, w = _CASCADE_GRAPHS[name]()
    h = oracle.Hierarchy(rp, col, w, seed=21)
    J = h.levels - 1
    assert J >= 2
    r = h.solve(trace=True)
    sizes = h.sizes()
    assert np.array_equal(r["start"][J], oracle.gaussian_start(21, sizes[J]))
    for j in range(J):
        P = _prolongation_matrix(h.agg(j), sizes[j + 1])
        assert np.array_equal(r["start"][j], P @ r["end"][j + 1])
        # each level's result is a unit vector orthogonal to 1 (Alg. 3)
        assert abs(np.linalg.norm(r["end"][j]) - 1) <= 1e-14
        assert abs(r["end"][j].sum()) <= 1e-13 * np.sqrt(sizes[j])
    # the returned vector is level 0's result with the sign rule applied
    assert np.array_equal(np.abs(r["u"]), np.abs(r["end"][0]))


@pytest.mark.parametrize("name", sorted(_CASCADE_GRAPHS))
def test_cascade_start_approximates_the_fiedler_vector(name):
    """On graphs with geometric structure (grids, a random geometric graph, a
    path) the coarse levels carry the Fiedler vector (Sec. 2, Step 3; Theorem
    3.10 in the geometric setting): the prolonged start of every level j < J,
    before any sweep, lies within a small angle of the exact Fiedler space of
    L^j (dense eigensolver).  A random unit vector orthogonal to 1 has a cosine
    of about 1/sqrt(n_j) <= 0.17 with it; a prolongation through a wrong map
    or a discarded coarse result falls to that level."""
    rp, col, w = _CASCADE_GRAPHS[name]()
    h = oracle.Hierarchy(rp, col, w)
    J = h.levels - 1
    r = h.solve(trace=True)
    for j in range(J):
        Q = _fiedler_space(dense_laplacian(*h.csr(j)))
        c = _subspace_cosine(r["start"][j], Q)
        assert c >= 0.85, (j, c)


@pytest.mark.parametrize("name", sorted(set(_CASCADE_GRAPHS) - {"grid_14x9_unit"}))
def test_cascade_cuts_the_level0_sweeps(name):
    """The point of Alg. 1 (Sec. 2, Table 3): level 0 starts close to the
    Fiedler vector, so its power iteration stops after a small fraction of the
    sweeps the same iteration needs from a Gaussian start at the same
    tolerance (graphs of 300 to 4,096 vertices; the 126-vertex grid has too
    few levels for a wide margin)."""
    rp, col, w = _CASCADE_GRAPHS[name]()
    n = len(rp) - 1
    h = oracle.Hierarchy(rp, col, w)
    k_cmg = int(h.solve()["sweeps"][0])
    _, k_gauss, _, capped = oracle.power_iteration(rp, col, w, oracle.gaussian_start(7, n))
    assert not capped
    assert k_cmg <= 0.1 * k_gauss, (k_cmg, k_gauss)


def test_resolve_from_a_given_start_vector():
    """Re-solve on a kept hierarchy from a caller's start vector (the repeated
    computations of the Remark after Alg. 1).  From the exact Fiedler vector
    of a path (closed form) level 0 stops after one sweep on that vector;
    from the coarsest level with Step 2's own Gaussian the result is the
    ordinary solve; from a mid level the levels above are not visited."""
    n = 300
    rp, col, w = inputs.path(n)
    h = oracle.Hierarchy(rp, col, w)
    J = h.levels - 1
    phi = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    phi /= np.linalg.norm(phi)
    r = h.solve(start_level=0, x0=phi)
    assert r["sweeps"][0] == 1 and (r["sweeps"][1:] == 0).all()
    assert np.linalg.norm(align(r["u"], phi) - phi) <= 1e-13
    assert r["lam"] == pytest.approx(2 - 2 * np.cos(np.pi / n), rel=1e-13)
    base = h.solve(seed=5)
    again = h.solve(start_level=J, x0=oracle.gaussian_start(5, h.sizes()[J]))
    assert np.array_equal(base["u"], again["u"])
    assert np.array_equal(base["sweeps"], again["sweeps"])
    mid = h.solve(start_level=1, x0=oracle.gaussian_start(3, h.sizes()[1]), trace=True)
    assert (mid["sweeps"][2:] == 0).all() and mid["sweeps"][1] >= 1
    assert all(v is None for v in mid["start"][2:])
    # a new seed moves the coarsest start, and with it the approximate vector
    other = h.solve(seed=6)
    assert not np.array_equal(base["u"], other["u"])


# ------------------------------------------------------------------ Alg. 4: geometric CMG
def _table4():
    with open(os.path.join(GOLDEN, "table4_gcmg.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    return [(int(r[0]), float(r[1]), float(r[2])) for r in rows]


def _within_print(x, printed):
    """x rounds to `printed` at five significant digits (half a unit in the
    last printed digit, with a little slack for the rounding of the print)."""
    e = np.floor(np.log10(abs(printed)))
    return abs(x - printed) <= 0.51 * 10 ** (e - 4)


def test_gcmg_reproduces_table4():
    """Alg. 4 in the setting of Sec. 4, Table 4 (2D Laplacian, N = 1025,
    beta = 4, k0 = 1, coarsest grid 33 x 33 solved exactly): both printed
    error columns, every level, to the five digits the paper prints."""
    r = oracle.gcmg_grid(2, 1025, 5, beta=4.0, k0=1)
    for lvl, e0, ek in _table4():
        N = (1024 >> lvl) + 1
        lam = 2 - 2 * np.cos(np.pi / N)       # lambda_2 of the N x N grid graph
        assert r["k"][lvl] == 4 ** lvl
        assert _within_print(abs(lam - r["r0"][lvl]), e0), (lvl, abs(lam - r["r0"][lvl]), e0)
        assert _within_print(abs(lam - r["rk"][lvl]), ek), (lvl, abs(lam - r["rk"][lvl]), ek)


def test_gcmg_coarsest_vector_is_an_exact_eigenvector():
    """The coarsest solve of Alg. 4 is exact: residual at rounding level
    against a dense eigensolver's lambda_2 of the 17 x 17 grid graph."""
    N = 17
    r = oracle.gcmg_grid(2, N, 0)
    rp, col, w = inputs.grid2d(N, N, "unit")
    L = dense_laplacian(rp, col, w)
    u = r["u"] / np.linalg.norm(r["u"])
    ev = np.linalg.eigvalsh(L)
    assert r["rk"][0] == pytest.approx(ev[1], rel=1e-13)
    assert np.linalg.norm(L @ u - ev[1] * u) <= 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_gcmg_prolongation_is_exact_on_multilinear_functions(dim):
    """Multilinear interpolation between nested grids reproduces every
    function that is linear in each coordinate: one level of Alg. 4 with no
    smoothing (k0 = 0) keeps such a start's Rayleigh quotient and, after
    Gram-Schmidt against 1, the vector itself.  Checked through a level
    whose start is x (dim 2) or x + 2y - z (dim 3), via the zero-sweep
    result compared with the same function on the fine grid."""
    # a two-level run from an exact coarse eigenvector: the level-0 start is
    # the interpolant of cos along x; compare with interpolating by hand
    N, J = 9, 1
    r = oracle.gcmg_grid(dim, N, J, k0=0)
    Nc = 5
    xc = np.cos(np.pi * (np.arange(Nc) + 0.5) / Nc)
    xf = np.empty(N)
    xf[0::2] = xc
    xf[1::2] = 0.5 * (xc[:-1] + xc[1:])
    f = np.tile(xf, N ** (dim - 1))
    f = f - f.mean()
    f /= np.linalg.norm(f)
    assert np.allclose(r["u"], f, rtol=0, atol=1e-15)
    # linear functions are interpolated exactly: interpolating xf's own
    # coarse samples of a linear function gives the function
    lin = np.arange(N, dtype=float) * 0.3 + 1.0
    assert np.allclose(0.5 * (lin[0:-2:2] + lin[2::2]), lin[1::2])


@pytest.mark.parametrize("dim,N,J", [(2, 129, 4), (3, 33, 3)])
def test_gcmg_smoothing_improves_every_level(dim, N, J):
    """Smoothing (the Richardson steps of Alg. 4) only improves the Rayleigh
    quotient on every level (Lemma 3.7: S = I - omega A contracts the error
    in the energy norm), and every Rayleigh quotient is an upper bound of
    lambda_2 of its level (Courant-Fischer)."""
    r = oracle.gcmg_grid(dim, N, J, beta=4.0, k0=1)
    for j in range(J):
        Nj = (N - 1) // 2 ** j + 1
        lam = 2 - 2 * np.cos(np.pi / Nj)
        assert r["r0"][j] >= lam - 1e-15 and r["rk"][j] >= lam - 1e-15
        assert r["rk"][j] - lam <= r["r0"][j] - lam + 1e-18


# ------------------------------------------------------------------ k eigenpairs (Remark after Alg. 4)
def _conv_pairs(rp, col, w, k, seed=1412):
    h = oracle.Hierarchy(rp, col, w, seed=seed)
    r = oracle.eigenpairs(h, k, converged=True, conv_rtol=1e-14)
    assert (r["res"] <= 1e-14 * oracle.gershgorin(rp, col, w)).all()
    return r


def test_eigenpairs_closed_form_path():
    """Path P_n: lambda_j = 2 - 2 cos(pi (j-1)/n), eigenvectors
    cos(pi (j-1)(x + 1/2)/n), all simple."""
    n, k = 60, 4
    rp, col, w = inputs.path(n)
    r = _conv_pairs(rp, col, w, k)
    x = np.arange(n)
    for i in range(k):
        m = i + 1
        assert r["lam"][i] == pytest.approx(2 - 2 * np.cos(np.pi * m / n), rel=1e-12)
        phi = np.cos(np.pi * m * (x + 0.5) / n)
        phi /= np.linalg.norm(phi)
        assert np.linalg.norm(align(r["U"][i], phi) - phi) <= 1e-9


def test_eigenpairs_grid_with_double_eigenvalues():
    """12 x 12 grid: lambda_2 = lambda_3 (x and y modes) and lambda_5 =
    lambda_6; the first four returned vectors span the eigenspaces of
    lambda_2..lambda_5 -- each cluster's vectors lie in its eigenspace."""
    a = 12
    rp, col, w = inputs.grid2d(a, a, "unit")
    r = _conv_pairs(rp, col, w, 4)
    L = dense_laplacian(rp, col, w)
    ev, V = np.linalg.eigh(L)
    assert np.allclose(r["lam"], ev[1:5], rtol=1e-12, atol=0)
    # lambda_2 = lambda_3 and lambda_4 (= 2 - 2cos(pi/12) + 2 - 2cos(pi/12)) alone
    assert subspace_residual(r["U"][0], V[:, 1:3]) <= 1e-9
    assert subspace_residual(r["U"][1], V[:, 1:3]) <= 1e-9
    assert subspace_residual(r["U"][2], V[:, 3:4]) <= 1e-9


@pytest.mark.parametrize("seed", range(3))
def test_eigenpairs_random_graphs_against_dense_eigensolver(seed):
    n = [80, 140, 200][seed]
    k = 3
    rp, col, w = inputs.random_connected(n, 2 * n, seed=300 + seed)
    ev, V = np.linalg.eigh(dense_laplacian(rp, col, w))
    r = _conv_pairs(rp, col, w, k, seed=seed)
    assert np.allclose(r["lam"], ev[1:k + 1], rtol=1e-12, atol=0)
    for i in range(k):
        gap = min(abs(ev[i + 1] - ev[i]), abs(ev[i + 2] - ev[i + 1]))
        if gap > 1e-3 * ev[i + 1]:
            assert np.linalg.norm(align(r["U"][i], V[:, i + 1]) - V[:, i + 1]) <= 1e-8


def test_eigenpairs_default_mode_invariants():
    """Default mode: orthonormal vectors orthogonal to 1 (Gram-Schmidt after
    every sweep), canonical signs, and Courant-Fischer: the Rayleigh
    quotients of an orthonormal k-frame bound the eigenvalues from above
    (the i-th largest quotient >= lambda_{i+1}, by the min-max principle
    applied to the frame's span)."""
    rp, col, w = inputs.rgg(1200, 8.0, seed=7)
    h = oracle.Hierarchy(rp, col, w)
    r = oracle.eigenpairs(h, 4)
    U = r["U"]
    assert np.allclose(U @ U.T, np.eye(4), atol=1e-13)
    assert np.abs(U.sum(axis=1)).max() <= 1e-12
    for u in U:
        assert u[np.argmax(np.abs(u))] > 0
    ev = np.linalg.eigvalsh(dense_laplacian(rp, col, w))
    assert (np.sort(r["lam"]) >= ev[1:5] - 1e-12).all()


def test_one_eigenpair_is_the_fiedler_solve():
    """With k = 1 the block cascade performs exactly the operations of the
    single-vector cascade (same start, projection, stop rule)."""
    rp, col, w = inputs.grid2d(40, 30, "uniform", seed=5)
    h = oracle.Hierarchy(rp, col, w, seed=9)
    a = h.solve()
    b = oracle.eigenpairs(h, 1)
    assert np.array_equal(a["sweeps"], b["sweeps"])
    assert np.array_equal(a["u"], b["U"][0]) and a["lam"] == b["lam"][0]
