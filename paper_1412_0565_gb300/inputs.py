"""Seeded synthetic graph generators.

This module holds no arithmetic of the CMG method; it only builds inputs.  Both
the CUDA path (tests, bench) and the CPU oracle consume the graphs it makes.
Every graph is returned as a symmetric CSR triple ``(row_ptr int64[n+1],
col int32[nnz], w float64[nnz])`` with ascending columns, no self-loops, no
duplicate entries and strictly positive weights -- the input contract of
``cmg_setup``.

The paper measures on graphs of the University of Florida sparse matrix
collection (Sec. 4, Table 2), which are not available here; the families below
stand in for them: structured grids (the Table 3 / Sec. 3 model problem),
Chung-Lu power-law graphs, random geometric graphs and Barabasi-Albert graphs.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "csr_from_edges", "grid2d", "grid3d", "path", "cycle", "complete", "star",
    "random_connected", "chung_lu", "rgg", "barabasi_albert", "largest_component",
    "batch_graphs", "batch_graph", "concat_csr", "serving_sizes", "serving_graphs", "hub_grid",
]


def _unique_sorted(k):
    """Sorted unique values of an int64 array (sort + mask; same result as
    np.unique, much faster on large arrays)."""
    k = np.sort(np.asarray(k, dtype=np.int64))
    if k.size == 0:
        return k
    keep = np.empty(k.size, dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def csr_from_edges(n: int, u, v, w):
    """Symmetric CSR from an undirected edge list (u != v, no duplicate pairs);
    rows and columns ascending.  Each edge {a < b} gives entry (a, b) of row a
    (after the row's smaller columns) and entry (b, a) of row b (before its
    larger columns), so two sorts of the edge list (by (a, b) and by (b, a))
    place every entry."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    if u.size and (np.any(u == v) or u.min() < 0 or v.min() < 0 or max(u.max(), v.max()) >= n):
        raise ValueError("bad edge list")
    a, b = np.minimum(u, v), np.maximum(u, v)
    m = a.size
    ou = np.argsort(a * n + b)          # keys are unique: any sort gives this order
    ol = np.argsort(b * n + a)
    ru, cu, wu = a[ou], b[ou], w[ou]    # upper entries: row a, column b > a
    rl, cl, wl = b[ol], a[ol], w[ol]    # lower entries: row b, column a < b
    cnt_u = np.bincount(ru, minlength=n)
    cnt_l = np.bincount(rl, minlength=n)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_u + cnt_l, out=rp[1:])
    off_u = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_u, out=off_u[1:])
    off_l = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_l, out=off_l[1:])
    idx = np.arange(m, dtype=np.int64)
    pos_l = rp[rl] + (idx - off_l[rl])
    pos_u = rp[ru] + cnt_l[ru] + (idx - off_u[ru])
    cols = np.empty(2 * m, dtype=np.int32)
    ww = np.empty(2 * m, dtype=np.float64)
    cols[pos_l] = cl
    ww[pos_l] = wl
    cols[pos_u] = cu
    ww[pos_u] = wu
    return rp, cols, ww


def _weights(m: int, weights, rng, lo=0.5, hi=1.5):
    if weights == "unit":
        return np.ones(m, dtype=np.float64)
    if weights == "uniform":
        return rng.uniform(lo, hi, size=m)
    if weights == "lognormal":
        return rng.lognormal(0.0, 1.0, size=m)
    raise ValueError(weights)


def grid2d(a: int, b: int, weights="unit", seed=1412):
    """a x b 5-point grid.  Vertex (x, y) has id y*a + x.  Edge weights are
    drawn in the order: all x-edges by id, then all y-edges by id."""
    rng = np.random.default_rng(seed)
    ids = np.arange(a * b, dtype=np.int64).reshape(b, a)
    ex = (ids[:, :-1].ravel(), ids[:, 1:].ravel())
    ey = (ids[:-1, :].ravel(), ids[1:, :].ravel())
    u = np.concatenate([ex[0], ey[0]])
    v = np.concatenate([ex[1], ey[1]])
    return csr_from_edges(a * b, u, v, _weights(u.size, weights, rng))


def grid3d(a: int, b: int, c: int, weights="uniform", seed=1412):
    """a x b x c 7-point grid.  Vertex (x, y, z) has id (z*b + y)*a + x.  Edge
    weights are drawn in the order: x-edges by id, y-edges by id, z-edges by id."""
    rng = np.random.default_rng(seed)
    ids = np.arange(a * b * c, dtype=np.int64).reshape(c, b, a)
    ex = (ids[:, :, :-1].ravel(), ids[:, :, 1:].ravel())
    ey = (ids[:, :-1, :].ravel(), ids[:, 1:, :].ravel())
    ez = (ids[:-1, :, :].ravel(), ids[1:, :, :].ravel())
    u = np.concatenate([ex[0], ey[0], ez[0]])
    v = np.concatenate([ex[1], ey[1], ez[1]])
    return csr_from_edges(a * b * c, u, v, _weights(u.size, weights, rng))


def hub_grid(a: int, b: int, hub_degree: int, seed=1412, hub_scale=1.0):
    """An a x b 5-point grid (U[0.5, 1.5] weights) plus one extra vertex, id
    a*b, joined to `hub_degree` distinct grid vertices drawn uniformly, with
    weights hub_scale * U[0.5, 1.5]: the hub row of a power-law graph in a
    graph small enough for exhaustive checks."""
    rng = np.random.default_rng(seed)
    rp, col, w = grid2d(a, b, "uniform", seed=seed + 1)
    n = a * b
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    keep = src < col
    tgt = rng.choice(n, size=hub_degree, replace=False)
    u = np.concatenate([src[keep], np.full(hub_degree, n, dtype=np.int64)])
    v = np.concatenate([col[keep].astype(np.int64), tgt])
    ww = np.concatenate([w[keep], hub_scale * rng.uniform(0.5, 1.5, size=hub_degree)])
    return csr_from_edges(n + 1, u, v, ww)


def path(n: int, w=None):
    """Path P_n; w (length n-1) gives the edge weights, default 1."""
    u = np.arange(n - 1)
    ww = np.ones(n - 1) if w is None else np.asarray(w, dtype=np.float64)
    return csr_from_edges(n, u, u + 1, ww)


def cycle(n: int, w=None):
    u = np.arange(n)
    v = (u + 1) % n
    ww = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    return csr_from_edges(n, np.minimum(u, v), np.maximum(u, v), ww)


def complete(n: int):
    iu = np.triu_indices(n, 1)
    return csr_from_edges(n, iu[0], iu[1], np.ones(iu[0].size))


def star(n: int):
    """Star with centre 0 and n-1 leaves."""
    return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), np.ones(n - 1))


def random_connected(n: int, extra: int, seed: int, weights="uniform", ties=False):
    """A random spanning tree plus `extra` random chords (duplicates merged).
    ties=True draws weights from {1, 2, 3} so that many heaviest-edge ties occur."""
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    u = np.concatenate([parent, rng.integers(0, n, size=extra)])
    v = np.concatenate([np.arange(1, n), rng.integers(0, n, size=extra)])
    keep = u != v
    a, b = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = _unique_sorted(a * n + b)
    a, b = key // n, key % n
    if ties:
        ww = rng.integers(1, 4, size=a.size).astype(np.float64)
    else:
        ww = _weights(a.size, weights, rng)
    return csr_from_edges(n, a, b, ww)


def largest_component(n: int, u, v):
    """Vertices of the largest connected component of an undirected edge list
    (lowest-id component on ties), as a boolean mask."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    A = sp.coo_matrix((np.ones(len(u), dtype=np.int8), (u, v)), shape=(n, n)).tocsr()
    ncomp, lab = connected_components(A, directed=False)
    sizes = np.bincount(lab, minlength=ncomp)
    return lab == int(np.argmax(sizes))


def _relabel_keep(n, u, v, w, mask):
    keep_e = mask[u] & mask[v]
    newid = np.cumsum(mask) - 1
    return int(mask.sum()), newid[u[keep_e]], newid[v[keep_e]], w[keep_e]


def chung_lu(n: int = 4_194_304, mean_deg: float = 16.0, gamma: float = 2.5, seed: int = 1412,
             weights="lognormal"):
    """Chung-Lu power-law graph.  Expected degrees w_i proportional to
    (i + 1)^(-1/(gamma-1)), scaled to mean `mean_deg` and capped at sqrt(n*mean_deg);
    m = n*mean_deg/2 endpoint pairs drawn independently with probability
    proportional to w; self-loops dropped, duplicates merged (one weight), the
    largest connected component kept and relabelled in id order.  Weights are
    lognormal(0, 1) per undirected edge (drawn after merging)."""
    rng = np.random.default_rng(seed)
    wt = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    wt *= mean_deg * n / wt.sum()
    np.minimum(wt, np.sqrt(n * mean_deg), out=wt)
    p = wt / wt.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    m = int(n * mean_deg / 2)
    # endpoints by inverse-CDF lookup of sorted uniforms (a fast merge-like
    # search); the second endpoints are then put in random order so that the
    # two endpoints of a pair are independent
    u = np.searchsorted(cdf, np.sort(rng.random(m)), side="right").astype(np.int64)
    v = np.searchsorted(cdf, np.sort(rng.random(m)), side="right").astype(np.int64)
    v = v[rng.permutation(m)]
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    keep = u != v
    a, b = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = _unique_sorted(a * n + b)
    a, b = key // n, key % n
    ww = _weights(a.size, weights, rng)
    mask = largest_component(n, a, b)
    n2, a, b, ww = _relabel_keep(n, a, b, ww, mask)
    return csr_from_edges(n2, a, b, ww)


def rgg(n: int, mean_deg: float = 8.0, seed: int = 1412, weights="uniform"):
    """Random geometric graph: n points uniform in the unit square, an edge for
    each pair closer than r = sqrt(mean_deg / (pi n)); the largest component is
    kept.  Weights U[0.5, 1.5] per edge."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = np.sqrt(mean_deg / (np.pi * n))
    ncell = max(1, int(1.0 / r))
    cell = np.minimum((pts * ncell).astype(np.int64), ncell - 1)
    cid = cell[:, 1] * ncell + cell[:, 0]
    order = np.argsort(cid, kind="stable")
    cstart = np.searchsorted(cid[order], np.arange(ncell * ncell + 1))
    us, vs = [], []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ncx = cell[:, 0] + dx
            ncy = cell[:, 1] + dy
            ok = (ncx >= 0) & (ncx < ncell) & (ncy >= 0) & (ncy < ncell)
            src = np.nonzero(ok)[0]
            nc = ncy[src] * ncell + ncx[src]
            cnt = cstart[nc + 1] - cstart[nc]
            rep_src = np.repeat(src, cnt)
            offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
            dst = order[np.repeat(cstart[nc], cnt) + offs]
            sel = rep_src < dst
            a, b = rep_src[sel], dst[sel]
            d2 = ((pts[a] - pts[b]) ** 2).sum(axis=1)
            close = d2 < r * r
            us.append(a[close])
            vs.append(b[close])
    a = np.concatenate(us)
    b = np.concatenate(vs)
    key = _unique_sorted(a * n + b)
    a, b = key // n, key % n
    ww = _weights(a.size, weights, rng)
    mask = largest_component(n, a, b)
    n2, a, b, ww = _relabel_keep(n, a, b, ww, mask)
    return csr_from_edges(n2, a, b, ww)


def barabasi_albert(n: int, m: int = 4, seed: int = 1412, weights="uniform"):
    """Barabasi-Albert preferential attachment from an (m+1)-clique: vertex t
    adds m edges whose far endpoints are copies of uniformly chosen earlier
    edge endpoints (probability proportional to degree).  Repeated targets of
    one vertex are merged into one edge."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    iu = np.triu_indices(m0, 1)
    e0 = iu[0].size
    ne = e0 + (n - m0) * m
    val = np.full(2 * ne, -1, dtype=np.int64)
    val[0:2 * e0:2] = iu[0]
    val[1:2 * e0:2] = iu[1]
    ptr = np.arange(2 * ne, dtype=np.int64)
    t = np.repeat(np.arange(m0, n, dtype=np.int64), m)
    e = e0 + np.arange((n - m0) * m, dtype=np.int64)
    val[2 * e] = t
    avail = 2 * (e0 + (t - m0) * m)          # endpoints of edges made before vertex t
    ptr[2 * e + 1] = np.floor(rng.random(e.size) * avail).astype(np.int64)
    unresolved = val < 0
    for _ in range(64):
        if not unresolved.any():
            break
        ptr[unresolved] = ptr[ptr[unresolved]]
        nv = val[ptr[unresolved]]
        idx = np.nonzero(unresolved)[0]
        val[idx] = nv
        unresolved = val < 0
    u = val[0::2]
    v = val[1::2]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = _unique_sorted(a * n + b)
    a, b = key // n, key % n
    return csr_from_edges(n, a, b, _weights(a.size, weights, rng))


def concat_csr(graphs):
    """Block-diagonal union of CSR graphs; returns (row_ptr, col, w, vertex_offsets)."""
    offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, (rp, _, _) in enumerate(graphs):
        offs[i + 1] = offs[i] + len(rp) - 1
    nnz_offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, (rp, _, _) in enumerate(graphs):
        nnz_offs[i + 1] = nnz_offs[i] + rp[-1]
    rp_all = np.empty(offs[-1] + 1, dtype=np.int64)
    col_all = np.empty(nnz_offs[-1], dtype=np.int32)
    w_all = np.empty(nnz_offs[-1], dtype=np.float64)
    for i, (rp, col, w) in enumerate(graphs):
        rp_all[offs[i]:offs[i + 1]] = rp[:-1] + nnz_offs[i]
        col_all[nnz_offs[i]:nnz_offs[i + 1]] = col + offs[i]
        w_all[nnz_offs[i]:nnz_offs[i + 1]] = w
    rp_all[-1] = nnz_offs[-1]
    return rp_all, col_all, w_all, offs


def _family_graph(i: int, nv: int, seed: int):
    """Graph i of a mixed batch: families round-robin (random geometric graph
    with mean degree 8, near-square 2D grid, Barabasi-Albert m=4), weights
    U[0.5, 1.5], seeded by (seed, i)."""
    fam = i % 3
    s = int(seed * 100003 + i)
    if fam == 0:
        return rgg(int(nv), 8.0, seed=s)
    if fam == 1:
        a = int(np.floor(np.sqrt(nv)))
        return grid2d(a, int(np.ceil(nv / a)), weights="uniform", seed=s)
    return barabasi_albert(int(nv), 4, seed=s)


def _family_chunk(args):
    seed, items = args
    return [_family_graph(i, nv, seed) for i, nv in items]


def batch_sizes(count: int = 4096, lo: int = 500, hi: int = 20000, seed: int = 1412):
    """Vertex counts of a mixed batch: log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)


def batch_graph(i: int, count: int = 4096, lo: int = 500, hi: int = 20000, seed: int = 1412):
    """Graph i of batch_graphs(count, lo, hi, seed), built alone."""
    return _family_graph(i, int(batch_sizes(count, lo, hi, seed)[i]), seed)


def batch_graphs(count: int = 4096, lo: int = 500, hi: int = 20000, seed: int = 1412,
                 workers: int = 0):
    """Mixed batch: sizes log-uniform in [lo, hi]; families round-robin
    (random geometric graph with mean degree 8, near-square 2D grid, Barabasi-Albert
    m=4); weights U[0.5, 1.5].  Returns a list of CSR triples.  workers > 1
    generates in that many spawned processes (same graphs)."""
    sizes = batch_sizes(count, lo, hi, seed)
    items = [(i, int(nv)) for i, nv in enumerate(sizes)]
    if workers <= 1:
        return _family_chunk((seed, items))
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunks = [items[k::workers] for k in range(workers)]
    out = [None] * count
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for chunk, res in zip(chunks, ex.map(_family_chunk, [(seed, c) for c in chunks])):
            for (i, _), g in zip(chunk, res):
                out[i] = g
    return out


def serving_sizes(count: int, lo: float = 1e3, hi: float = 2e6, seed: int = 1412):
    """Request sizes: log n ~ Normal truncated to [ln lo, ln hi], mean at the
    midpoint, standard deviation (ln hi - ln lo) / 6."""
    rng = np.random.default_rng(seed)
    a, b = np.log(lo), np.log(hi)
    mu, sd = 0.5 * (a + b), (b - a) / 6.0
    out = []
    while len(out) < count:
        x = rng.normal(mu, sd, size=count)
        out.extend(x[(x >= a) & (x <= b)].tolist())
    return np.exp(np.array(out[:count])).astype(np.int64)


def serving_graphs(count: int, lo: float = 1e3, hi: float = 2e6, seed: int = 1412,
                   workers: int = 0):
    """Graphs of a serving workload: sizes from serving_sizes, families and
    weights as in batch_graphs (graph i is family i mod 3)."""
    sizes = serving_sizes(count, lo, hi, seed)
    items = [(i, int(nv)) for i, nv in enumerate(sizes)]
    if workers <= 1:
        return _family_chunk((seed + 7, items))
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    # largest first, so the pool's chunks are balanced
    order = sorted(items, key=lambda t: -t[1])
    chunks = [order[k::workers] for k in range(workers)]
    out = [None] * count
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        for chunk, res in zip(chunks, ex.map(_family_chunk, [(seed + 7, c) for c in chunks])):
            for (i, _), g in zip(chunk, res):
                out[i] = g
    return out
