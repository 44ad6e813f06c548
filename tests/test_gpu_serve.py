"""Serving loop: results do not depend on the mix a request ran in.

Requests for graphs of different sizes go through a server with several
workers and batching (small graphs share batched jobs, large ones run alone
with resident hierarchies); every result must equal the result of the same
request run alone (one worker, no batching) within the FP64 parity
tolerances, and match the oracle.  Also: warm solves on resident
hierarchies, admission under a small memory budget, and a request that can
never fit.
"""
import threading

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


def graphs():
    return [
        inputs.rgg(1500, 8.0, seed=41),
        inputs.grid2d(40, 45, "uniform", seed=42),
        inputs.barabasi_albert(3000, 4, seed=43),
        inputs.random_connected(9000, 27000, seed=44),    # above batch_max_n: alone
        inputs.rgg(12000, 8.0, seed=45),                  # above batch_max_n: alone
        inputs.path(30),
        inputs.cycle(400),
        inputs.grid2d(20, 20, "uniform", seed=46),
        inputs.barabasi_albert(800, 4, seed=47),
        inputs.complete(50),
    ]


def run_all(server, gids, concurrent):
    out = {}
    if concurrent:
        tickets = [(g, server.submit(g)) for g in gids]
        for g, t in tickets:
            out[g] = server.wait(t, timeout_s=300)
    else:
        for g in gids:
            out[g] = server.wait(server.submit(g), timeout_s=300)
    return out


def test_same_result_alone_and_in_the_mix():
    gs = graphs()
    with cmg.Server(workers=3, max_batch=64, batch_max_n=5000, min_batch=2, seed=1412) as mix:
        ids = [mix.add_graph(*g) for g in gs]
        res_mix = run_all(mix, ids, concurrent=True)
        st = mix.stats()
        assert st["completed"] == len(gs)
        assert st["batch_jobs"] >= 1 and st["single_jobs"] >= 2
        assert st["peak_bytes"] <= st["budget_bytes"]
    assert any(r[1]["batch_size"] > 1 for r in res_mix.values())
    with cmg.Server(workers=1, max_batch=1, seed=1412) as alone:
        ids2 = [alone.add_graph(*g) for g in gs]
        res_alone = run_all(alone, ids2, concurrent=False)
    for k, g in enumerate(gs):
        u1, r1 = res_mix[ids[k]]
        u2, r2 = res_alone[ids2[k]]
        assert r1["status"] == "OK" and r2["status"] == "OK"
        assert r2["batch_size"] == 1
        assert aligned_err(u1, u2) <= VEC_TOL, k
        assert abs(r1["lambda2"] - r2["lambda2"]) <= LAM_TOL * abs(r2["lambda2"]), k
        ref_u, ref_lam, _, _, _ = oracle.fiedler(*g, seed=1412)
        assert aligned_err(u1, ref_u) <= VEC_TOL, k
        assert abs(r1["lambda2"] - ref_lam) <= LAM_TOL * abs(ref_lam), k


def test_requests_from_several_threads_and_warm_solves():
    gs = graphs()[3:5]
    with cmg.Server(workers=2, batch_max_n=5000, seed=1412) as srv:
        ids = [srv.add_graph(*g) for g in gs]
        cold = {g: srv.wait(srv.submit(g)) for g in ids}
        results = {}

        def client(g):
            results[g] = [srv.wait(srv.submit(g)) for _ in range(3)]

        th = [threading.Thread(target=client, args=(g,)) for g in ids]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for g in ids:
            assert not cold[g][1]["warm"]
            for u, r in results[g]:
                assert r["warm"]
                assert np.array_equal(u, cold[g][0]) and r["lambda2"] == cold[g][1]["lambda2"]
        assert srv.stats()["warm_jobs"] == 6 and srv.stats()["resident"] == 2


def test_admission_under_a_small_memory_budget():
    import gc
    gc.collect()                 # hierarchies of earlier tests leave the pool
    torch.cuda.synchronize()
    gs = graphs()
    est = [cmg.estimate_device_bytes(len(g[0]) - 1, int(g[0][-1])) for g in gs]
    budget = max(est) + 1
    with cmg.Server(workers=4, max_batch=64, batch_max_n=5000, min_batch=2, mem_budget=budget,
                    seed=1412) as srv:
        ids = [srv.add_graph(*g) for g in gs]
        res = run_all(srv, ids, concurrent=True)
        st = srv.stats()
        assert st["peak_bytes"] <= budget
        # what the device actually held from the library's pool, measured
        assert 0 < st["measured_peak_bytes"] <= budget
        assert st["evictions"] >= 1          # resident hierarchies made room
    for k, g in enumerate(gs):
        ref_u, ref_lam, _, _, _ = oracle.fiedler(*g, seed=1412)
        assert aligned_err(res[ids[k]][0], ref_u) <= VEC_TOL


def test_request_that_can_never_fit_fails_cleanly():
    g = inputs.grid2d(60, 60, "uniform", seed=48)
    with cmg.Server(workers=2, mem_budget=1024, seed=1412) as srv:
        gid = srv.add_graph(*g)
        with pytest.raises(cmg.CmgError) as e:
            srv.wait(srv.submit(gid))
        assert e.value.name == "ERR_TOO_LARGE"


def test_repeated_graphs_under_poisson_arrivals_all_complete():
    """A request trace that repeats graphs, arriving over time: every request
    completes once (no request lost or run twice), results equal the alone
    results; waits are bounded so a lost request fails instead of hanging."""
    import time
    gs = graphs()
    rng = np.random.default_rng(5)
    trace = rng.integers(0, len(gs), size=40)
    alone = {}
    with cmg.Server(workers=1, max_batch=1, seed=1412) as srv:
        ids = [srv.add_graph(*g) for g in gs]
        for k in sorted(set(trace.tolist())):
            alone[k] = srv.wait(srv.submit(ids[k]), timeout_s=120)
    with cmg.Server(workers=4, max_batch=64, batch_max_n=5000, min_batch=2, seed=1412) as srv:
        ids = [srv.add_graph(*g) for g in gs]
        arr = np.cumsum(rng.exponential(0.004, size=len(trace)))
        t0 = time.perf_counter()
        tickets = []
        for k, ta in zip(trace, arr):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append((k, srv.submit(ids[k])))
        for k, t in tickets:
            u, r = srv.wait(t, timeout_s=120)
            assert r["status"] == "OK"
            assert aligned_err(u, alone[k][0]) <= VEC_TOL, k
            assert abs(r["lambda2"] - alone[k][1]["lambda2"]) <= LAM_TOL * abs(alone[k][1]["lambda2"])
        st = srv.stats()
        assert st["completed"] == len(trace)
        assert st["single_jobs"] + st["warm_jobs"] + st["batch_jobs"] <= len(trace)
