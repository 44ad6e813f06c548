"""Input validation and error paths of cmg_setup / cmg_fiedler on the GPU.

Failures are made on the host side (malformed inputs, an injected allocation
failure); nothing here faults the device."""
import numpy as np
import pytest

from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def setup_status(rp, col, w, **kw):
    try:
        h = cmg.Hierarchy(rp, col, w, **kw)
        h.close()
        return "OK"
    except cmg.CmgError as e:
        return e.name


def base():
    rp, col, w = inputs.grid2d(6, 5, "uniform", seed=1)
    return rp.copy(), col.copy(), w.copy()


def test_valid_input_accepted():
    assert setup_status(*base()) == "OK"


def test_asymmetric_weight_rejected():
    rp, col, w = base()
    w[3] *= 1.0 + 2 ** -40
    assert setup_status(rp, col, w) == "ERR_NOT_SYMMETRIC"


def test_missing_mirror_rejected():
    rp, col, w = inputs.csr_from_edges(3, [0, 1], [1, 2], [1.0, 1.0])
    # drop entry (2, 1): row 2 becomes empty as well
    rp2 = rp.copy()
    rp2[3] = rp[3] - 1
    assert setup_status(rp2, col[:-1].copy(), w[:-1].copy()) in ("ERR_NOT_SYMMETRIC",
                                                                 "ERR_ISOLATED_VERTEX")


def test_self_loop_rejected():
    rp, col, w = inputs.csr_from_edges(3, [0, 1], [1, 2], [1.0, 1.0])
    rp2 = np.array([0, 2, 4, 5], dtype=np.int64)
    col2 = np.array([0, 1, 0, 2, 1], dtype=np.int32)
    w2 = np.ones(5)
    assert setup_status(rp2, col2, w2) == "ERR_SELF_LOOP"


@pytest.mark.parametrize("bad", [0.0, -1.0, np.nan, np.inf])
def test_bad_weight_rejected(bad):
    rp, col, w = base()
    w[:] = 1.0
    w[0] = bad
    st = setup_status(rp, col, w)
    assert st in ("ERR_BAD_WEIGHT",)


def test_unsorted_or_out_of_range_columns_rejected():
    rp, col, w = base()
    c2 = col.copy()
    c2[rp[7]], c2[rp[7] + 1] = c2[rp[7] + 1], c2[rp[7]]
    assert setup_status(rp, c2, w) == "ERR_BAD_CSR"
    c3 = col.copy()
    c3[0] = 10**6
    assert setup_status(rp, c3, w) == "ERR_BAD_CSR"
    rp4 = rp.copy()
    rp4[5] = rp4[6] + 1
    assert setup_status(rp4, col, w) == "ERR_BAD_CSR"


def test_isolated_vertex_rejected():
    rp, col, w = inputs.csr_from_edges(4, [0, 1], [1, 2], [1.0, 1.0])
    assert setup_status(rp, col, w) == "ERR_ISOLATED_VERTEX"


def test_too_small():
    assert setup_status(np.array([0, 0], dtype=np.int64), np.zeros(0, np.int32),
                        np.zeros(0)) == "ERR_TOO_SMALL"


def test_injected_allocation_failures_are_reported_and_recoverable():
    rp, col, w = inputs.grid2d(40, 30, "uniform", seed=2)
    ok_u, ok_lam, _ = cmg.fiedler(rp, col, w)
    seen = set()
    for k in range(0, 60, 3):
        cmg.debug_fail_alloc_after(k)
        try:
            h = cmg.Hierarchy(rp, col, w)
            try:
                u, lam, _ = h.fiedler()
                assert lam == ok_lam
            finally:
                h.close()
            seen.add("OK")
        except cmg.CmgError as e:
            assert e.name == "ERR_OOM"
            seen.add("OOM")
        finally:
            cmg.debug_fail_alloc_after(-1)
    assert "OOM" in seen
    u, lam, _ = cmg.fiedler(rp, col, w)
    assert np.array_equal(u, ok_u) and lam == ok_lam


# ------------------------------------------------------------------ device-side waits that run out
# The stall hook makes one grid barrier of one launch never release, so every
# CTA's bounded wait there runs out (20 ms), the kernel returns, and the call
# must report ERR_DEVICE_TIMEOUT even though later launches of the same call
# (the next levels, the final pass) run after it.  No fault is involved: the
# waits are the library's own bounded spins, and the context stays usable.
def _stalled(fn, launch=0, barrier=1):
    cmg.debug_stall_barrier(launch, barrier)
    try:
        fn()
    except cmg.CmgError as e:
        return e.name
    finally:
        cmg.debug_stall_barrier(-1, 0)
    return "OK"


def test_timeout_in_a_non_final_launch_reaches_cmg_fiedler():
    rp, col, w = inputs.grid2d(200, 200, "uniform", seed=4)
    with cmg.Hierarchy(rp, col, w) as h:
        kinds, _ = h.level_kernels()
        assert kinds[0] in (1, 2)            # level 0 runs the multi-CTA slice kernel
        ok_u, ok_lam, _ = h.fiedler()
        # the first multi-CTA launch of the solve is a power-iteration launch;
        # the final-vector launch (and maybe more levels) follow it
        assert _stalled(h.fiedler) == "ERR_DEVICE_TIMEOUT"
        u, lam, _ = h.fiedler()
        assert np.array_equal(u, ok_u) and lam == ok_lam


def test_timeout_in_setup_is_reported():
    rp, col, w = inputs.grid2d(200, 200, "uniform", seed=4)
    ok_u, ok_lam, _ = cmg.fiedler(rp, col, w)
    # the coarsening kernel of level 0 is the first multi-CTA launch of setup
    assert _stalled(lambda: cmg.Hierarchy(rp, col, w).close(), barrier=0) == "ERR_DEVICE_TIMEOUT"
    u, lam, _ = cmg.fiedler(rp, col, w)
    assert np.array_equal(u, ok_u) and lam == ok_lam


@pytest.mark.parametrize("entry", ["power_sweeps", "power_sweeps_noalloc"])
def test_timeout_in_the_sweep_launch_reaches_the_step_entry_points(entry):
    rp, col, w = inputs.grid2d(200, 200, "uniform", seed=4)
    dev = torch.device("cuda")
    rp32 = torch.tensor(rp.astype(np.int32), device=dev)
    c = torch.tensor(col, device=dev)
    wt = torch.tensor(w, device=dev)
    x = torch.tensor(np.random.default_rng(3).standard_normal(len(rp) - 1), device=dev)
    fn = getattr(cmg, entry)
    u0, cos0 = fn(rp32, c, wt, x, 40)
    # the sweep launch is followed by the final-vector launch in the same call
    assert _stalled(lambda: fn(rp32, c, wt, x, 40)) == "ERR_DEVICE_TIMEOUT"
    u1, cos1 = fn(rp32, c, wt, x, 40)
    assert torch.equal(u0, u1) and cos0 == cos1


def test_stall_hook_rejects_a_bad_barrier_index():
    with pytest.raises(cmg.CmgError):
        cmg.debug_stall_barrier(0, 255)
    cmg.debug_stall_barrier(-1, 0)
