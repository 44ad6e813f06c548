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
