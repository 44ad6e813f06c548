"""The two-phase sweep kernel (k_power_2p) against the CPU oracle.

The kernel is forced on every level with a sweep layout (CMG_2P=1), with
small source blocks and pass buffers so that small graphs still take many
source blocks, many passes and several dest blocks per CTA.  FP64: identical
per-level sweep counts, vector within 1e-10, lambda2 within 1e-12 (the same
bar as the slice kernel).  FP32 sweep form: lambda2 within 1e-6 and angle
within 1e-4 rad of the oracle replayed with the same sweep counts.  Repeated
solves are bit-identical (rows sum in 64-bit fixed point: integer adds
commute, so the order of the shared-memory atomics does not matter)."""
import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KIND_TWO_PHASE = 4

CASES = {
    "chung_lu": lambda: inputs.chung_lu(30000, seed=7),
    "random": lambda: inputs.random_connected(20000, 90000, seed=3),
    "grid_ragged": lambda: inputs.grid2d(145, 171, "uniform", seed=2),
    "ba": lambda: inputs.barabasi_albert(20000, 4, seed=6),
    # one row of 12,000 entries, summed by all 31 row warps of its CTA
    "hub": lambda: inputs.hub_grid(120, 110, 12000, seed=5),
}

# knobs: (source block vertices, bytes per pass buffer)
KNOBS = {
    "blocks": (1024, 1 << 20),
    "passes": (4096, 96 << 10),
    "both": (300, 48 << 10),
}


def aligned_err(u, ref):
    if np.dot(u, ref) < 0:
        u = -u
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def angle(u, ref):
    c = abs(np.dot(u, ref)) / (np.linalg.norm(u) * np.linalg.norm(ref))
    return float(np.arccos(min(1.0, c)))


def two_phase(monkeypatch, knobs):
    sb, xcap = KNOBS[knobs]
    monkeypatch.setenv("CMG_2P", "1")
    monkeypatch.setenv("CMG_2P_SB", str(sb))
    monkeypatch.setenv("CMG_2P_XCAP", str(xcap))


@pytest.mark.parametrize("knobs", sorted(KNOBS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_two_phase_fp64_matches_oracle(monkeypatch, name, knobs):
    rp, col, w = CASES[name]()
    two_phase(monkeypatch, knobs)
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    kind, _ = h.level_kernels()
    assert KIND_TWO_PHASE in kind
    assert all(k in (0, KIND_TWO_PHASE, 5) for k in kind)   # 5: cluster kernel on small FP64 levels
    u, lam, st = h.fiedler()
    u2, lam2, _ = h.fiedler()
    h.close()
    assert np.array_equal(u, u2) and lam == lam2
    ref_u, ref_lam, _, oh, ref = oracle.fiedler(rp, col, w, seed=1412)
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref_u) <= 1e-10
    assert abs(lam - ref_lam) <= 1e-12 * abs(ref_lam)


@pytest.mark.parametrize("name", sorted(CASES))
def test_two_phase_fp32_form_accuracy(monkeypatch, name):
    rp, col, w = CASES[name]()
    two_phase(monkeypatch, "both")
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    ref = oh.solve()
    h = cmg.Hierarchy(rp, col, w, seed=1412, precision="fp32", schedule="replay",
                      replay_sweeps=ref["sweeps"].tolist())
    kind, _ = h.level_kernels()
    assert KIND_TWO_PHASE in kind
    u, lam, st = h.fiedler()
    u2, lam2, _ = h.fiedler()
    h.close()
    assert np.array_equal(u, u2) and lam == lam2
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert abs(lam - ref["lam"]) <= 1e-6 * abs(ref["lam"])
    assert angle(u, ref["u"]) <= 1e-4


def test_two_phase_default_knobs_on_a_power_law_graph(monkeypatch):
    """The default layout (192 KB source blocks, 32 MB pass buffers) on a
    Chung-Lu graph whose level 0 takes several passes and source blocks."""
    monkeypatch.setenv("CMG_2P", "1")
    monkeypatch.delenv("CMG_2P_SB", raising=False)
    monkeypatch.delenv("CMG_2P_XCAP", raising=False)
    rp, col, w = inputs.chung_lu(600000, seed=12)
    h = cmg.Hierarchy(rp, col, w, seed=1412)
    kind, _ = h.level_kernels()
    assert kind[0] == KIND_TWO_PHASE
    u, lam, st = h.fiedler()
    h.close()
    ref_u, ref_lam, _, oh, ref = oracle.fiedler(rp, col, w, seed=1412)
    assert st["sweeps"] == ref["sweeps"].tolist()
    assert aligned_err(u, ref_u) <= 1e-10
    assert abs(lam - ref_lam) <= 1e-12 * abs(ref_lam)


def test_two_phase_only_on_request(monkeypatch):
    monkeypatch.delenv("CMG_2P", raising=False)
    h = cmg.Hierarchy(*inputs.chung_lu(600000, seed=12), seed=1412)
    kind, _ = h.level_kernels()
    h.close()
    assert KIND_TWO_PHASE not in kind
