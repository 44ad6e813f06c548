"""k eigenpairs by the cascade (cmg_eigenpairs; the Remark after Alg. 4)
against the CPU oracle's block power iteration.

FP64 parity: identical per-level sweep counts, every vector within 1e-10
relative 2-norm (both sides apply the sign rule to each vector), every
Rayleigh quotient within 1e-12 relative.  The GPU orthonormalises by a
Cholesky QR of the block, the oracle by modified Gram-Schmidt: the same
vectors in exact arithmetic.
"""
import numpy as np
import pytest

import oracle
from paper_1412_0565_gb300 import cmg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VEC_TOL = 1e-10
LAM_TOL = 1e-12

CASES = {
    "grid_ragged": lambda: inputs.grid2d(45, 71, "uniform", seed=2),
    "grid64_unit": lambda: inputs.grid2d(64, 64, "unit"),
    "rgg": lambda: inputs.rgg(6000, 8.0, seed=5),
    "random": lambda: inputs.random_connected(4000, 12000, seed=3),
    "path": lambda: inputs.path(300),
    "grid_200": lambda: inputs.grid2d(200, 200, "uniform", seed=4),
}


def check(U, lam, st, ref):
    assert st["sweeps"] == ref["sweeps"].tolist()
    for i in range(len(lam)):
        u, r = U[i], ref["U"][i]
        assert np.linalg.norm(u - r) / np.linalg.norm(r) <= VEC_TOL, i
        assert abs(lam[i] - ref["lam"][i]) <= LAM_TOL * abs(ref["lam"][i]), i


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("k", [1, 3, 8])
def test_eigenpairs_match_oracle(name, k):
    rp, col, w = CASES[name]()
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    with cmg.Hierarchy(rp, col, w, seed=1412) as h:
        if k > h.sizes()[0][-1] - 1:
            pytest.skip("coarsest level too small for k vectors")
        U, lam, res, st = h.eigenpairs(k)
    ref = oracle.eigenpairs(oh, k)
    check(U, lam, st, ref)
    # orthonormal, orthogonal to 1
    assert np.allclose(U @ U.T, np.eye(k), atol=1e-12)
    assert np.abs(U.sum(axis=1)).max() <= 1e-11


def test_one_eigenpair_is_the_fiedler_solve():
    rp, col, w = CASES["grid_ragged"]()
    with cmg.Hierarchy(rp, col, w, seed=7) as h:
        u, lam, st = h.fiedler()
        U, lams, _, st2 = h.eigenpairs(1)
    assert st2["sweeps"] == st["sweeps"]
    assert np.linalg.norm(U[0] - u) <= VEC_TOL and abs(lams[0] - lam) <= LAM_TOL * lam


def test_eigenpairs_new_seed_replay_and_device_output():
    rp, col, w = CASES["rgg"]()
    oh = oracle.Hierarchy(rp, col, w, seed=1412)
    base = oracle.eigenpairs(oh, 4, seed=99)
    reps = [max(1, s // 2) for s in base["sweeps"]]
    ref = oracle.eigenpairs(oh, 4, seed=99, replay=reps)
    n = len(rp) - 1
    with cmg.Hierarchy(rp, col, w, seed=1412, schedule="replay", replay_sweeps=reps) as h:
        Ud = torch.empty(4 * n, dtype=torch.float64, device="cuda")
        _, lam, res, st = h.eigenpairs(4, seed=99, U_out=Ud)
    check(Ud.cpu().numpy().reshape(4, n), lam, st, ref)


@pytest.mark.parametrize("k", [0, 17])
def test_eigenpairs_rejects_bad_k(k):
    rp, col, w = CASES["path"]()
    with cmg.Hierarchy(rp, col, w) as h:
        with pytest.raises(cmg.CmgError) as e:
            h.eigenpairs(k)
        assert e.value.name == "ERR_INVALID_ARG"
