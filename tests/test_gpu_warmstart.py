"""GPU test of the learned warm start: a network trained by the library's own
tensor-core kernels on batched solutions of a parametric SOS family lowers
the ADMM iterations to a 1e-4 residual on unseen members, and the
warm-started solves reach the same optimum as cold starts and as the FP64
oracle.  ADMM converges from any start (eq. (20) is an averaged fixed-point
iteration), so the start changes only the iteration count, never the limit."""

import os

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1708_04174_gb300 import build, capi, warmstart

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return capi, warmstart


def test_warm_start_gain(env):
    capi, warmstart = env
    K = 8
    fam = W.ParametricPOP(n=4, K=K, seed=1)  # Gram 15 x 15, m = 70
    th_train = W.ParametricPOP.thetas(2048, 11, K=K)
    th_test = W.ParametricPOP.thetas(128, 12, K=K)
    ws = warmstart.WarmStart(fam, hidden=256, seed=0, precision=capi.PREC_MIXED)
    res, dims, _, _ = ws.solve(th_train, 1e-4, 20000)
    ok = np.array([r["status"] == capi.SOLVED for r in res])
    assert ok.mean() > 0.95
    targets = warmstart.solution_vectors([r for r, k in zip(res, ok) if k], [d for d, k in zip(dims, ok) if k])
    losses = ws.train(th_train[ok], targets, epochs=200, batch=256, lr=1e-3)
    assert len(losses) == 200 and losses[-1] < 0.5 * losses[0], losses[::20]
    pred = ws.predict(th_test)
    assert pred.shape == (128, targets.shape[1]) and np.isfinite(pred).all()
    warm, _, _, _ = ws.solve(th_test, 1e-4, 20000, start=pred)
    cold, _, _, _ = ws.solve(th_test, 1e-4, 20000)
    it_w = np.array([r["iters"] for r in warm])
    it_c = np.array([r["iters"] for r in cold])
    st_w = np.array([r["status"] for r in warm])
    st_c = np.array([r["status"] for r in cold])
    assert (st_w == capi.SOLVED).sum() >= (st_c == capi.SOLVED).sum() - 1
    # the gain: fewer iterations on average and at the median
    assert it_w.mean() <= 0.9 * it_c.mean(), (it_w.mean(), it_c.mean())
    assert np.median(it_w) <= 0.9 * np.median(it_c), (np.median(it_w), np.median(it_c))
    # same optimum: at a 1e-4 relative gap both objectives sit within a few
    # 1e-4 of the optimal value
    both = (st_w == capi.SOLVED) & (st_c == capi.SOLVED)
    for a, b in zip(np.array(warm)[both], np.array(cold)[both]):
        assert abs(a["obj_primal"] - b["obj_primal"]) <= 5e-3 * max(1.0, abs(b["obj_primal"]))
    # and against the FP64 oracle run to 1e-7 on a sample of warm-started members
    for i in np.flatnonzero(st_w == capi.SOLVED)[:3]:
        ro = admm.solve(conic.build(fam.program(th_test[i])), tol=1e-7, max_iter=200000, k_check=50)
        assert ro.status == admm.SOLVED
        assert abs(warm[i]["obj_primal"] - ro.res["pobj"]) <= 5e-3 * max(1.0, abs(ro.res["pobj"]))
