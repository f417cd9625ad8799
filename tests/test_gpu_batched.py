"""GPU tests of the batched persistent solver (one cooperative launch runs
all iterations; device-side residual checks and per-instance termination),
against the FP64 oracle and against the per-phase kernel path."""

import os

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1708_04174_gb300 import build, capi as c

    if not os.path.exists(c.LIB_PATH):
        build.build()
    return c


def _packed(prog, u, v):
    cd = conic.build(prog)
    return (np.concatenate([conic.vec_to_packed(cd, u[:cd.nx]), u[cd.nx:]]),
            np.concatenate([conic.vec_to_packed(cd, v[:cd.nx]), v[cd.nx:]]))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


MIXED_BATCH = [W.quartic_pop(3, 0), W.ball_pop(2, 1), W.lyapunov_cubic(2, 5), W.univariate_pop(6, 3),
               W.lyapunov_cubic(3, 2), W.quartic_pop(4, 1), W.lyapunov_linear(3, 0), W.paper_pop(4)]


def test_persistent_fp64_iterates_match_oracle(capi):
    iters = 60
    s = capi.Solver(MIXED_BATCH, precision=capi.PREC_FP64, solve_mode=2)
    assert s.tuning()["persistent"] == 1 and s.tuning()["candidates"] >= 2
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    for (xg, yg, tg), (zg, sg, kg), prog in zip(s.split(ug), s.split(vg), MIXED_BATCH):
        hs = admm.HSDE(conic.build(prog))
        uo, vo = _packed(prog, *hs.run(iters))
        assert _rel(np.concatenate([xg, yg, [tg]]), uo) < 1e-9
        assert _rel(np.concatenate([zg, sg, [kg]]), vo) < 1e-9
    s.close()


def test_persistent_fp64_iterates_full_size_blocks(capi):
    """The largest blocks of the 4096-search batch (n = 5, 6: Gram blocks of
    21/56 and 28/84, the 512-thread size classes) through the persistent
    launch: FP64 iterates within 1e-9 of the oracle."""
    iters = 40
    progs = W.lyapunov_batch(4, seed=3, n_min=5, n_max=6)
    assert {max(b.size(p.n) for c in p.constraints for b in c.blocks) for p in progs} == {56, 84}
    s = capi.Solver(progs, precision=capi.PREC_FP64, solve_mode=2)
    assert s.tuning()["persistent"] == 1
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    for (xg, yg, tg), (zg, sg, kg), prog in zip(s.split(ug), s.split(vg), progs):
        hs = admm.HSDE(conic.build(prog))
        uo, vo = _packed(prog, *hs.run(iters))
        assert _rel(np.concatenate([xg, yg, [tg]]), uo) < 1e-9
        assert _rel(np.concatenate([zg, sg, [kg]]), vo) < 1e-9
    s.close()


def test_persistent_solve_matches_kernel_path(capi):
    """Same iterates, same checks: statuses, iteration counts and objectives of
    the device-side termination equal the host-side loop of the per-phase path."""
    a = capi.Solver(MIXED_BATCH, precision=capi.PREC_FP64, k_check=10, solve_mode=2)
    b = capi.Solver(MIXED_BATCH, precision=capi.PREC_FP64, k_check=10, solve_mode=1)
    ra = a.solve(1e-6, 20000)
    rb = b.solve(1e-6, 20000)
    for x, y in zip(ra, rb):
        assert x["status"] == y["status"] and x["iters"] == y["iters"], (x["status"], y["status"], x["iters"], y["iters"])
        if x["status"] == capi.SOLVED:
            assert abs(x["obj_primal"] - y["obj_primal"]) <= 1e-9 * max(1.0, abs(y["obj_primal"]))
    a.close()
    b.close()


def test_persistent_statuses_match_oracle(capi):
    progs = W.lyapunov_batch(24, seed=7, n_min=2, n_max=3)
    s = capi.Solver(progs, precision=capi.PREC_FP64, k_check=10, solve_mode=2)
    res = s.solve(1e-5, 20000, want_solution=False)
    s.close()
    for prog, r in zip(progs, res):
        ro = admm.solve(conic.build(prog), 1e-5, 20000, k_check=10)
        assert r["status"] == ro.status, (prog.name, r["status"], ro.status)
        assert r["iters"] == ro.iters, (prog.name, r["iters"], ro.iters)


def test_batched_mixed_lyapunov_form(capi):
    """Batched form (FP64 iterates, FP32 projections, autotuned launch) on a
    seeded Lyapunov batch: its statuses agree with the plain FP64 form (itself
    checked against the oracle) on at least 95% of the instances, and with the
    FP64 oracle on a sample of small ones."""
    progs = W.lyapunov_batch(128, seed=11, n_min=2, n_max=4)
    s = capi.Solver(progs, precision=capi.PREC_MIXED, k_check=10)
    assert s.tuning()["candidates"] >= 3
    res = s.solve(1e-4, 5000, want_solution=False)
    s.close()
    f = capi.Solver(progs, precision=capi.PREC_FP64, k_check=10)
    ref = f.solve(1e-4, 5000, want_solution=False)
    f.close()
    agree = np.mean([a["status"] == b["status"] for a, b in zip(res, ref)])
    assert agree >= 0.95, agree
    small = [i for i, p in enumerate(progs) if p.n == 2][:8]
    for i in small:
        ro = admm.solve(conic.build(progs[i]), 1e-4, 5000, k_check=10)
        assert res[i]["status"] == ro.status, (progs[i].name, res[i]["status"], ro.status)
