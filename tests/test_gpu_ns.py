"""GPU tests of the Newton-Schulz PSD projection on the tensor cores
(tcgen05, BF16 three-part split operands, FP32 accumulation), used for large
Gram blocks in the FP32-projection forms: the mixed form with it reaches the
oracle's objective within the error its tolerance allows."""

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


@pytest.mark.parametrize("name,make", [("quartic_n15_N136", lambda: W.quartic_pop(15, 0)),
                                       ("config1_ball_n20_N231", lambda: W.ball_pop(20, 0))])
def test_ns_mixed_form_objective(capi, name, make):
    prog = make()
    ro = admm.solve(conic.build(prog), 1e-7, 50000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_MIXED, k_check=10, large_method=2)
    r = s.solve(1e-4, 20000)[0]
    st = s.stats()
    s.close()
    assert r["status"] == capi.SOLVED, r
    err = abs(r["obj_primal"] - ro.res["pobj"]) / abs(ro.res["pobj"])
    assert err < 1e-3, err
    assert 5 <= st["max_sweeps"] < 60, st  # Newton-Schulz iterations of the last projection


def test_ns_iterates_track_oracle(capi):
    """40 iterations with the tensor-core projection stay within 1e-4 of the
    FP64 oracle's iterates (relative, max-norm)."""
    prog = W.quartic_pop(15, 0)
    cd = conic.build(prog)
    u, v = admm.HSDE(cd).run(40)
    uo = np.concatenate([conic.vec_to_packed(cd, u[:cd.nx]), u[cd.nx:]])
    s = capi.Solver(prog, precision=capi.PREC_MIXED, large_method=2)
    s.iterate(40)
    s.sync()
    ug, _ = s.get_iterate()
    s.close()
    assert np.abs(ug - uo).max() / np.abs(uo).max() < 1e-4
