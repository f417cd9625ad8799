"""Failure paths of the solver, made on the host and reported as statuses --
never a GPU fault:

* a grid-wide wait of a cooperative kernel bounded so tightly that it runs
  out gives SOS_ERR_TIMEOUT at the next synchronising call, and the same
  handle then iterates on (from a restored iterate) in agreement with the
  oracle;
* a non-finite value planted in the iterate through sos_set_iterate gives
  SOS_NUMERICAL at the same residual check as the oracle started from the
  same point.
"""

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    import os

    from paper_1708_04174_gb300 import build, capi as c

    if not os.path.exists(c.LIB_PATH):
        build.build()
    return c


def packed(cd, x):
    return np.concatenate([conic.vec_to_packed(cd, x[:cd.nx]), x[cd.nx:]])


def test_wait_limit_expiry_reports_timeout_and_context_survives(capi):
    prog = W.ball_pop(20, 0)  # Gram 231 x 231: cooperative projection kernels with grid barriers
    cd = conic.build(prog)
    hs = admm.HSDE(cd)
    u0, v0 = hs.start()
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    s.iterate(2)
    s.sync()
    # 1 us: CTAs without work in a phase reach the first grid barrier long
    # before the others and give up waiting
    s.set_wait_limit(1)
    s.iterate(1)
    with pytest.raises(RuntimeError, match="wait expired"):
        s.sync()
    s.set_wait_limit(0)
    s.set_iterate(packed(cd, u0), packed(cd, v0))
    s.iterate(5)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    u, v = hs.run(5)
    uo, vo = packed(cd, u), packed(cd, v)
    assert np.abs(ug - uo).max() <= 1e-9 * np.abs(uo).max()
    assert np.abs(vg - vo).max() <= 1e-9 * np.abs(vo).max()


def test_non_finite_iterate_reports_numerical(capi):
    prog = W.quartic_pop(6, 0)
    cd = conic.build(prog)
    hs = admm.HSDE(cd)
    u, v = hs.start()
    u = u.copy()
    u[0] = np.nan  # the free variable (gamma)
    ro = admm.solve(cd, 1e-8, 100, k_check=10, u0=u, v0=v)
    assert ro.status == admm.NUMERICAL
    s = capi.Solver(prog, precision=capi.PREC_FP64, k_check=10)
    s.set_iterate(packed(cd, u), packed(cd, v))
    r = s.solve(1e-8, 100, want_solution=False)[0]
    s.close()
    assert r["status"] == capi.NUMERICAL
    assert r["iters"] == ro.iters
