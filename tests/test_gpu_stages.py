"""GPU tests of the profiling boundary and of the host-side row order:
sos_run_stage runs every stage and single kernel, sos_stage_bytes is
consistent with its definition (sums of the single kernels and of the whole
iteration), running stages 0..2 once equals one full iteration, and an
iterate round-trips bit-exactly through sos_set_iterate / sos_get_iterate
(the device numbers constraint rows by length; the host sees the row order
of the program)."""

import os

import numpy as np
import pytest

from instances import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1708_04174_gb300 import build, capi as c

    if not os.path.exists(c.LIB_PATH):
        build.build()
    return c


BATCH = [W.lyapunov_cubic(3, 2), W.ball_pop(3, 1), W.quartic_pop(4, 0), W.lyapunov_cubic(2, 5)]


def test_stage_bytes_consistent(capi):
    s = capi.Solver(BATCH, precision=capi.PREC_FP64, k_check=10, solve_mode=1)
    b = [s.stage_bytes(k) for k in range(10)]
    assert all(x > 0 for x in b[4:10]), b
    assert b[0] == sum(b[4:10])
    assert b[3] == b[0] + b[1] + b[2]
    for k in range(10):
        s.run_stage(k)
    s.sync()
    with pytest.raises(RuntimeError):
        s.stage_bytes(16)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stages_compose_to_an_iteration(capi, precision):
    prec = {"fp64": capi.PREC_FP64, "mixed": capi.PREC_MIXED}[precision]
    a = capi.Solver(BATCH, precision=prec, k_check=10, solve_mode=1)
    b = capi.Solver(BATCH, precision=prec, k_check=10, solve_mode=1)
    a.iterate(5)
    b.iterate(5)
    a.iterate(1)
    for st in (0, 1, 2):
        b.run_stage(st)
    a.sync()
    b.sync()
    ua, va = a.get_iterate()
    ub, vb = b.get_iterate()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_iterate_round_trip_keeps_row_order(capi):
    s = capi.Solver(BATCH, precision=capi.PREC_FP64, k_check=10)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(s.total)
    v = rng.standard_normal(s.total)
    s.set_iterate(u, v)
    u2, v2 = s.get_iterate()
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    # the split into (xi, y, tau) per instance follows the program's rows
    pos = 0
    for d in s.dims:
        nx, m = d[0], d[1]
        assert np.array_equal(u2[pos + nx:pos + nx + m], u[pos + nx:pos + nx + m])
        pos += nx + m + 1
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_device_iterate_exchange(capi, precision):
    # sos_get_iterate_device / sos_set_iterate_device: the same layout and row
    # order as the host calls; iterating after a device set equals iterating
    # after a host set of the same values
    import torch

    prec = {"fp64": capi.PREC_FP64, "mixed": capi.PREC_MIXED, "fp32": capi.PREC_FP32}[precision]
    # one launch path for both (the autotuner may otherwise pick different ones)
    a = capi.Solver(BATCH, precision=prec, k_check=10, solve_mode=1)
    b = capi.Solver(BATCH, precision=prec, k_check=10, solve_mode=1)
    # the same history on both: the Jacobi projections start from the
    # previous iteration's eigenvectors, so only equal histories give
    # bit-equal iterates
    a.iterate(7)
    b.iterate(7)
    a.sync()
    b.sync()
    uh, vh = a.get_iterate()
    ud = torch.empty(a.total, dtype=torch.float64, device="cuda")
    vd = torch.empty(a.total, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    a.get_iterate_device(ud.data_ptr(), vd.data_ptr())
    a.sync()
    assert np.array_equal(ud.cpu().numpy(), uh) and np.array_equal(vd.cpu().numpy(), vh)

    rng = np.random.default_rng(3)
    u = rng.standard_normal(a.total)
    v = rng.standard_normal(a.total)
    pos = 0
    for d in a.dims:  # tau > 0 and kappa >= 0 as after any ADMM step
        pos += d[0] + d[1]
        u[pos], v[pos] = 1.0 + abs(u[pos]), abs(v[pos])
        pos += 1
    ud.copy_(torch.from_numpy(u))
    vd.copy_(torch.from_numpy(v))
    torch.cuda.synchronize()
    a.set_iterate_device(ud.data_ptr(), vd.data_ptr())
    a.sync()
    b.set_iterate(u, v)
    ua, va = a.get_iterate()
    ub, vb = b.get_iterate()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    if precision != "fp32":
        assert np.array_equal(ua, u) and np.array_equal(va, v)
    a.iterate(5)
    b.iterate(5)
    a.sync()
    b.sync()
    ua, va = a.get_iterate()
    ub, vb = b.get_iterate()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    a.close()
    b.close()
