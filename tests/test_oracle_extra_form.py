"""Pins of the oracle's extra-polynomial form (end of Section II) and of the
eq. (42) rule: the rewritten program has the same optimal value as the
weighted one, its sizes follow closed-form monomial counts, and on an
interval the bound is the exact minimum (Markov-Lukacs: a univariate
polynomial of degree 2k that is nonnegative on [-1, 1] equals
s0 + (1 - x^2) s1 with s0, s1 SOS of degrees 2k and 2k - 2)."""

from math import comb

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic, extra_form


@pytest.mark.parametrize("make", [lambda: W.ball_pop(3, 0), lambda: W.lyapunov_local(3, 1),
                                  lambda: W.interval_pop(8, 2)])
def test_same_optimum_both_forms(make):
    prog = make()
    a = admm.solve(conic.build(prog), 1e-9, 400000, k_check=10)
    b = admm.solve(conic.build(extra_form.extra_form(prog)), 1e-9, 400000, k_check=10)
    assert a.status == admm.SOLVED and b.status == admm.SOLVED
    assert abs(a.res["pobj"] - b.res["pobj"]) <= 1e-6 * max(1.0, abs(a.res["pobj"]))


@pytest.mark.parametrize("deg,seed", [(6, 0), (8, 1), (10, 3)])
def test_interval_minimum_exact(deg, seed):
    prog = W.interval_pop(deg, seed)
    assert extra_form.prefers_extra(prog)  # deg >= 6: the multiplier's core is wider than m
    r = admm.solve(conic.build(extra_form.extra_form(prog)), 1e-10, 400000, k_check=10)
    assert r.status == admm.SOLVED
    x = np.linspace(-1.0, 1.0, 2000001)
    pmin = np.min(sum(c * x ** e[0] for e, c in prog.meta["p"].items()))
    assert abs(-r.res["pobj"] - pmin) <= 1e-7 * max(1.0, abs(pmin))


@pytest.mark.parametrize("n,seed", [(2, 0), (4, 2)])
def test_extra_form_sizes(n, seed):
    # ball multiplier s1 with basis v_1: r has C(n+2, 2) coefficients, and the
    # new identity has that many rows and one plain (n+1) x (n+1) block
    prog = W.ball_pop(n, seed)
    cd0 = conic.build(prog)
    cd = conic.build(extra_form.extra_form(prog))
    k = comb(n + 2, 2)
    assert cd.t == cd0.t + k and cd.m == cd0.m + k
    assert not any(b.weighted for b in cd.blocks)
    assert [b.N for b in cd.blocks] == [comb(n + 2, 2), n + 1]
    assert len(cd.lowrank_cols) == cd.t


def test_eq42_rule():
    # direct while t + sum N_i (N_i + 1) / 2 < m
    assert not extra_form.prefers_extra(W.interval_pop(4, 0))   # 1 + 3 < 5
    assert extra_form.prefers_extra(W.interval_pop(8, 0))       # 1 + 10 >= 9
    assert not extra_form.prefers_extra(W.ball_pop(20, 0))      # 1 + 231 < 10626
    assert not extra_form.prefers_extra(W.quartic_pop(3, 0))    # no weighted block
    assert extra_form.direct_width(W.ball_pop(20, 0)) == 232
