"""Pins of the oracle's whole HSDE ADMM (eq. (20)) against results the paper
and the mathematics fix: cone invariants of every iterate, univariate POPs
(nonnegative univariate polynomials are SOS), the closed-form Lyapunov
solution, rank-one moment certificates, Table II, and infeasibility
certificates of the embedding."""

import os

import numpy as np
import pytest

from instances import workloads as W
from instances.program import Block, Constraint, SOSProgram
from oracle import admm, conic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pval(p, x):
    return sum(c * np.prod(np.asarray(x, float) ** np.array(e)) for e, c in p.items())


@pytest.mark.parametrize("make", [lambda: W.quartic_pop(3, 0), lambda: W.ball_pop(2, 0),
                                  lambda: W.lyapunov_cubic(2, 1)])
def test_iterates_stay_in_cones(make):
    """After every step u in C, v in C*, u^T v = 0 and v_y = 0 (eq. (19)-(20))."""
    cd = conic.build(make())
    hs = admm.HSDE(cd)
    u, v = hs.start()
    nx, m, t = hs.nx, hs.m, cd.t
    for _ in range(30):
        u, v = hs.step(u, v)
        scale = max(1.0, np.abs(u).max(), np.abs(v).max())
        assert u[-1] >= 0 and v[-1] >= -1e-12 * scale
        assert np.abs(v[:t]).max(initial=0) <= 1e-12 * scale  # dual of free is {0}
        assert np.abs(v[nx:nx + m]).max() <= 1e-12 * scale  # s = 0
        for b in cd.blocks:
            U = u[b.offset: b.offset + b.N ** 2].reshape(b.N, b.N)
            Z = v[b.offset: b.offset + b.N ** 2].reshape(b.N, b.N)
            assert np.linalg.eigvalsh(U).min() >= -1e-12 * scale
            assert np.linalg.eigvalsh(Z).min() >= -1e-12 * scale
        assert abs(u @ v) <= 1e-10 * scale ** 2


def _grid_min(p):
    xs = np.linspace(-6, 6, 1_200_001)
    vals = np.zeros_like(xs)
    for (e,), c in p.items():
        vals += c * xs ** e
    x = xs[np.argmin(vals)]
    dp = {(e - 1,): c * e for (e,), c in p.items() if e > 0}
    ddp = {(e - 2,): c * e * (e - 1) for (e,), c in p.items() if e > 1}
    for _ in range(30):  # Newton polish on p'
        x -= _pval(dp, [x]) / _pval(ddp, [x])
    return _pval(p, [x])


@pytest.mark.parametrize("deg,seed", [(4, 0), (6, 1), (8, 2)])
def test_univariate_pop_reaches_global_min(deg, seed):
    prog = W.univariate_pop(deg, seed)
    r = admm.solve(conic.build(prog), 1e-10, 100000, k_check=10)
    assert r.status == admm.SOLVED
    gamma = -r.res["pobj"]
    assert abs(gamma - _grid_min(prog.meta["p"])) <= 1e-6 * max(1.0, abs(gamma))


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2)])
def test_lyapunov_quadratic_closed_form(n, seed):
    prog = W.lyapunov_linear(n, seed)
    A = prog.meta["A"]
    K = np.kron(np.eye(n), A.T) + np.kron(A.T, np.eye(n))  # vec(A^T P + P A)
    Pstar = np.linalg.solve(K, -np.eye(n).reshape(-1, order="F")).reshape(n, n, order="F")
    Pstar = 0.5 * (Pstar + Pstar.T)
    assert np.linalg.eigvalsh(Pstar).min() > prog.meta["eps"]
    r = admm.solve(conic.build(prog), 1e-9, 200000, k_check=10)
    assert r.status == admm.SOLVED
    u = r.u[: prog.t] / r.u[-1]
    want = np.array([Pstar[i, j] for (i, j) in prog.meta["pairs"]])
    assert np.allclose(u, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
    assert abs(r.res["pobj"] - np.trace(Pstar)) <= 1e-6 * np.trace(Pstar)


def _moment_certificate(prog, cd, r):
    """Dual y of eq. (17) gives moments mu = -y/tau (mu_0 = 1); if the moment
    matrix is rank one, x* = (mu_{e_1}, ..., mu_{e_n}) is a minimiser."""
    tau = r.u[-1]
    mu = -r.u[cd.nx: cd.nx + cd.m] / tau
    idx = {e: k for k, e in enumerate(cd.rows[0])}
    bas = cd.blocks[0].basis
    Mm = np.array([[mu[idx[tuple(a + b for a, b in zip(b1, b2))]] for b2 in bas] for b1 in bas])
    ev = np.linalg.eigvalsh(Mm)
    return mu, ev


def test_quartic_pop_rank_one_certificate():
    prog = W.quartic_pop(6, 0)
    cd = conic.build(prog)
    r = admm.solve(cd, 1e-9, 50000, k_check=25)
    assert r.status == admm.SOLVED
    mu, ev = _moment_certificate(prog, cd, r)
    assert abs(mu[0] - 1) < 1e-8 and ev[-2] < 1e-7 * ev[-1]
    x = mu[1:prog.n + 1]
    gamma = -r.res["pobj"]
    assert abs(_pval(W.quartic_poly(6, 0), x) - gamma) < 1e-6 * max(1, abs(gamma))


def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_eq46.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, v = line.split()
                rows[int(n)] = float(v)
    return rows


@pytest.mark.parametrize("n", [10, 12, 14])
def test_eq46_relaxation_matches_table2(n):
    """The order-2 relaxation of eq. (46) is exact (rank-one moments at a
    feasible x* with p(x*) = gamma*), and it lies within the 0.5% band the
    paper quotes around its interior-point values (Table II)."""
    prog = W.paper_pop(n)
    cd = conic.build(prog)
    r = admm.solve(cd, 1e-9, 50000, k_check=25)
    assert r.status == admm.SOLVED
    gamma = -r.res["pobj"]
    mu, ev = _moment_certificate(prog, cd, r)
    x = mu[1:n + 1]
    assert ev[-2] < 1e-7 * ev[-1]
    assert np.linalg.norm(x) <= 1 + 1e-6
    assert abs(_pval(W.paper_pop_poly(n), x) - gamma) < 1e-6 * abs(gamma)
    ipm = _table2()[n]
    assert abs(gamma - ipm) <= 0.005 * abs(ipm)


def test_infeasibility_certificates():
    # -1 - u x^2 is never SOS (constant term -1): primal infeasible
    p = SOSProgram(n=1, w=np.array([0.0]),
                   constraints=[Constraint(2, {(0,): -1.0}, [{(2,): 1.0}], [Block(1)])])
    r = admm.solve(conic.build(p), 1e-6, 5000)
    assert r.status == admm.PRIMAL_INFEASIBLE
    # min u s.t. (1 - u) x^2 SOS is unbounded below: dual infeasible
    p = SOSProgram(n=1, w=np.array([1.0]),
                   constraints=[Constraint(2, {(2,): 1.0}, [{(2,): 1.0}], [Block(1)])])
    r = admm.solve(conic.build(p), 1e-6, 5000)
    assert r.status == admm.DUAL_INFEASIBLE


def test_no_false_certificate_for_large_objective():
    # max g s.t. x^4 - 3x^2 + x + 2000 - g is SOS: feasible, optimal value
    # 2000 + min_x (x^4 - 3x^2 + x) against |c| = 1.  Early iterates sit at
    # tau = 0 with |A^T u_y + v_z| / b^T u_y < 1e-3, so a certificate test at
    # the residual tolerance 1e-3 would declare the program infeasible; at its
    # own tolerance (1e-7, taken only while kappa > tau) the solve ends SOLVED
    # at the value a fine grid gives (univariate nonnegative = SOS).
    C = 2000.0
    p = SOSProgram(n=1, w=np.array([-1.0]),
                   constraints=[Constraint(4, g0={(4,): 1.0, (2,): -3.0, (1,): 1.0, (0,): C},
                                           g=[{(0,): 1.0}], blocks=[Block(2)])])
    r = admm.solve(conic.build(p), 1e-3, 20000, k_check=10)
    assert r.status == admm.SOLVED, (r.status, r.res)
    assert any(h["pinf"] <= 1e-3 for h in r.history)  # the unguarded test would have fired
    x = np.linspace(-3, 3, 600001)
    gamma = C + np.min(x ** 4 - 3 * x ** 2 + x)
    assert abs(-r.res["pobj"] - gamma) <= 2e-3 * gamma


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1)])
def test_local_lyapunov_linear_limit(n, seed):
    # Local (ball) Lyapunov program with the Positivstellensatz multiplier and
    # no cubic terms: the left side is a quadratic form, so the multiplier and
    # the quartic part of s0 vanish at the optimum and min trace P is the
    # Lyapunov solution of A^T P + P A + I = 0 (Kronecker form), as in the
    # global linear case; the weighted multiplier block is carried along.
    prog = W.lyapunov_local(n, seed, sigma=0.0)
    A = prog.meta["A"]
    K = np.kron(np.eye(n), A.T) + np.kron(A.T, np.eye(n))
    Pstar = np.linalg.solve(K, -np.eye(n).reshape(-1, order="F")).reshape(n, n, order="F")
    Pstar = 0.5 * (Pstar + Pstar.T)
    assert np.linalg.eigvalsh(Pstar).min() > prog.meta["eps"]
    r = admm.solve(conic.build(prog), 1e-9, 400000, k_check=10)
    assert r.status == admm.SOLVED
    assert abs(r.res["pobj"] - np.trace(Pstar)) <= 1e-5 * np.trace(Pstar)


def test_local_lyapunov_cubic_needs_more():
    # with cubic terms the local certificate exists (linearly stable origin,
    # small ball) and cannot beat the linear optimum: the extra terms only
    # tighten the second identity on the ball
    prog = W.lyapunov_local(3, 1, sigma=1.0)
    lin = W.lyapunov_local(3, 1, sigma=0.0)
    r = admm.solve(conic.build(prog), 1e-8, 400000, k_check=10)
    rl = admm.solve(conic.build(lin), 1e-8, 400000, k_check=10)
    assert r.status == admm.SOLVED and rl.status == admm.SOLVED
    assert r.res["pobj"] >= rl.res["pobj"] * (1 - 1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_binary_quartic_form_reduced_basis(seed):
    # A nonnegative binary form is a sum of squares of forms (Hilbert), so
    # max gamma s.t. p - gamma (x^2 + y^2)^2 SOS, with the Gram basis
    # [x^2, xy, y^2] (degree 2 only) and coefficients matched on the quartic
    # monomials only, is the minimum of p on the unit circle.  This pins the
    # reduced bases (no constant or linear monomials) against brute force.
    rng = np.random.default_rng(seed)
    p = {(4 - k, k): float(v) for k, v in enumerate(rng.standard_normal(5))}
    p[(4, 0)] += 3.0
    p[(0, 4)] += 3.0
    circ = {(4, 0): 1.0, (2, 2): 2.0, (0, 4): 1.0}
    prog = SOSProgram(n=2, w=np.array([-1.0]),
                      constraints=[Constraint(degree=4, g0=p, g=[circ], blocks=[Block(2, min_degree=2)],
                                              min_degree=4)])
    cd = conic.build(prog)
    assert cd.A.shape == (5, 1 + 9) and cd.blocks[0].N == 3
    r = admm.solve(cd, 1e-10, 200000, k_check=10)
    assert r.status == admm.SOLVED
    th = np.linspace(0.0, np.pi, 2000001)  # p is even: half the circle suffices
    gmin = np.min(sum(c * np.cos(th) ** e[0] * np.sin(th) ** e[1] for e, c in p.items()))
    assert abs(-r.res["pobj"] - gmin) <= 1e-6 * max(1.0, abs(gmin))


def test_non_finite_start_is_a_numerical_failure():
    # IEEE propagation: a NaN in the iterate reaches every component through
    # the affine step and the projections, and the first residual check
    # classifies the run as a numerical failure (not a solve, not a raise)
    cd = conic.build(W.quartic_pop(4, 0))
    hs = admm.HSDE(cd)
    u, v = hs.start()
    u = u.copy()
    u[0] = np.nan
    r = admm.solve(cd, 1e-8, 50, k_check=10, u0=u, v0=v)
    assert r.status == admm.NUMERICAL and r.iters == 10
    assert np.isnan(admm.proj_psd(np.array([[1.0, np.nan], [np.nan, 1.0]]))).all()
