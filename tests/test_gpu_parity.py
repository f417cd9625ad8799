"""GPU parity: libsos (CUDA, through the C-ABI) against the FP64 CPU oracle on
the same seeded programs.

* plain FP64 form: the HSDE iterates after a fixed number of ADMM iterations
  agree within 1e-9 relative (max-norm, per vector);
* converged objectives agree within 1e-6 relative; statuses agree;
* FP32 form: iterates and objectives within the error that FP32 projections
  allow (bounds stated in each test).
"""

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1708_04174_gb300 import build, capi as c

    import os

    if not os.path.exists(c.LIB_PATH):
        build.build()
    return c


def oracle_packed(prog, iters):
    cd = conic.build(prog)
    hs = admm.HSDE(cd)
    u, v = hs.run(iters)
    uo = np.concatenate([conic.vec_to_packed(cd, u[:cd.nx]), u[cd.nx:]])
    vo = np.concatenate([conic.vec_to_packed(cd, v[:cd.nx]), v[cd.nx:]])
    return uo, vo


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    ("quartic_n3", lambda: W.quartic_pop(3, 0), 60),
    ("config0_quartic_n6", lambda: W.quartic_pop(6, 0), 200),
    ("univariate_odd_N", lambda: W.univariate_pop(4, 1), 80),
    ("ball_n2_weighted", lambda: W.ball_pop(2, 1), 80),
    ("ball_n5_weighted", lambda: W.ball_pop(5, 0), 60),
    ("lyapunov_cubic_n2", lambda: W.lyapunov_cubic(2, 5), 60),
    ("lyapunov_cubic_n3", lambda: W.lyapunov_cubic(3, 1), 40),
    ("lyapunov_linear_n4", lambda: W.lyapunov_linear(4, 3), 60),
    ("eq46_n6", lambda: W.paper_pop(6), 60),
    ("lyapunov_local_n4_ball", lambda: W.lyapunov_local(4, 2), 60),
    ("lyapunov_local_n7_grid", lambda: W.lyapunov_local(7, 0), 40),  # N = 36: one program, FP64 grid path
    ("matrix_n2_r2", lambda: W.matrix_pop(2, 2, 0), 60),  # matrix-valued (Section V): Y 12 x 12
    ("matrix_n3_r3", lambda: W.matrix_pop(3, 3, 1), 60),
    ("matrix_n6_r3_grid", lambda: W.matrix_pop(6, 3, 0), 40),  # Y 84 x 84: FP64 grid path
    ("scalar_and_matrix", lambda: _scalar_and_matrix(), 60),
]


def _scalar_and_matrix():
    from instances.program import Block, Constraint, SOSProgram

    mp = W.matrix_pop(2, 2, 3)
    sc = Constraint(degree=4, g0=W.quartic_poly(2, 3), g=[{(0, 0): 1.0}],
                    blocks=[Block(2), Block(1, {(0, 0): 1.0, (2, 0): -1.0})])
    return SOSProgram(n=2, w=np.array([-1.0]), constraints=[sc, mp.constraints[0]])


@pytest.mark.parametrize("name,make,iters", CASES, ids=[c[0] for c in CASES])
def test_fp64_iterates_match_oracle(capi, name, make, iters):
    prog = make()
    uo, vo = oracle_packed(prog, iters)
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    assert rel(ug, uo) < 1e-9, rel(ug, uo)
    assert rel(vg, vo) < 1e-9, rel(vg, vo)


def test_fp64_batch_matches_oracle_per_instance(capi):
    progs = [W.quartic_pop(3, 0), W.ball_pop(2, 1), W.lyapunov_cubic(2, 5), W.univariate_pop(6, 3),
             W.lyapunov_cubic(3, 2)]
    iters = 50
    s = capi.Solver(progs, precision=capi.PREC_FP64)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    for (xg, yg, tg), (zg, sg, kg), prog in zip(s.split(ug), s.split(vg), progs):
        uo, vo = oracle_packed(prog, iters)
        assert rel(np.concatenate([xg, yg, [tg]]), uo) < 1e-9
        assert rel(np.concatenate([zg, sg, [kg]]), vo) < 1e-9
    s.close()


def test_fp64_large_block_config1(capi):
    """Constrained quartic POP n = 20 (Gram 231 + weighted 21, m = 10626):
    the large-block (grid Jacobi) path with a ragged tile tail."""
    prog = W.ball_pop(20, 0)
    iters = 12
    uo, vo = oracle_packed(prog, iters)
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    assert rel(ug, uo) < 1e-9, rel(ug, uo)
    assert rel(vg, vo) < 1e-9, rel(vg, vo)


def test_fp64_config1_warm_attempts_keep_parity(capi):
    """Config 1 over 240 iterations: from about iteration 17 on, each
    iteration first refines the previous iteration's eigenvectors (the cold
    tridiagonal path runs only when that attempt gives up); the FP64 iterates
    stay within 1e-9 of the oracle."""
    prog = W.ball_pop(20, 0)
    iters = 240
    uo, vo = oracle_packed(prog, iters)
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    assert rel(ug, uo) < 1e-9, rel(ug, uo)
    assert rel(vg, vo) < 1e-9, rel(vg, vo)


def test_fp64_config1_solve_to_1e6(capi):
    """Constrained quartic POP n = 20 (Gram 231 + weighted 21) solved to a
    1e-6 residual: the same number of iterations as the oracle (same checks
    every 10 iterations) and the objective within 1e-6 relative."""
    prog = W.ball_pop(20, 0)
    ro = admm.solve(conic.build(prog), 1e-6, 5000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_FP64, k_check=10)
    r = s.solve(1e-6, 5000, want_solution=False)[0]
    s.close()
    assert r["status"] == capi.SOLVED and ro.status == admm.SOLVED
    assert r["iters"] == ro.iters, (r["iters"], ro.iters)
    assert abs(r["obj_primal"] - ro.res["pobj"]) <= 1e-6 * abs(ro.res["pobj"])


def test_fp64_solve_objective_and_status(capi):
    prog = W.quartic_pop(6, 0)
    cd = conic.build(prog)
    ro = admm.solve(cd, 1e-8, 50000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_FP64, k_check=10)
    r = s.solve(1e-8, 50000)[0]
    s.close()
    assert r["status"] == capi.SOLVED and ro.status == admm.SOLVED
    assert abs(r["obj_primal"] - ro.res["pobj"]) <= 1e-6 * abs(ro.res["pobj"])
    assert r["iters"] == ro.iters  # same iterates, same checks


def test_infeasibility_statuses(capi):
    from instances.program import Block, Constraint, SOSProgram

    pinf = SOSProgram(n=1, w=np.array([0.0]),
                      constraints=[Constraint(2, {(0,): -1.0}, [{(2,): 1.0}], [Block(1)])])
    dinf = SOSProgram(n=1, w=np.array([1.0]),
                      constraints=[Constraint(2, {(2,): 1.0}, [{(2,): 1.0}], [Block(1)])])
    s = capi.Solver([pinf, dinf], precision=capi.PREC_FP64, k_check=1)
    r = s.solve(1e-6, 5000)
    s.close()
    assert r[0]["status"] == capi.PRIMAL_INFEASIBLE
    assert r[1]["status"] == capi.DUAL_INFEASIBLE


@pytest.mark.parametrize("name,make", [("config0_quartic_n6", lambda: W.quartic_pop(6, 0)),
                                       ("ball_n6_weighted", lambda: W.ball_pop(6, 1)),
                                       ("config1_ball_n20", lambda: W.ball_pop(20, 0))])
def test_mixed_form_objective_error_vs_oracle(capi, name, make):
    """FP64 iterates with FP32 projections reach the 1e-4 residual, and their
    objective is within 1e-3 relative of the FP64 oracle's (solved to 1e-7).
    At tolerance 1e-4 the termination rule itself admits objective errors of
    a few times 1e-4 (gap <= 1e-4 (1 + |c^T x| + |b^T y|) plus the primal and
    dual residuals), so the bound is 1e-3."""
    prog = make()
    cd = conic.build(prog)
    ro = admm.solve(cd, 1e-7, 50000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_MIXED, k_check=10)
    r = s.solve(1e-4, 20000)[0]
    s.close()
    assert r["status"] == capi.SOLVED, r
    err = abs(r["obj_primal"] - ro.res["pobj"]) / abs(ro.res["pobj"])
    assert err < 1e-3, err


def test_mixed_form_iterates_close_to_oracle(capi):
    """After 100 iterations the FP32-projection iterates stay within the FP32
    rounding of the projections of the FP64 oracle's iterates."""
    prog = W.quartic_pop(6, 0)
    uo, vo = oracle_packed(prog, 100)
    s = capi.Solver(prog, precision=capi.PREC_MIXED)
    s.iterate(100)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    assert rel(ug, uo) < 1e-4 and rel(vg, vo) < 1e-4, (rel(ug, uo), rel(vg, vo))


def test_fp32_iterate_form_error_vs_oracle(capi):
    prog = W.quartic_pop(6, 0)
    cd = conic.build(prog)
    ro = admm.solve(cd, 1e-6, 50000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_FP32, k_check=10)
    r = s.solve(1e-4, 50000)[0]
    s.close()
    assert r["status"] == capi.SOLVED
    err = abs(r["obj_primal"] - ro.res["pobj"]) / abs(ro.res["pobj"])
    assert err < 1e-3, err


def test_warm_start_keeps_fp64_parity_over_many_iterations(capi):
    """Eigenvectors kept across iterations (warm Jacobi) do not change the FP64
    iterates beyond rounding: 400 iterations of config 0 stay within 1e-9."""
    prog = W.quartic_pop(6, 0)
    uo, vo = oracle_packed(prog, 400)
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    s.iterate(400)
    s.sync()
    ug, vg = s.get_iterate()
    st = s.stats()
    s.close()
    assert rel(ug, uo) < 1e-9 and rel(vg, vo) < 1e-9, (rel(ug, uo), rel(vg, vo))
    assert st["max_sweeps"] <= 6, st  # warm start: a few sweeps instead of ~9


def test_local_lyapunov_linear_limit_gpu(capi):
    # the Positivstellensatz program without cubic terms: min trace P is the
    # Lyapunov solution of A^T P + P A + I = 0 (Kronecker form)
    prog = W.lyapunov_local(3, 1, sigma=0.0)
    A = prog.meta["A"]
    n = 3
    K = np.kron(np.eye(n), A.T) + np.kron(A.T, np.eye(n))
    Pstar = np.linalg.solve(K, -np.eye(n).reshape(-1, order="F")).reshape(n, n, order="F")
    s = capi.Solver(prog, precision=capi.PREC_FP64)
    r = s.solve(1e-9, 400000)[0]
    s.close()
    assert r["status"] == capi.SOLVED
    assert abs(r["obj_primal"] - np.trace(Pstar)) <= 1e-6 * np.trace(Pstar)


@pytest.mark.parametrize("precision,make,tol", [
    ("fp64", lambda: W.matrix_pop(1, 3, 2), 1e-6),
    ("mixed", lambda: W.matrix_pop(6, 3, 0), 1e-3),   # Y 84: FP32 Jacobi + refinement
    ("mixed", lambda: W.matrix_pop(8, 3, 0), 1e-3),   # Y 135: tensor-core Newton-Schulz
])
def test_matrix_valued_objective_vs_oracle(capi, precision, make, tol):
    """Matrix-valued SOS (Section V): the plain form solved to 1e-8 gives the
    oracle's objective within 1e-6 (same iteration count); the mixed form
    solved to 1e-4 within 1e-3 (the termination rule's own slack)."""
    prog = make()
    ro = admm.solve(conic.build(prog), 1e-7 if precision == "mixed" else 1e-8, 50000, k_check=10)
    prec = capi.PREC_FP64 if precision == "fp64" else capi.PREC_MIXED
    s = capi.Solver(prog, precision=prec, k_check=10)
    r = s.solve(1e-8 if precision == "fp64" else 1e-4, 50000)[0]
    s.close()
    assert r["status"] == capi.SOLVED and ro.status == admm.SOLVED
    assert abs(r["obj_primal"] - ro.res["pobj"]) <= tol * abs(ro.res["pobj"])
    if precision == "fp64":
        assert r["iters"] == ro.iters


@pytest.mark.parametrize("make,iters", [(lambda: W.ball_pop(4, 2), 60), (lambda: W.lyapunov_local(4, 2), 60),
                                        (lambda: W.interval_pop(8, 0), 80)])
def test_extra_form_iterates_match_oracle(capi, make, iters):
    """Weighted blocks rewritten with extra polynomials (end of Section II) by
    the library's setup: FP64 iterates within 1e-9 of the oracle run on its
    own rewrite of the program."""
    from oracle import extra_form

    prog = make()
    uo, vo = oracle_packed(extra_form.extra_form(prog), iters)
    s = capi.Solver(prog, precision=capi.PREC_FP64, weighted_form=2)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    s.close()
    assert rel(ug, uo) < 1e-9, rel(ug, uo)
    assert rel(vg, vo) < 1e-9, rel(vg, vo)


@pytest.mark.parametrize("deg,seed", [(8, 1), (12, 4)])
def test_interval_minimum_by_eq42_choice(capi, deg, seed):
    """The automatic choice takes the extra form here (eq. (42) fails) and the
    solve reaches the exact minimum on [-1, 1] (Markov-Lukacs)."""
    prog = W.interval_pop(deg, seed)
    s = capi.Solver(prog, precision=capi.PREC_FP64, k_check=10)
    assert s.dims[0][2] > prog.t  # the extra coefficients joined u
    r = s.solve(1e-10, 200000)[0]
    s.close()
    assert r["status"] == capi.SOLVED
    x = np.linspace(-1.0, 1.0, 2000001)
    pmin = np.min(sum(c * x ** e[0] for e, c in prog.meta["p"].items()))
    assert abs(-r["obj_primal"] - pmin) <= 1e-7 * max(1.0, abs(pmin))


def test_batch_with_per_instance_weighted_form(capi):
    """eq. (42) is applied per program: in one batch an interval POP of
    degree 8 takes the extra form and a ball POP the direct one; each
    instance's FP64 iterates match the oracle on that instance's form."""
    from oracle import extra_form

    progs = [W.interval_pop(8, 5), W.ball_pop(3, 2), W.interval_pop(4, 6), W.matrix_pop(2, 2, 4)]
    iters = 50
    s = capi.Solver(progs, precision=capi.PREC_FP64)
    s.iterate(iters)
    s.sync()
    ug, vg = s.get_iterate()
    for (xg, yg, tg), (zg, sg, kg), prog in zip(s.split(ug), s.split(vg), progs):
        form = extra_form.extra_form(prog) if extra_form.prefers_extra(prog) else prog
        uo, vo = oracle_packed(form, iters)
        assert rel(np.concatenate([xg, yg, [tg]]), uo) < 1e-9
        assert rel(np.concatenate([zg, sg, [kg]]), vo) < 1e-9
    assert [d[2] for d in s.dims] == [8, 1, 1, 1]
    s.close()
