"""CPU tests of libsos's host side: the library loads and exports every symbol
of include/sos.h, its monomial enumeration follows eq. (4), and its host
setup (index map of eq. (8)/(38), P of Prop. 1, b, zeta^T h of eq. (25)) is
bit-exact against the oracle's independent construction.  No GPU needed."""

import os
import re

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, basis, conic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1708_04174_gb300 import build, capi as c

    if not os.path.exists(c.LIB_PATH):
        build.build()
    c.lib()
    return c


def test_exports_match_header(capi):
    hdr = open(os.path.join(ROOT, "include", "sos.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|void\*|void|const char\*)\s+(sos_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(capi.lib(), name), name
    assert declared == set(capi.EXPORTS), declared ^ set(capi.EXPORTS)


@pytest.mark.parametrize("n,d", [(1, 5), (2, 3), (3, 2), (6, 2), (5, 3), (30, 2)])
def test_monomials_match_oracle(capi, n, d):
    assert np.array_equal(capi.monomials(n, d), np.array(basis.monomials(n, d), dtype=np.int32))


PROGS = [
    lambda: W.quartic_pop(3, 0),
    lambda: W.quartic_pop(6, 0),
    lambda: W.ball_pop(2, 1),
    lambda: W.ball_pop(4, 2),
    lambda: W.lyapunov_cubic(2, 5),
    lambda: W.lyapunov_cubic(3, 7),
    lambda: W.lyapunov_linear(3, 0),
    lambda: W.paper_pop(5),
    lambda: W.univariate_pop(6, 2),
    lambda: W.lyapunov_local(4, 2),  # reduced bases and rows
    lambda: W.lyapunov_local(10, 10),
    lambda: W.matrix_pop(2, 2, 0),  # matrix-valued (Section V)
    lambda: W.matrix_pop(3, 3, 1),
    lambda: W.matrix_pop(1, 4, 2),
    lambda: _scalar_and_matrix(),
]


def _scalar_and_matrix():
    # one u shared by a scalar and a matrix-valued constraint (the scalar one's
    # exponents are padded with the matrix encoding's extra variables)
    from instances.program import Block, Constraint, SOSProgram

    mp = W.matrix_pop(2, 2, 3)
    sc = Constraint(degree=4, g0=W.quartic_poly(2, 3), g=[{(0, 0): 1.0}], blocks=[Block(2), Block(1, {(0, 0): 1.0, (2, 0): -1.0})])
    return SOSProgram(n=2, w=np.array([-1.0]), constraints=[sc, mp.constraints[0]])


@pytest.mark.parametrize("make", PROGS)
def test_index_map_bit_exact(capi, make):
    prog = make()
    _check_index_map(capi.host_plan(prog, weighted_form=1), conic.build(prog))


def _two_weighted_constraints():
    # constraint 0: s0 + (1 - x^2 - y^2) s1 + (x + 2) s2 (two weighted blocks);
    # constraint 1: s3 + (4 - y^2) s4; one shared u
    from instances.program import Block, Constraint, SOSProgram

    p = W.quartic_poly(2, 7)
    c0 = Constraint(degree=4, g0=p, g=[{(0, 0): 1.0}],
                    blocks=[Block(2), Block(1, {(0, 0): 1.0, (2, 0): -1.0, (0, 2): -1.0}), Block(1, {(1, 0): 1.0, (0, 0): 2.0})])
    q = W.quartic_poly(2, 8)
    c1 = Constraint(degree=4, g0=q, g=[{(0, 0): 1.0}], blocks=[Block(2), Block(1, {(0, 0): 4.0, (0, 2): -1.0})])
    return SOSProgram(n=2, w=np.array([-1.0]), constraints=[c0, c1])


@pytest.mark.parametrize("make", [lambda: W.ball_pop(2, 1), lambda: W.ball_pop(4, 2), lambda: W.lyapunov_local(4, 2),
                                  lambda: W.interval_pop(8, 0), lambda: _scalar_and_matrix(),
                                  lambda: _two_weighted_constraints()])
def test_extra_form_index_map_bit_exact(capi, make):
    # weighted blocks rewritten with extra polynomials (end of Section II): the
    # library's own rewrite against the oracle's, entry by entry
    from oracle import extra_form

    prog = make()
    _check_index_map(capi.host_plan(prog, weighted_form=2), conic.build(extra_form.extra_form(prog)))


@pytest.mark.parametrize("make", [lambda: W.interval_pop(4, 0), lambda: W.interval_pop(8, 0),
                                  lambda: W.interval_pop(12, 1), lambda: W.ball_pop(3, 0), lambda: W.quartic_pop(3, 0)])
def test_eq42_choice(capi, make):
    # the automatic choice follows eq. (42) as the oracle states it
    from oracle import extra_form

    prog = make()
    want = conic.build(extra_form.extra_form(prog) if extra_form.prefers_extra(prog) else prog)
    assert capi.host_plan(prog)["dims"][2] == want.t


def _check_index_map(hp, cd):
    hs = admm.HSDE(cd)
    nx, m, t, teff, nb, nent = hp["dims"]
    assert (m, t, nb) == (cd.m, cd.t, len(cd.blocks))
    assert nx == conic.packed_length(cd) and nent == nx - t
    assert teff == cd.t + sum(b.N * (b.N + 1) // 2 for b in cd.blocks if b.weighted)
    # oracle: row of each plain Gram entry (column i + j N of vec X has one nonzero)
    A = cd.A.tocsc()
    want = [-1] * cd.t
    for blk in cd.blocks:
        for j in range(blk.N):
            for i in range(j, blk.N):
                if blk.weighted:
                    want.append(-1)
                else:
                    col = A[:, blk.offset + i + j * blk.N]
                    assert col.nnz == 1
                    want.append(int(col.indices[0]))
    assert np.array_equal(hp["ent_row"], np.array(want, dtype=np.int32))
    assert np.array_equal(hp["p_diag"], hs.P)  # 1 + n_alpha, exact small integers
    assert np.array_equal(hp["b"], cd.b)
    assert abs(hp["zeta_h"] - hs.zeta @ hs.h) <= 1e-12 * max(1.0, abs(hs.zeta @ hs.h))


def test_local_lyapunov_matches_table3_shape(capi):
    # n = 10: largest cone N = 65 and factorized width t = n (n + 1) = 110,
    # as in Table III (m differs by the rows this formulation leaves out)
    hp = capi.host_plan(W.lyapunov_local(10, 10))
    nx, m, t, teff, nb, nent = hp["dims"]
    assert teff == 110 and t == 55 and m == 1045


def test_extra_form_of_two_weighted_constraints_keeps_the_optimum(capi):
    # the rewrite with three weighted blocks in two constraints: same optimum
    # as the direct form (oracle), and the library's sizes equal the oracle's
    from oracle import extra_form

    prog = _two_weighted_constraints()
    ex = extra_form.extra_form(prog)
    a = admm.solve(conic.build(prog), 1e-9, 400000, k_check=10)
    b = admm.solve(conic.build(ex), 1e-9, 400000, k_check=10)
    assert a.status == admm.SOLVED and b.status == admm.SOLVED
    assert abs(a.res["pobj"] - b.res["pobj"]) <= 1e-6 * max(1.0, abs(a.res["pobj"]))
    hp = capi.host_plan(prog, weighted_form=2)
    assert hp["dims"][2] == 1 + 3 * 6 and hp["dims"][4] == 5  # 3 x C(4, 2) coefficients; blocks 2 + 3


@pytest.mark.parametrize("defect", ["terms", "weights", "blocks", "negative_terms"])
@pytest.mark.parametrize("form", [0, 2])
def test_setup_rejects_missing_arrays(capi, defect, form):
    # programs built directly as C structs with a count but no array: setup
    # reports INVALID_ARG (before the extra-polynomial rewrite reads anything)
    import ctypes as C

    n = 1
    rows = np.ascontiguousarray([[0], [1], [2]], dtype=np.int32)
    bas = np.ascontiguousarray([[0], [1]], dtype=np.int32)
    wexp = np.ascontiguousarray([[0], [2]], dtype=np.int32)
    wcoef = np.ascontiguousarray([1.0, -1.0])
    tp = np.ascontiguousarray([0, 1], dtype=np.int32)
    te = np.ascontiguousarray([[2], [0]], dtype=np.int32)
    tc = np.ascontiguousarray([1.0, 1.0])
    w = np.ascontiguousarray([-1.0])
    blk = (capi.sos_block * 2)()
    for b in blk:
        b.N = 2
        b.basis_exps = bas.ctypes.data_as(C.POINTER(C.c_int32))
    blk[1].N = 1
    blk[1].n_weight_terms = 2
    blk[1].weight_exps = None if defect == "weights" else wexp.ctypes.data_as(C.POINTER(C.c_int32))
    blk[1].weight_coef = wcoef.ctypes.data_as(C.POINTER(C.c_double))
    con = (capi.sos_constraint * 1)()
    con[0].n_rows = 3
    con[0].row_exps = rows.ctypes.data_as(C.POINTER(C.c_int32))
    con[0].n_terms = -1 if defect == "negative_terms" else 2
    con[0].term_poly = None if defect == "terms" else tp.ctypes.data_as(C.POINTER(C.c_int32))
    con[0].term_exps = te.ctypes.data_as(C.POINTER(C.c_int32))
    con[0].term_coef = tc.ctypes.data_as(C.POINTER(C.c_double))
    con[0].n_blocks = 2
    con[0].blocks = None if defect == "blocks" else blk
    prog = (capi.sos_program * 1)()
    prog[0].n_vars = n
    prog[0].t = 1
    prog[0].w = w.ctypes.data_as(C.POINTER(C.c_double))
    prog[0].n_constraints = 1
    prog[0].constraints = con
    dims = (C.c_int64 * 6)()
    rc = capi.lib().sos_host_plan(prog, form, dims, None, None, None, None)
    assert rc == capi.SOS_ERR_INVALID_ARG


def test_factor_failure_is_reported(capi):
    # a NaN coefficient makes the Woodbury core non-finite; the threaded
    # Cholesky (core of order 420) stops in every thread and setup reports it
    prog = W.lyapunov_local(20, 20)
    g = prog.constraints[1].g[0]
    g[next(iter(g))] = float("nan")
    with pytest.raises(RuntimeError, match="positive definite"):
        capi.host_plan(prog)


def test_setup_rejects_bad_input(capi):
    from instances.program import Block, Constraint, SOSProgram

    # g_1 has a monomial of degree 5 that is not among the degree-4 rows
    bad = SOSProgram(n=1, w=np.array([1.0]), constraints=[Constraint(4, {(0,): 1.0}, [{(5,): 1.0}], [Block(2)])])
    with pytest.raises(RuntimeError, match="not among"):
        capi.host_plan(bad)
    # a Gram block whose products exceed the rows
    bad = SOSProgram(n=1, w=np.array([1.0]), constraints=[Constraint(2, {(0,): 1.0}, [{(0,): 1.0}], [Block(2)])])
    with pytest.raises(RuntimeError, match="not among"):
        capi.host_plan(bad)


@pytest.mark.parametrize("kw,msg", [(dict(warm_restart=-1), "warm_restart"), (dict(infeas_tol=-1.0), "infeas_tol"),
                                    (dict(weighted_form=3), "weighted_form"),
                                    (dict(precision=7), "precision"), (dict(solve_mode=3), "solve_mode"),
                                    (dict(large_method=5), "large_method")])
def test_setup_rejects_bad_options(capi, kw, msg):
    # option checks run before any CUDA call, so they need no GPU
    with pytest.raises(RuntimeError, match=msg):
        capi.Solver(W.quartic_pop(3, 0), **kw)


def test_native_matrix_constraint_rows_by_hand(capi):
    """A matrix-valued constraint (Section V) built directly in the C structs,
    with literal arrays only -- no coefficient arithmetic on the Python side:
    P_0(x) - u P_1 = (I_2 (x) v)^T Y (I_2 (x) v), P_0 = [[1 + x^2, x], [x, 2]],
    P_1 = I, v = (1, x).  Prop. 2 rows (alpha, i, j), i <= j, pairs row-major
    then alpha in (1, x, x^2): b holds (P_0)_ii and 2 (P_0)_01 (both Y_01 and
    Y_10 enter the same row); P = I + A_D A_D^T counts every packed Gram
    entry of a row once, with weight 1 on the diagonal of Y and 2 off it."""
    import ctypes as C

    row_exps = (C.c_int32 * 3)(0, 1, 2)
    # terms: (poly, exponent, coefficient, pair)
    term_poly = (C.c_int32 * 6)(0, 0, 0, 0, 1, 1)
    term_exps = (C.c_int32 * 6)(0, 2, 1, 0, 0, 0)
    term_coef = (C.c_double * 6)(1.0, 1.0, 1.0, 2.0, 1.0, 1.0)
    term_pair = (C.c_int32 * 12)(0, 0, 0, 0, 0, 1, 1, 1, 0, 0, 1, 1)
    basis_exps = (C.c_int32 * 2)(0, 1)
    blk = (capi.sos_block * 1)()
    blk[0].N = 2
    blk[0].basis_exps = C.cast(basis_exps, C.POINTER(C.c_int32))
    blk[0].n_weight_terms = 0
    con = (capi.sos_constraint * 1)()
    con[0].n_rows = 3
    con[0].row_exps = C.cast(row_exps, C.POINTER(C.c_int32))
    con[0].n_terms = 6
    con[0].term_poly = C.cast(term_poly, C.POINTER(C.c_int32))
    con[0].term_exps = C.cast(term_exps, C.POINTER(C.c_int32))
    con[0].term_coef = C.cast(term_coef, C.POINTER(C.c_double))
    con[0].n_blocks = 1
    con[0].blocks = blk
    con[0].matrix_r = 2
    con[0].term_pair = C.cast(term_pair, C.POINTER(C.c_int32))
    w = (C.c_double * 1)(-1.0)
    prog = (capi.sos_program * 1)()
    prog[0].n_vars = 1
    prog[0].t = 1
    prog[0].w = C.cast(w, C.POINTER(C.c_double))
    prog[0].n_constraints = 1
    prog[0].constraints = con
    lib = capi.lib()
    dims = (C.c_int64 * 6)()
    assert lib.sos_host_plan(prog, 1, dims, None, None, None, None) == capi.SOS_OK
    assert (dims[0], dims[1]) == (1 + 10, 9)  # u, then the packed 4 x 4 Y; 3 pairs x 3 monomials
    ent = np.zeros(dims[0], dtype=np.int32)
    pd = np.zeros(dims[1])
    b = np.zeros(dims[1])
    zh = C.c_double(0)
    assert lib.sos_host_plan(prog, 1, dims, ent.ctypes.data_as(C.POINTER(C.c_int32)),
                             pd.ctypes.data_as(C.POINTER(C.c_double)), b.ctypes.data_as(C.POINTER(C.c_double)),
                             C.byref(zh)) == capi.SOS_OK
    #               (0,0): 1  x  x^2   (0,1): 1  x  x^2   (1,1): 1  x  x^2
    assert b.tolist() == [1.0, 0.0, 1.0, 0.0, 2.0, 0.0, 2.0, 0.0, 0.0]
    assert pd.tolist() == [2.0, 3.0, 2.0, 3.0, 5.0, 3.0, 2.0, 3.0, 2.0]
