"""Pins of the oracle's matrix-valued SOS construction (Section V) against
what the mathematics fixes: Prop. 2 (the Gram part of A has orthogonal rows,
one per triple (alpha, i, j)), the reduction to the scalar case at r = 1, the
constant case (an eigenvalue), the univariate case (a PSD univariate matrix
polynomial is an SOS matrix, so the bound is the minimum of lambda_min over
the line), and the Gram identity (I (x) v)^T Y (I (x) v) = P(x) - gamma I
evaluated pointwise."""

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from instances import workloads as W
from instances.program import Block, Constraint, MatrixConstraint, SOSProgram
from oracle import admm, basis, conic


def _peval(p, x):
    return sum(c * np.prod(np.asarray(x, float) ** np.array(e)) for e, c in p.items())


def _meval(P, x):
    r = len(P)
    return np.array([[_peval(P[i][j], x) for j in range(r)] for i in range(r)])


@pytest.mark.parametrize("n,r", [(2, 2), (3, 3), (1, 4)])
def test_prop2_gram_rows_orthogonal(n, r):
    prog = W.matrix_pop(n, r, 1)
    cd = conic.build(prog)
    A2 = cd.A.tocsc()[:, cd.diag_cols]
    assert np.all(np.diff(A2.indptr) == 1)  # one nonzero per Gram column
    G = (A2 @ A2.T).toarray()
    assert np.count_nonzero(G - np.diag(np.diag(G))) == 0
    # rows (alpha, i, i) count the pairs of the scalar basis (Prop. 1); rows
    # (alpha, i, j), i < j, see both blocks Y_ij and Y_ji: twice as many
    scalar = conic.build(SOSProgram(n=n, w=np.array([-1.0]), constraints=[
        Constraint(degree=4, g0={}, g=[{}], blocks=[Block(2)])]))
    d1 = np.diag((scalar.A @ scalar.A.T).toarray())
    idx = {trip: k for k, trip in enumerate(cd.rows[0])}
    for (a, i, j), k in idx.items():
        k1 = scalar.rows[0].index(a)
        assert G[k, k] == (1 if i == j else 2) * d1[k1]
    assert G.trace() == (r * len(basis.monomials(n, 2))) ** 2


def test_r1_equals_scalar():
    P = W.matrix_poly(3, 1, 4)
    one = [[{(0, 0, 0): 1.0}]]
    mat = SOSProgram(n=3, w=np.array([-1.0]), constraints=[MatrixConstraint(1, 4, P, [one], Block(2))])
    sca = SOSProgram(n=3, w=np.array([-1.0]), constraints=[
        Constraint(degree=4, g0=P[0][0], g=[{(0, 0, 0): 1.0}], blocks=[Block(2)])])
    a, b = conic.build(mat), conic.build(sca)
    assert (a.A != b.A).nnz == 0 and np.array_equal(a.b, b.b) and np.array_equal(a.c, b.c)


@pytest.mark.parametrize("r,seed", [(3, 0), (5, 1)])
def test_constant_matrix_gives_lambda_min(r, seed):
    # degree 0: C - gamma I = Y with Y PSD, so max gamma = lambda_min(C)
    rng = np.random.default_rng(seed)
    Cm = rng.standard_normal((r, r))
    Cm = Cm + Cm.T
    z = (0, 0)
    P0 = [[{z: float(Cm[i, j])} for j in range(r)] for i in range(r)]
    eye = [[({z: 1.0} if i == j else {}) for j in range(r)] for i in range(r)]
    prog = SOSProgram(n=2, w=np.array([-1.0]), constraints=[MatrixConstraint(r, 0, P0, [eye], Block(0))])
    cd = conic.build(prog)
    assert cd.m == r * (r + 1) // 2 and cd.blocks[0].N == r
    res = admm.solve(cd, 1e-11, 200000, k_check=10)
    assert res.status == admm.SOLVED
    assert abs(-res.res["pobj"] - np.linalg.eigvalsh(Cm)[0]) <= 1e-8 * max(1.0, np.abs(Cm).max())


def _line_min_lambda(P):
    xs = np.linspace(-4.0, 4.0, 80001)
    lam = np.array([np.linalg.eigvalsh(_meval(P, [x]))[0] for x in xs[::10]])
    x0 = xs[::10][np.argmin(lam)]
    f = lambda x: np.linalg.eigvalsh(_meval(P, [x]))[0]  # noqa: E731
    return minimize_scalar(f, bounds=(x0 - 2e-3, x0 + 2e-3), method="bounded",
                           options={"xatol": 1e-12}).fun


@pytest.mark.parametrize("r,seed", [(2, 0), (2, 1), (3, 2)])
def test_univariate_matrix_polynomial_minimum(r, seed):
    # a univariate matrix polynomial that is PSD on the line is an SOS matrix
    # with factors of half its degree, so the bound equals min_x lambda_min
    prog = W.matrix_pop(1, r, seed)
    res = admm.solve(conic.build(prog), 1e-10, 400000, k_check=10)
    assert res.status == admm.SOLVED
    gamma = -res.res["pobj"]
    assert abs(gamma - _line_min_lambda(prog.meta["P"])) <= 1e-6 * max(1.0, abs(gamma))


def test_gram_identity_pointwise():
    # at the solution, (I (x) v(x))^T Y (I (x) v(x)) = P(x) - gamma I at any x,
    # evaluated directly (not through A); and gamma is a valid lower bound of
    # lambda_min(P(x)) on samples
    n, r = 2, 3
    prog = W.matrix_pop(n, r, 5)
    cd = conic.build(prog)
    res = admm.solve(cd, 1e-10, 400000, k_check=10)
    assert res.status == admm.SOLVED
    tau = res.u[-1]
    x = res.u[:cd.nx] / tau
    gamma = x[0]
    blk = cd.blocks[0]
    Y = x[blk.offset: blk.offset + blk.N ** 2].reshape(blk.N, blk.N, order="F")
    assert np.linalg.eigvalsh(0.5 * (Y + Y.T))[0] >= -1e-8
    bas = basis.monomials(n, 2)
    rng = np.random.default_rng(0)
    P = prog.meta["P"]
    worst = np.inf
    for _ in range(50):
        pt = rng.uniform(-1.5, 1.5, n)
        v = np.array([np.prod(pt ** np.array(e)) for e in bas])
        Iv = np.kron(np.eye(r), v[:, None])  # (r N) x r
        lhs = Iv.T @ Y @ Iv
        rhs = _meval(P, pt) - gamma * np.eye(r)
        assert np.abs(lhs - rhs).max() <= 1e-6 * max(1.0, np.abs(rhs).max())
        worst = min(worst, np.linalg.eigvalsh(_meval(P, pt))[0])
    assert gamma <= worst + 1e-8
