"""Pins of the oracle's monomial basis and conic structure against what the
paper fixes: eq. (4) ordering and size, eq. (8) indicator matrices, Prop. 1
(A2 A2^T = diag(n_alpha)), Prop. 3 (weighted case), and the svec isometry."""

import itertools
from math import comb

import numpy as np
import pytest

from instances import workloads as W
from oracle import basis, conic


def test_basis_eq4_prefix_and_size():
    # eq. (4): v_d = [1, x1, ..., xn, x1^2, x1 x2, ..., xn^d]
    v = basis.monomials(3, 2)
    assert v[:10] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                      (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for n, d in [(1, 4), (2, 3), (4, 2), (6, 2), (5, 3)]:
        v = basis.monomials(n, d)
        assert len(v) == comb(n + d, d) == len(set(v))
        # graded, then lexicographically decreasing within a degree
        for a, b in zip(v, v[1:]):
            assert sum(a) < sum(b) or (sum(a) == sum(b) and a > b)
        # every exponent of degree <= d appears
        brute = {e for e in itertools.product(range(d + 1), repeat=n) if sum(e) <= d}
        assert set(v) == brute


@pytest.mark.parametrize("n,lo,d", [(2, 1, 2), (3, 2, 4), (4, 1, 1), (5, 0, 3), (3, 3, 3)])
def test_basis_range(n, lo, d):
    # the reduced basis is v_d restricted to degrees lo..d, in v_d's order
    from instances.program import Block

    v = basis.monomials_range(n, lo, d)
    brute = {e for e in itertools.product(range(d + 1), repeat=n) if lo <= sum(e) <= d}
    assert set(v) == brute and len(v) == len(brute) == Block(d, min_degree=lo).size(n)
    full = basis.monomials(n, d)
    assert v == [e for e in full if sum(e) >= lo]


def _pair_counts(bas):
    cnt = {}
    for b1 in bas:
        for b2 in bas:
            a = tuple(x + y for x, y in zip(b1, b2))
            cnt[a] = cnt.get(a, 0) + 1
    return cnt


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2)])
def test_prop1_diagonal_equals_pair_counts(n, seed):
    cd = conic.build(W.quartic_pop(n, seed))
    A2 = cd.A[:, cd.diag_cols].toarray()
    G = A2 @ A2.T
    off = G - np.diag(np.diag(G))
    assert np.all(off == 0.0)  # Prop. 1: rows of A2 are orthogonal
    bas = cd.blocks[0].basis
    cnt = _pair_counts(bas)
    rows = cd.rows[0]
    expect = np.array([cnt.get(a, 0) for a in rows], dtype=float)
    assert np.array_equal(np.diag(G), expect)  # n_alpha = #{(b,g): b+g = alpha}
    assert expect.sum() == len(bas) ** 2


def test_config0_index_counts():
    # n = 6, 2d = 4: N = 28, m = 210, sum n_alpha = 784, max n_alpha = 6
    cd = conic.build(W.quartic_pop(6, 0))
    assert cd.m == comb(10, 4) == 210
    assert cd.blocks[0].N == comb(8, 2) == 28
    A2 = cd.A[:, cd.diag_cols]
    nalpha = np.asarray(A2.multiply(A2).sum(axis=1)).ravel()
    assert nalpha.sum() == 784 and nalpha.max() == 6 and nalpha.min() >= 1
    # b holds g_0 = p, the u column holds g_1 = 1 (constant row only), c = [w; 0]
    assert cd.A[:, 0].nnz == 1 and cd.A[0, 0] == 1.0
    assert cd.c[0] == -1.0 and np.all(cd.c[1:] == 0.0)


def test_prop3_weighted_block():
    cd = conic.build(W.ball_pop(3, 0))
    A = cd.A.toarray()
    A3 = A[:, cd.diag_cols]
    G3 = A3 @ A3.T
    assert np.all(G3 - np.diag(np.diag(G3)) == 0.0)  # Prop. 3: A3 A3^T diagonal
    wb = [b for b in cd.blocks if b.weighted][0]
    A2 = A[:, wb.offset: wb.offset + wb.N ** 2]
    G2 = A2 @ A2.T
    assert np.any(G2 - np.diag(np.diag(G2)) != 0.0)  # weighted rows overlap (Section VI)
    # each weighted entry (i,k) carries p(x) x^(b_i+b_k): one row per term of p
    nterms = len(W.ball_pop(3, 0).constraints[0].blocks[1].weight)
    assert np.all(np.count_nonzero(A2, axis=0) == nterms)


def test_svec_isometry():
    cd = conic.build(W.ball_pop(2, 0))
    rng = np.random.default_rng(0)
    x = rng.standard_normal(cd.nx)
    y = rng.standard_normal(cd.nx)

    def sym(v):
        out = v.copy()
        for b in cd.blocks:
            X = v[b.offset: b.offset + b.N ** 2].reshape(b.N, b.N, order="F")
            out[b.offset: b.offset + b.N ** 2] = (0.5 * (X + X.T)).reshape(-1, order="F")
        return out

    xs, ys = sym(x), sym(y)
    xp, yp = conic.vec_to_packed(cd, xs), conic.vec_to_packed(cd, ys)
    assert len(xp) == conic.packed_length(cd)
    assert np.isclose(xp @ yp, xs @ ys, rtol=1e-13)
    assert np.allclose(conic.packed_to_vec(cd, xp), xs, atol=1e-14)
    # A acting on symmetric vec equals A acting through the packed map
    Ax = cd.A @ xs
    assert np.allclose(cd.A @ conic.packed_to_vec(cd, xp), Ax, atol=1e-12)
