"""Plain data description of an SOS program in the standard form of eq. (7)
(with the weighted-SOS extension of eq. (37)).

An SOS program has decision variables ``u in R^t`` with cost ``w`` and ``k``
polynomial identities

    g^j_0(x) - sum_i u_i g^j_i(x) = sum_b  p_b(x) * v_{d_b}(x)^T X_b v_{d_b}(x),

one per constraint ``j``.  Each Gram block ``X_b`` (PSD) belongs to exactly one
constraint; ``p_b`` is 1 for a plain SOS block and a fixed polynomial for a
weighted block (Section VI).  Coefficients are matched for every monomial of
degree ``Constraint.min_degree`` .. ``Constraint.degree``.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from math import comb
from typing import Dict, List, Optional, Tuple

import numpy as np

Exp = Tuple[int, ...]
Poly = Dict[Exp, float]


@dataclass
class Block:
    """One Gram block: basis = all monomials of degree ``min_degree`` ..
    ``basis_degree`` in the order of eq. (4) (``min_degree`` 0: the full
    basis v_d).  A smaller basis drops monomials that cannot appear, e.g. the
    constant when the polynomial vanishes to second order at the origin; the
    row structure of Prop. 1 holds for any basis.

    ``weight`` is None for an ordinary SOS block, else the sparse polynomial
    multiplying the Gram form (eq. (38))."""

    basis_degree: int
    weight: Optional[Poly] = None
    min_degree: int = 0

    def size(self, n: int) -> int:
        """N, the number of basis monomials in n variables."""
        low = comb(n + self.min_degree - 1, self.min_degree - 1) if self.min_degree > 0 else 0
        return comb(n + self.basis_degree, self.basis_degree) - low


class Constraint:
    """One polynomial identity of eq. (7).

    ``g`` lists the t polynomials g_1..g_t as sparse dicts.  A generator may
    instead give them as flat term arrays ``term_arrays = (t, index, exps,
    coef)`` (term k adds coef[k] x^exps[k] to g_{index[k]+1}); the dict view
    is then built on first access."""

    def __init__(self, degree: int, g0: Optional[Poly] = None, g: Optional[List[Poly]] = None,
                 blocks: Optional[List[Block]] = None, term_arrays=None, g0_arrays=None, min_degree: int = 0):
        self.degree = degree  # rows: all monomials of degree min_degree .. degree
        self.min_degree = min_degree
        self._g0 = g0
        self._g = g
        self.blocks = list(blocks or [])
        self.term_arrays = term_arrays
        self.g0_arrays = g0_arrays  # (exps [K x n] int, coef [K]) alternative to the dict g0

    @property
    def g0(self) -> Poly:
        if self._g0 is None:
            exps, coef = self.g0_arrays
            self._g0 = {}
            for e, c in zip(map(tuple, np.asarray(exps).tolist()), np.asarray(coef).tolist()):
                if c != 0.0:
                    self._g0[e] = self._g0.get(e, 0.0) + c
        return self._g0

    @property
    def g(self) -> List[Poly]:
        if self._g is None:
            t, idx, exps, coef = self.term_arrays
            out: List[Poly] = [dict() for _ in range(t)]
            for i, e, c in zip(idx.tolist(), map(tuple, exps.tolist()), coef.tolist()):
                out[i][e] = out[i].get(e, 0.0) + c
            self._g = out
        return self._g


class MatrixConstraint:
    """One matrix-valued SOS identity (Section V, eq. (47)-(48)):

        P_0(x) - sum_h u_h P_h(x) = (I_r (x) v(x))^T Y (I_r (x) v(x)),   Y PSD,

    Y of size r N, v the basis of ``block`` (plain, unweighted).  ``P0`` and
    each of the t entries of ``P`` are r x r nested lists of sparse
    polynomials; the matrices are symmetric and only entries [i][j] with
    i <= j are read.  Coefficients are matched for every triple
    (alpha, i, j), i <= j, alpha of degree ``min_degree`` .. ``degree``; the
    rows are ordered by the pairs (i, j) row-major, then alpha in the order
    of eq. (4).  Y's rows and columns are ordered block-major: index
    i N + a is basis monomial a of block row i."""

    def __init__(self, r: int, degree: int, P0, P, block: Block, min_degree: int = 0):
        self.r = r
        self.degree = degree
        self.min_degree = min_degree
        self.P0 = P0
        self.P = list(P)
        self.block = block
        assert block.weight is None

    @property
    def pairs(self) -> List[Tuple[int, int]]:
        return [(i, j) for i in range(self.r) for j in range(i, self.r)]


@dataclass
class SOSProgram:
    n: int
    w: np.ndarray  # (t,)
    constraints: List[Constraint]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def t(self) -> int:
        return int(len(self.w))
