"""Plain data description of an SOS program in the standard form of eq. (7)
(with the weighted-SOS extension of eq. (37)).

An SOS program has decision variables ``u in R^t`` with cost ``w`` and ``k``
polynomial identities

    g^j_0(x) - sum_i u_i g^j_i(x) = sum_b  p_b(x) * v_{d_b}(x)^T X_b v_{d_b}(x),

one per constraint ``j``.  Each Gram block ``X_b`` (PSD) belongs to exactly one
constraint; ``p_b`` is 1 for a plain SOS block and a fixed polynomial for a
weighted block (Section VI).  Coefficients are matched for every monomial of
degree <= ``Constraint.degree``.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

Exp = Tuple[int, ...]
Poly = Dict[Exp, float]


@dataclass
class Block:
    """One Gram block: basis = all monomials of degree <= ``basis_degree``.

    ``weight`` is None for an ordinary SOS block, else the sparse polynomial
    multiplying the Gram form (eq. (38))."""

    basis_degree: int
    weight: Optional[Poly] = None


@dataclass
class Constraint:
    """One polynomial identity of eq. (7)."""

    degree: int  # rows: all monomials of degree <= degree
    g0: Poly
    g: List[Poly]  # t polynomials, one per decision variable
    blocks: List[Block]


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
