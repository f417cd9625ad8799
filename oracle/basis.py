"""Monomial bases (oracle; test infrastructure only).

``v_d(x)`` lists every monomial of degree <= d, graded, and within a degree in
lexicographic order with x1 > x2 > ... > xn, i.e. [1, x1, ..., xn, x1^2,
x1 x2, ..., xn^d] as printed in eq. (4).  Its length is C(n+d, d) (Section II-C).
"""

from __future__ import annotations

from math import comb
from typing import List, Tuple

Exp = Tuple[int, ...]


def _level(deg: int, n: int) -> List[Exp]:
    """All exponent vectors of total degree ``deg``, x1-major descending."""
    if n == 1:
        return [(deg,)]
    out: List[Exp] = []
    for first in range(deg, -1, -1):
        for rest in _level(deg - first, n - 1):
            out.append((first,) + rest)
    return out


def monomials(n: int, d: int) -> List[Exp]:
    """Exponents of v_d(x) for n variables (eq. (4))."""
    out: List[Exp] = []
    for deg in range(d + 1):
        out.extend(_level(deg, n))
    assert len(out) == comb(n + d, d)
    return out


def monomials_range(n: int, lo: int, d: int) -> List[Exp]:
    """The monomials of v_d(x) with degree >= lo, in the same order: v_d
    without its first C(n+lo-1, lo-1) entries."""
    out = monomials(n, d)[comb(n + lo - 1, lo - 1) if lo > 0 else 0:]
    assert all(sum(e) >= lo for e in out)
    return out
