"""Extra-polynomial form of weighted SOS constraints (oracle; test
infrastructure only).

End of Section II: an SOS condition on a semialgebraic set,
g(x) = s_0(x) + sum_i p_i(x) s_i(x), can be put in the unweighted standard
form of eq. (7) by making each multiplier a free polynomial r_i (its
coefficients join the optimisation vector u) and adding the constraint that
r_i is SOS.  Section VI handles the weighted term directly instead and
gives, in eq. (42), the condition under which that pays off: the low-rank
width t + sum_i (size of X_i) must stay below the number of rows m.  Sizes of
X_i are counted packed here, N_i (N_i + 1) / 2, as everywhere in this
project.

Layout of the result (shared with the library's form, which is built by its
own code): the coefficients r_beta of each weighted block follow the t
original variables (blocks in program order, beta over the monomials of
v v^T in the order of eq. (4)); the identity r(x) = v^T X v of each block
follows the original constraints; the weighted block leaves its constraint.
"""

from __future__ import annotations

from typing import List, Tuple

import numpy as np

from instances.program import Block, Constraint, MatrixConstraint, SOSProgram

from . import basis

Exp = Tuple[int, ...]


def _basis(n: int, blk: Block) -> List[Exp]:
    return basis.monomials_range(n, blk.min_degree, blk.basis_degree)


def products(n: int, blk: Block) -> List[Exp]:
    """The monomials of v v^T (every x^(a+b), a, b in the basis), graded and
    x1-major descending within a degree as in eq. (4)."""
    bas = _basis(n, blk)
    s = {tuple(x + y for x, y in zip(a, b)) for a in bas for b in bas}
    return sorted(s, key=lambda e: (sum(e), tuple(-v for v in e)))


def direct_width(prog: SOSProgram) -> int:
    """t plus the packed size of every weighted Gram block (the order of the
    Woodbury core of the direct form)."""
    w = prog.t
    for con in prog.constraints:
        for blk in getattr(con, "blocks", []):
            if blk.weight is not None:
                N = len(_basis(prog.n, blk))
                w += N * (N + 1) // 2
    return w


def n_rows(prog: SOSProgram) -> int:
    return sum(len(basis.monomials_range(prog.n, getattr(c, "min_degree", 0), c.degree)) for c in prog.constraints)


def prefers_extra(prog: SOSProgram) -> bool:
    """eq. (42) fails: the direct form's core is at least as wide as m."""
    has = any(blk.weight is not None for con in prog.constraints for blk in getattr(con, "blocks", []))
    return has and direct_width(prog) >= n_rows(prog)


def extra_form(prog: SOSProgram) -> SOSProgram:
    """The program with every weighted term p(x) v^T X v replaced by p(x) r(x)
    and a new constraint r(x) = v^T X v, X PSD (end of Section II)."""
    n, t = prog.n, prog.t
    new_vars: List[Tuple[Tuple[int, int], Block, Exp]] = []  # ((constraint, block), block, beta)
    for j, con in enumerate(prog.constraints):
        for bi, blk in enumerate(getattr(con, "blocks", [])):
            if blk.weight is not None:
                new_vars.extend(((j, bi), blk, beta) for beta in products(n, blk))
    t2 = t + len(new_vars)
    w = np.concatenate([np.asarray(prog.w, float), np.zeros(t2 - t)])

    cons: List[Constraint] = []
    for j, con in enumerate(prog.constraints):
        if isinstance(con, MatrixConstraint):  # no weighted blocks: unchanged, zero P_h for the new u
            zero = [[{} for _ in range(con.r)] for _ in range(con.r)]
            cons.append(MatrixConstraint(con.r, con.degree, con.P0, list(con.P) + [zero] * len(new_vars), con.block,
                                         con.min_degree))
            continue
        g = [dict(gi) for gi in con.g] + [dict() for _ in new_vars]
        for k, ((jj, _), blk, beta) in enumerate(new_vars):
            if jj != j:
                continue
            # g_0 - sum u_i g_i - sum r_beta p x^beta = plain Gram forms
            for d, c in blk.weight.items():
                e = tuple(a + b for a, b in zip(beta, d))
                g[t + k][e] = g[t + k].get(e, 0.0) + c
        cons.append(Constraint(degree=con.degree, g0=dict(con.g0), g=g,
                               blocks=[b for b in con.blocks if b.weight is None],
                               min_degree=getattr(con, "min_degree", 0)))
    keys = []
    for key, blk, _ in new_vars:
        if not keys or keys[-1][0] != key:
            keys.append((key, blk))
    for key, blk in keys:
        g = [dict() for _ in range(t2)]
        for k, (kk, _, beta) in enumerate(new_vars):
            if kk == key:
                g[t + k] = {beta: -1.0}  # 0 - sum_beta r_beta (-x^beta) = v^T X v
        cons.append(Constraint(degree=2 * blk.basis_degree, g0={}, g=g,
                               blocks=[Block(blk.basis_degree, None, blk.min_degree)],
                               min_degree=2 * blk.min_degree))
    return SOSProgram(n=n, w=w, constraints=cons, name=prog.name + "+extra", meta=dict(prog.meta))
