"""Seeded workload generators shaped like the paper's experiments.

Every generator returns an :class:`instances.SOSProgram`.  Random coefficients
come from ``numpy.random.default_rng(seed)`` and are drawn in graded
lexicographic order of their support, so a (generator, seed) pair names one
fixed problem.

Workloads:

* ``quartic_pop``      - unconstrained quartic POP  max g s.t. p - g SOS (eq. (9)),
                          p = (sum x_i^2)^2 + sum_{|a|<=3} c_a x^a, c_a ~ N(0,1).
* ``ball_pop``         - the same p on the unit ball through the order-2 Lasserre
                          relaxation p - g = s0 + s1 (1 - |x|^2) (eq. (12)-(13)),
                          with s1 handled as a weighted SOS block (Section VI).
* ``paper_pop``        - the constrained quartic POP of eq. (46) (Tables I-II).
* ``univariate_pop``   - n = 1, where nonnegative polynomials are SOS.
* ``lyapunov_linear``  - quadratic V for x' = A x, cost trace(P) (closed form).
* ``lyapunov_cubic``   - global Lyapunov search for x' = -x + cubic(x) with a
                          degree-4 V (eq. (10) with an eps |x|^2 margin).
* ``parametric_pop``   - p = p0 + sum_k theta_k q_k (learned warm-start family).
"""

from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

from .program import Block, Constraint, MatrixConstraint, SOSProgram

Exp = Tuple[int, ...]
Poly = Dict[Exp, float]


# --------------------------------------------------------------------------
# sparse polynomial helpers used only to *write down* input polynomials
# --------------------------------------------------------------------------

def _compositions_desc(total: int, parts: int):
    """All exponent tuples of length ``parts`` summing to ``total``, in
    decreasing lexicographic order."""
    if parts == 1:
        yield (total,)
        return
    for first in range(total, -1, -1):
        for rest in _compositions_desc(total - first, parts - 1):
            yield (first,) + rest


def _support(n: int, max_deg: int, min_deg: int = 0) -> List[Exp]:
    """Exponents of degree min_deg..max_deg, graded, then x1 > x2 > ... lex.

    Used only to fix the order in which random coefficients are drawn."""
    out: List[Exp] = []
    for deg in range(min_deg, max_deg + 1):
        out.extend(_compositions_desc(deg, n))
    return out


def _unit(n: int, i: int, k: int = 1) -> Exp:
    e = [0] * n
    e[i] = k
    return tuple(e)


def _zero(n: int) -> Exp:
    return tuple([0] * n)


def padd(*ps: Poly, scale: Sequence[float] | None = None) -> Poly:
    out: Poly = {}
    for idx, p in enumerate(ps):
        s = 1.0 if scale is None else float(scale[idx])
        for e, c in p.items():
            out[e] = out.get(e, 0.0) + s * c
    return {e: c for e, c in out.items() if c != 0.0}


def pmul(p: Poly, q: Poly) -> Poly:
    out: Poly = {}
    for e1, c1 in p.items():
        for e2, c2 in q.items():
            e = tuple(a + b for a, b in zip(e1, e2))
            out[e] = out.get(e, 0.0) + c1 * c2
    return {e: c for e, c in out.items() if c != 0.0}


def pdiff(p: Poly, i: int) -> Poly:
    out: Poly = {}
    for e, c in p.items():
        if e[i] > 0:
            f = list(e)
            f[i] -= 1
            out[tuple(f)] = out.get(tuple(f), 0.0) + c * e[i]
    return out


def sq_norm(n: int, scale: float = 1.0) -> Poly:
    return {_unit(n, i, 2): scale for i in range(n)}


def _random_low_part(n: int, rng: np.random.Generator, deg: int = 3) -> Poly:
    sup = _support(n, deg)
    coef = rng.standard_normal(len(sup))
    return {e: float(c) for e, c in zip(sup, coef)}


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def quartic_poly(n: int, seed: int) -> Poly:
    """p = (sum x_i^2)^2 + sum_{|a|<=3} c_a x^a with c_a ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    s = sq_norm(n)
    return padd(pmul(s, s), _random_low_part(n, rng))


def _pop_program(n: int, p: Poly, name: str, ball: bool) -> SOSProgram:
    blocks = [Block(2)]
    if ball:
        blocks.append(Block(1, padd({_zero(n): 1.0}, sq_norm(n, -1.0))))
    con = Constraint(degree=4, g0=p, g=[{_zero(n): 1.0}], blocks=blocks)
    return SOSProgram(n=n, w=np.array([-1.0]), constraints=[con], name=name)


def quartic_pop(n: int, seed: int = 0) -> SOSProgram:
    """Unconstrained quartic POP: min -g s.t. p - g is SOS (eq. (9))."""
    return _pop_program(n, quartic_poly(n, seed), f"quartic_pop(n={n},seed={seed})", ball=False)


def ball_pop(n: int, seed: int = 0) -> SOSProgram:
    """Quartic POP on the unit ball, order-2 Lasserre relaxation as a weighted
    SOS constraint: p - g = s0 + s1 (1 - |x|^2), s0 deg 4, s1 deg 2."""
    return _pop_program(n, quartic_poly(n, seed), f"ball_pop(n={n},seed={seed})", ball=True)


def interval_pop(deg: int, seed: int = 0) -> SOSProgram:
    """min of a random univariate polynomial of even degree ``deg``
    (coefficients N(0,1), drawn from x^0 up) on [-1, 1]:
    max g s.t. p - g = s0 + (1 - x^2) s1, s0 with basis v_{deg/2}, s1 with
    basis v_{deg/2 - 1} (a weighted block, eq. (37))."""
    rng = np.random.default_rng(seed)
    p = {(k,): float(c) for k, c in enumerate(rng.standard_normal(deg + 1))}
    con = Constraint(degree=deg, g0=p, g=[{(0,): 1.0}],
                     blocks=[Block(deg // 2), Block(deg // 2 - 1, {(0,): 1.0, (2,): -1.0})])
    return SOSProgram(n=1, w=np.array([-1.0]), constraints=[con], name=f"interval_pop(deg={deg},seed={seed})",
                      meta={"p": p})


def matrix_poly(n: int, r: int, seed: int) -> List[List[Poly]]:
    """Symmetric r x r quartic matrix polynomial
    P(x) = (sum x_i^2)^2 I_r + sum_{|a|<=3} C_a x^a, the entries of C_a ~ N(0,1)
    drawn for i <= j (pairs row-major), then a in graded order."""
    rng = np.random.default_rng(seed)
    s = sq_norm(n)
    lead = pmul(s, s)
    P: List[List[Poly]] = [[{} for _ in range(r)] for _ in range(r)]
    for i in range(r):
        for j in range(i, r):
            low = _random_low_part(n, rng)
            P[i][j] = padd(lead, low) if i == j else low
            P[j][i] = P[i][j]
    return P


def matrix_pop(n: int, r: int, seed: int = 0) -> SOSProgram:
    """Lower bound on min_x lambda_min(P(x)) for the matrix polynomial of
    ``matrix_poly``: max g s.t. P(x) - g I_r is an SOS matrix (Section V,
    eq. (47)-(48)) with the basis I_r (x) v_2(x); Y is r C(n+2,2) square."""
    P = matrix_poly(n, r, seed)
    eye = [[({_zero(n): 1.0} if i == j else {}) for j in range(r)] for i in range(r)]
    con = MatrixConstraint(r=r, degree=4, P0=P, P=[eye], block=Block(2))
    return SOSProgram(n=n, w=np.array([-1.0]), constraints=[con], name=f"matrix_pop(n={n},r={r},seed={seed})",
                      meta={"P": P})


def paper_pop_poly(n: int) -> Poly:
    """Objective of eq. (46): sum_{i<j} (x_i x_j + x_i^2 x_j - x_j^3 - x_i^2 x_j^2)."""
    p: Poly = {}
    for j in range(n):
        for i in range(j):
            for e, c in (
                (tuple(a + b for a, b in zip(_unit(n, i), _unit(n, j))), 1.0),
                (tuple(a + b for a, b in zip(_unit(n, i, 2), _unit(n, j))), 1.0),
                (_unit(n, j, 3), -1.0),
                (tuple(a + b for a, b in zip(_unit(n, i, 2), _unit(n, j, 2))), -1.0),
            ):
                p[e] = p.get(e, 0.0) + c
    return {e: c for e, c in p.items() if c != 0.0}


def paper_pop(n: int) -> SOSProgram:
    """Constrained POP of eq. (46) on the unit ball, order 2d = 4."""
    return _pop_program(n, paper_pop_poly(n), f"paper_pop(n={n})", ball=True)


def univariate_pop(degree: int, seed: int) -> SOSProgram:
    """p(x) = x^degree + sum_{k<degree} c_k x^k, c_k ~ N(0,1); degree even."""
    assert degree % 2 == 0
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal(degree)
    p: Poly = {(degree,): 1.0}
    for k in range(degree):
        p[(k,)] = float(coef[k])
    con = Constraint(degree=degree, g0=p, g=[{(0,): 1.0}], blocks=[Block(degree // 2)])
    return SOSProgram(n=1, w=np.array([-1.0]), constraints=[con], name=f"univariate(deg={degree},seed={seed})",
                      meta={"p": p})


def hurwitz_matrix(n: int, seed: int) -> np.ndarray:
    """Random A with spectral abscissa <= -0.5 (shifted Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) / np.sqrt(n)
    shift = np.max(np.linalg.eigvals(a).real) + 0.5
    return a - shift * np.eye(n)


def lyapunov_linear(n: int, seed: int, eps: float = 1e-3) -> SOSProgram:
    """min trace(P) s.t. V - eps|x|^2 SOS and -grad V . (A x) - x^T x SOS,
    V(x) = x^T P x.  Decision variables: P_ij, i <= j (t = n(n+1)/2).

    The constraints read P - eps I >= 0 and -(A^T P + P A) - I >= 0, so the
    optimum is the Lyapunov solution of A^T P + P A + I = 0 when it is
    >= eps I."""
    A = hurwitz_matrix(n, seed)
    pairs = [(i, j) for j in range(n) for i in range(j + 1)]
    # V = sum_{i<=j} P_ij m_ij(x) with m_ii = x_i^2, m_ij = 2 x_i x_j
    mons: List[Poly] = []
    for (i, j) in pairs:
        e = tuple(a + b for a, b in zip(_unit(n, i), _unit(n, j)))
        mons.append({e: 1.0 if i == j else 2.0})
    fx = [{_unit(n, k): float(A[r, k]) for k in range(n) if A[r, k] != 0.0} for r in range(n)]
    w = np.array([1.0 if i == j else 0.0 for (i, j) in pairs])
    # s1 = V - eps|x|^2 = g0 - sum u_i g_i with g_i = -m_i
    c1 = Constraint(degree=2, g0=sq_norm(n, -eps), g=[{e: -c for e, c in m.items()} for m in mons],
                    blocks=[Block(1, min_degree=1)], min_degree=2)
    # s2 = -grad V . f - |x|^2 = g0 - sum u_i g_i with g_i = grad m_i . f
    g2 = []
    for m in mons:
        gi: Poly = {}
        for r in range(n):
            gi = padd(gi, pmul(pdiff(m, r), fx[r]))
        g2.append(gi)
    c2 = Constraint(degree=2, g0=sq_norm(n, -1.0), g=g2, blocks=[Block(1)])
    return SOSProgram(n=n, w=w, constraints=[c1, c2], name=f"lyapunov_linear(n={n},seed={seed})",
                      meta={"A": A, "pairs": pairs, "eps": eps})


def lyapunov_cubic(n: int, seed: int, eps: float = 1e-3, sigma: float = 0.1) -> SOSProgram:
    """Global Lyapunov search for x' = f(x) = -x + cubic(x).

    Each component of f gets every cubic monomial with a N(0, sigma^2)
    coefficient.  V = sum_i u_i m_i over the monomials of degree 2..4 and
    feasibility (w = 0) of

        V - eps |x|^2 SOS (degree 4, basis degree 2),
        -grad V . f - eps |x|^2 SOS (degree 6, basis degree 3).

    The g polynomials of the second identity, grad m_i . f, are built with
    array arithmetic (exponents packed base 16) and handed over as term
    arrays."""
    rng = np.random.default_rng(seed)
    cubic = np.array(_support(n, 3, 3), dtype=np.int64)
    fcoef = np.stack([sigma * rng.standard_normal(len(cubic)) for _ in range(n)])  # [n, K]
    vmons = _support(n, 4, 2)
    V = np.array(vmons, dtype=np.int64)  # [t, n]
    t = len(vmons)
    base = 16 ** np.arange(n, dtype=np.int64)
    # f_r terms: cubic monomials plus -x_r
    idx_l, key_l, coef_l = [], [], []
    eye = np.eye(n, dtype=np.int64)
    for r in range(n):
        a_r = V[:, r]  # d m_i / d x_r = a_r x^(a - e_r)
        sel = np.nonzero(a_r > 0)[0]
        if len(sel) == 0:
            continue
        dexp = V[sel] - eye[r]  # [s, n]
        fe = np.concatenate([cubic, eye[r:r + 1]])  # [K+1, n]
        fc = np.concatenate([fcoef[r], [-1.0]])
        ex = dexp[:, None, :] + fe[None, :, :]  # [s, K+1, n]
        co = a_r[sel][:, None] * fc[None, :]
        idx_l.append(np.repeat(sel, fe.shape[0]))
        key_l.append((ex.reshape(-1, n) * base).sum(axis=1))
        coef_l.append(co.reshape(-1))
    idx = np.concatenate(idx_l)
    key = np.concatenate(key_l)
    coef = np.concatenate(coef_l)
    comb = idx * (16 ** n) + key
    uniq, inv = np.unique(comb, return_inverse=True)
    csum = np.bincount(inv, weights=coef)
    keep = csum != 0.0
    uniq, csum = uniq[keep], csum[keep]
    gi = uniq // (16 ** n)
    gk = uniq % (16 ** n)
    gexp = (gk[:, None] // base[None, :]) % 16
    c1 = Constraint(degree=4, g0=sq_norm(n, -eps), g=[{m: -1.0} for m in vmons], blocks=[Block(2)])
    c2 = Constraint(degree=6, g0=sq_norm(n, -eps), blocks=[Block(3)],
                    term_arrays=(t, gi.astype(np.int64), gexp.astype(np.int32), csum))
    fx = [dict(zip(map(tuple, np.concatenate([cubic, eye[r:r + 1]]).tolist()),
                   np.concatenate([fcoef[r], [-1.0]]).tolist())) for r in range(n)]
    return SOSProgram(n=n, w=np.zeros(t), constraints=[c1, c2],
                      name=f"lyapunov_cubic(n={n},seed={seed})", meta={"f": fx})


def lyapunov_local(n: int, seed: int, r2: float = 0.1, eps: float = 1e-3, sigma: float = 1.0,
                   cubic_terms: int = 0) -> SOSProgram:
    """Local stability of x' = f(x) = A x + cubic(x) (A Hurwitz) in the ball
    |x|^2 <= r2 with a quadratic V(x) = x^T P x, by the Positivstellensatz:

        min trace(P)  s.t.  V - eps |x|^2 SOS                       (degree 2)
                            -grad V . f - |x|^2 = s0(x) + s1(x) (r2 - |x|^2)
                            s0 SOS, s1 SOS.

    Every polynomial here vanishes to second order at the origin (f(0) = 0,
    V quadratic), so the bases leave out the constant: s0 on the monomials of
    degree 1..2 (N = C(n+2,2) - 1), s1 and the Gram form of V - eps|x|^2 on
    x_1..x_n, and coefficients are matched on the monomials of degree >= 2.
    With the constant kept, its row would force a zero row and column in the
    Gram matrices of s0 and s1, and the SDP would have no strictly feasible
    point.  The low-rank width (the P entries plus the s1 Gram entries) is
    then n(n+1), the size of the factorized matrix in Table III.

    Each component of f gets ``cubic_terms`` (default n) random cubic
    monomials with N(0, sigma^2) coefficients.  Decision variables: P_ij,
    i <= j.  With sigma = 0 the multiplier vanishes at the optimum and P
    solves A^T P + P A + I = 0 (when P >= eps I)."""
    A = hurwitz_matrix(n, seed)
    rng = np.random.default_rng(seed + 1)
    cub = _support(n, 3, 3)
    k = cubic_terms if cubic_terms > 0 else n
    fx: List[Poly] = []
    for r in range(n):
        fr: Poly = {_unit(n, q): float(A[r, q]) for q in range(n) if A[r, q] != 0.0}
        if sigma > 0.0:
            for idx in rng.choice(len(cub), size=min(k, len(cub)), replace=False):
                e = tuple(cub[idx])
                fr[e] = fr.get(e, 0.0) + sigma * float(rng.standard_normal())
        fx.append(fr)
    pairs = [(i, j) for j in range(n) for i in range(j + 1)]
    mons: List[Poly] = []
    for (i, j) in pairs:
        e = tuple(a + b for a, b in zip(_unit(n, i), _unit(n, j)))
        mons.append({e: 1.0 if i == j else 2.0})
    w = np.array([1.0 if i == j else 0.0 for (i, j) in pairs])
    c1 = Constraint(degree=2, g0=sq_norm(n, -eps), g=[{e: -c for e, c in m.items()} for m in mons],
                    blocks=[Block(1, min_degree=1)], min_degree=2)
    g2 = []
    for m in mons:
        gi: Poly = {}
        for r in range(n):
            gi = padd(gi, pmul(pdiff(m, r), fx[r]))
        g2.append(gi)
    ball = padd({_zero(n): r2}, sq_norm(n, -1.0))
    c2 = Constraint(degree=4, g0=sq_norm(n, -1.0), g=g2,
                    blocks=[Block(2, min_degree=1), Block(1, ball, min_degree=1)], min_degree=2)
    return SOSProgram(n=n, w=w, constraints=[c1, c2], name=f"lyapunov_local(n={n},seed={seed})",
                      meta={"A": A, "pairs": pairs, "eps": eps, "r2": r2})


def lyapunov_batch(count: int, seed: int = 0, n_min: int = 2, n_max: int = 6) -> List[SOSProgram]:
    """``count`` cubic Lyapunov searches with n ~ U{n_min..n_max}."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_min, n_max + 1, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [lyapunov_cubic(int(n), int(s)) for n, s in zip(ns, seeds)]


class ParametricPOP:
    """p(theta) = p0 + sum_{k=1..K} theta_k q_k on monomials of degree <= 3
    (p0 also carries (sum x_i^2)^2 so every member is coercive)."""

    def __init__(self, n: int = 10, K: int = 16, seed: int = 0):
        self.n, self.K = n, K
        self.p0 = quartic_poly(n, seed)
        self.q = []
        for k in range(1, K + 1):
            self.q.append(_random_low_part(n, np.random.default_rng(seed + k)))

    def poly(self, theta: np.ndarray) -> Poly:
        return padd(self.p0, *self.q, scale=[1.0] + [float(x) for x in theta])

    def program(self, theta: np.ndarray) -> SOSProgram:
        return _pop_program(self.n, self.poly(theta), f"parametric_pop(n={self.n})", ball=False)

    def programs(self, thetas: np.ndarray) -> List[SOSProgram]:
        """Programs for many parameter vectors at once: every member has the
        same support, so its coefficients are one row of [1, theta] C."""
        support = sorted(set(self.p0).union(*[set(q) for q in self.q]), key=lambda e: (sum(e), tuple(-x for x in e)))
        index = {e: i for i, e in enumerate(support)}
        Cm = np.zeros((len(support), 1 + self.K))
        for e, c in self.p0.items():
            Cm[index[e], 0] = c
        for k, q in enumerate(self.q):
            for e, c in q.items():
                Cm[index[e], 1 + k] = c
        coefs = np.hstack([np.ones((len(thetas), 1)), np.asarray(thetas, float)]) @ Cm.T
        exps = np.array(support, dtype=np.int32)
        z = _zero(self.n)
        out = []
        for i in range(len(thetas)):
            con = Constraint(degree=4, g=[{z: 1.0}], blocks=[Block(2)], g0_arrays=(exps, coefs[i]))
            out.append(SOSProgram(n=self.n, w=np.array([-1.0]), constraints=[con], name=f"parametric_pop(n={self.n})"))
        return out

    @staticmethod
    def thetas(count: int, seed: int, K: int = 16) -> np.ndarray:
        return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(count, K))
