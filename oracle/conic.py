"""SOS program -> conic program data (oracle; test infrastructure only).

Follows the paper's construction literally, with full ``vec`` Gram columns:

* Coefficient matching (eq. (11)-(12)): for every monomial x^alpha of a
  constraint's row set, <B_alpha, X> + sum_i u_i g_{i,alpha} = g_{0,alpha}.
* B_alpha is the 0/1 indicator of the entries (beta, gamma) of v_d v_d^T with
  beta + gamma = alpha (eq. (8)).
* A = [A1 A2], b = g_0 coefficients, c = [w; 0], xi = [u; vec X],
  K = R^t x S_+ (eq. (14)-(16)); vec stacks columns (Section III).
* Several SOS constraints each own their rows and Gram blocks (eq. (7), remark
  after eq. (13)); a weighted block p(x) v v^T contributes the coefficients of
  p(x) x^(beta+gamma) (Section VI, eq. (38)-(40)).
* A matrix-valued constraint (Section V) has one row per triple
  (alpha, i, j): <E_i^T Y E_j, B_alpha> = (C_alpha)_ij (eq. (49)-(50)), Y of
  size r N.  Y is symmetric, so the triples (alpha, i, j) and (alpha, j, i)
  state one equation; the row is kept once, for i <= j, and for i < j it
  collects both blocks Y_ij and Y_ji, with right side 2 (C_alpha)_ij.

Column classes (Prop. 1 and Prop. 3): columns of unweighted Gram blocks form
the orthogonal part (each has exactly one nonzero, so its rows' products are
diagonal); the free u columns and the weighted-block columns form the
low-rank part handled by the matrix inversion lemma (Section IV, Section VI).
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from instances.program import MatrixConstraint

from . import basis

Exp = Tuple[int, ...]


@dataclass
class BlockInfo:
    offset: int  # first column of vec(X_b) in xi
    N: int
    weighted: bool
    constraint: int
    basis: List[Exp]


@dataclass
class ConicData:
    A: sp.csr_matrix  # m x (t + sum N_b^2)
    b: np.ndarray
    c: np.ndarray
    t: int
    blocks: List[BlockInfo]
    row_offsets: List[int]  # first row of each constraint
    rows: List[List[Exp]]  # row monomials per constraint
    lowrank_cols: np.ndarray
    diag_cols: np.ndarray

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def nx(self) -> int:
        return self.A.shape[1]


def _add(e1: Exp, e2: Exp) -> Exp:
    return tuple(a + b for a, b in zip(e1, e2))


def build(prog) -> ConicData:
    """Conic data of eq. (14)-(15) for an ``instances.SOSProgram``."""
    n, t = prog.n, prog.t
    rows: List[List[Exp]] = []
    row_index: List[Dict[Exp, int]] = []
    row_offsets: List[int] = []
    m = 0
    for con in prog.constraints:
        if isinstance(con, MatrixConstraint):
            al = basis.monomials_range(n, con.min_degree, con.degree)
            r = [(a, i, j) for i in range(con.r) for j in range(i, con.r) for a in al]
        else:
            r = basis.monomials_range(n, getattr(con, "min_degree", 0), con.degree)
        rows.append(r)
        row_index.append({e: m + k for k, e in enumerate(r)})
        row_offsets.append(m)
        m += len(r)

    I: List[int] = []
    J: List[int] = []
    V: List[float] = []
    b = np.zeros(m)
    for j, con in enumerate(prog.constraints):
        if isinstance(con, MatrixConstraint):
            assert len(con.P) == t
            for (i1, i2) in con.pairs:
                sym = 1.0 if i1 == i2 else 2.0  # (C_alpha)_ij + (C_alpha)_ji
                for e, coef in con.P0[i1][i2].items():
                    b[row_index[j][(e, i1, i2)]] += sym * coef
                for h, Ph in enumerate(con.P):
                    for e, coef in Ph[i1][i2].items():
                        I.append(row_index[j][(e, i1, i2)])
                        J.append(h)
                        V.append(sym * coef)
            continue
        for e, coef in con.g0.items():
            b[row_index[j][e]] += coef
        assert len(con.g) == t
        for i, gi in enumerate(con.g):
            for e, coef in gi.items():
                I.append(row_index[j][e])
                J.append(i)
                V.append(coef)

    blocks: List[BlockInfo] = []
    col = t
    lowrank = list(range(t))
    diag: List[int] = []
    for j, con in enumerate(prog.constraints):
        if isinstance(con, MatrixConstraint):
            bas = basis.monomials_range(n, con.block.min_degree, con.block.basis_degree)
            N = len(bas)
            L = con.r * N
            blocks.append(BlockInfo(col, L, False, j, [(i, e) for i in range(con.r) for e in bas]))
            for kk in range(L):
                bk, ek = divmod(kk, N)  # block column, basis monomial
                for ii in range(L):
                    bi, ei = divmod(ii, N)
                    cidx = col + ii + kk * L
                    I.append(row_index[j][(_add(bas[ei], bas[ek]), min(bi, bk), max(bi, bk))])
                    J.append(cidx)
                    V.append(1.0)
                    diag.append(cidx)
            col += L * L
            continue
        for blk in con.blocks:
            bas = basis.monomials_range(n, getattr(blk, "min_degree", 0), blk.basis_degree)
            N = len(bas)
            weighted = blk.weight is not None
            blocks.append(BlockInfo(col, N, weighted, j, bas))
            for kk in range(N):  # column index of X
                for ii in range(N):  # row index of X; vec position ii + kk*N
                    cidx = col + ii + kk * N
                    a = _add(bas[ii], bas[kk])
                    if not weighted:
                        I.append(row_index[j][a])
                        J.append(cidx)
                        V.append(1.0)
                    else:
                        for dlt, pd in blk.weight.items():
                            I.append(row_index[j][_add(a, dlt)])
                            J.append(cidx)
                            V.append(pd)
                    (lowrank if weighted else diag).append(cidx)
            col += N * N

    A = sp.coo_matrix((V, (I, J)), shape=(m, col)).tocsr()
    A.sum_duplicates()
    c = np.zeros(col)
    c[:t] = prog.w
    return ConicData(A=A, b=b, c=c, t=t, blocks=blocks, row_offsets=row_offsets, rows=rows,
                     lowrank_cols=np.array(lowrank, dtype=np.int64), diag_cols=np.array(diag, dtype=np.int64))


# --------------------------------------------------------------------------
# packed (isometric svec) view of xi, used to compare with packed iterates
# --------------------------------------------------------------------------
# Packed order: free u first, then each block's lower triangle column by
# column (column j holds rows j..N-1); off-diagonal entries carry sqrt(2) so
# the map is an isometry between symmetric matrices and R^{N(N+1)/2}.

def packed_length(cd: ConicData) -> int:
    return cd.t + sum(b.N * (b.N + 1) // 2 for b in cd.blocks)


def vec_to_packed(cd: ConicData, x: np.ndarray) -> np.ndarray:
    out = [x[: cd.t]]
    r2 = np.sqrt(2.0)
    for blk in cd.blocks:
        X = x[blk.offset: blk.offset + blk.N * blk.N].reshape(blk.N, blk.N, order="F")
        X = 0.5 * (X + X.T)
        for j in range(blk.N):
            col = X[j:, j].copy()
            col[1:] *= r2
            out.append(col)
    return np.concatenate(out)


def packed_to_vec(cd: ConicData, xp: np.ndarray) -> np.ndarray:
    x = np.zeros(cd.nx)
    x[: cd.t] = xp[: cd.t]
    pos = cd.t
    r2 = np.sqrt(2.0)
    for blk in cd.blocks:
        N = blk.N
        X = np.zeros((N, N))
        for j in range(N):
            col = xp[pos: pos + N - j].copy()
            pos += N - j
            col[1:] /= r2
            X[j:, j] = col
            X[j, j:] = col
        x[blk.offset: blk.offset + N * N] = X.reshape(-1, order="F")
    return x
