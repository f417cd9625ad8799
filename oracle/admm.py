"""HSDE ADMM of eq. (20) with the paper's affine step (oracle; test
infrastructure only).  Everything is FP64.

Iteration k (eq. (20a-c)):

    u_hat = (I + Q)^{-1} (u + v)
    u     = P_C(u_hat - v)
    v     = v - u_hat + u

with u = (xi, y, tau), v = (z, s, kappa), Q the skew matrix of eq. (19) and
C = K x R^m x R_+.  The solve with I + Q follows Section IV step by step:

* eliminate u_hat_3 (eq. (23)-(24)) and apply Sherman-Morrison to the rank-one
  term zeta zeta^T, zeta = [c; -b] (eq. (25)); M^{-1} zeta is precomputed;
* solve with M = [I -A^T; A I] by eliminating sigma_1 (eq. (26)-(27)):
  sigma_1 = w1 + A^T sigma_2, (I + A A^T) sigma_2 = w2 - A w1;
* (I + A A^T) = P + A_L A_L^T with P diagonal (Prop. 1/3); invert it with the
  matrix inversion lemma and a cached Cholesky factor of I + A_L^T P^{-1} A_L
  (eq. (28) and the per-iteration recipe of the Appendix).

Readings where the paper is silent (each listed in the design notes):
start u0 = v0 = (0, 0, 1); no scaling, no over-relaxation; residuals and
termination as in ``residuals``; PSD projection by a symmetric eigensolver
with negative eigenvalues clamped to zero.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla

from .conic import ConicData

SOLVED, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE, MAX_ITER, NUMERICAL = 1, 2, 3, 4, 5


def proj_psd(S: np.ndarray) -> np.ndarray:
    """Projection of a symmetric matrix onto S_+: V max(Lambda, 0) V^T."""
    if not np.all(np.isfinite(S)):
        # IEEE propagation: a non-finite entry makes the whole projection
        # NaN, and the next residual check reports the iterate non-finite
        return np.full_like(S, np.nan)
    lam, V = np.linalg.eigh(S)
    return (V * np.maximum(lam, 0.0)) @ V.T


class HSDE:
    def __init__(self, cd: ConicData):
        self.cd = cd
        A = cd.A.tocsc()
        self.A = cd.A.tocsr()
        self.At = self.A.T.tocsr()
        m, nx = A.shape
        self.m, self.nx = m, nx
        self.b, self.c = cd.b.astype(float), cd.c.astype(float)

        # Prop. 1 / Prop. 3: every column of the orthogonal part has a single
        # nonzero, so A_D A_D^T is diagonal and P = I + A_D A_D^T.
        AD = A[:, cd.diag_cols]
        nnz_per_col = np.diff(AD.indptr)
        assert np.all(nnz_per_col == 1), "orthogonal part must have one nonzero per column"
        self.P = 1.0 + np.asarray(AD.multiply(AD).sum(axis=1)).ravel()

        # low-rank part (free u columns + weighted-block columns), dense
        self.AL = A[:, cd.lowrank_cols].toarray()
        tL = self.AL.shape[1]
        core = np.eye(tL) + self.AL.T @ (self.AL / self.P[:, None])  # eq. (28)
        self.L = np.linalg.cholesky(core)  # cached factor (Section IV, Appendix)

        # Sherman-Morrison data (eq. (25)): h = M^{-1} zeta, zeta = [c; -b]
        h1, h2 = self.solve_M(self.c.copy(), -self.b)
        self.h = np.concatenate([h1, h2])
        self.zeta = np.concatenate([self.c, -self.b])
        self.one_plus_zh = 1.0 + self.zeta @ self.h

    # ---- linear algebra of Section IV --------------------------------
    def solve_IAAt(self, r: np.ndarray) -> np.ndarray:
        """(I + A A^T)^{-1} r = (P + A_L A_L^T)^{-1} r via Woodbury (Appendix)."""
        x = r / self.P
        y = self.AL.T @ x
        # check_finite=False: a non-finite iterate propagates (IEEE) to the
        # residual check, which classifies it, instead of raising here
        z = sla.solve_triangular(self.L, y, lower=True, check_finite=False)
        z = sla.solve_triangular(self.L.T, z, lower=False, check_finite=False)
        return x - (self.AL @ z) / self.P

    def solve_M(self, w1: np.ndarray, w2: np.ndarray):
        """[I -A^T; A I] [s1; s2] = [w1; w2] (eq. (26)-(27))."""
        s2 = self.solve_IAAt(w2 - self.A @ w1)
        s1 = w1 + self.At @ s2
        return s1, s2

    def affine(self, omega: np.ndarray) -> np.ndarray:
        """u_hat = (I + Q)^{-1} omega (eq. (20a)) by eq. (23)-(25)."""
        nx, m = self.nx, self.m
        w1, w2, w3 = omega[:nx], omega[nx:nx + m], omega[nx + m]
        s1, s2 = self.solve_M(w1 - self.c * w3, w2 + self.b * w3)
        sig = np.concatenate([s1, s2])
        u12 = sig - self.h * ((self.zeta @ sig) / self.one_plus_zh)
        u3 = w3 + self.c @ u12[:nx] - self.b @ u12[nx:]
        return np.concatenate([u12, [u3]])

    # ---- cone projection (eq. (20b)) -------------------------------
    def proj_C(self, x: np.ndarray) -> np.ndarray:
        """P_C for C = R^t x S_+ x ... x R^m x R_+ (vec coordinates)."""
        out = x.copy()
        for blk in self.cd.blocks:
            N = blk.N
            sl = slice(blk.offset, blk.offset + N * N)
            X = x[sl].reshape(N, N, order="F")
            S = 0.5 * (X + X.T)  # nearest symmetric matrix, then PSD projection
            out[sl] = proj_psd(S).reshape(-1, order="F")
        out[-1] = max(x[-1], 0.0)
        return out

    # ---- iteration (eq. (20)) -------------------------------------
    def start(self):
        n = self.nx + self.m + 1
        u = np.zeros(n)
        v = np.zeros(n)
        u[-1] = 1.0
        v[-1] = 1.0
        return u, v

    def step(self, u: np.ndarray, v: np.ndarray):
        uh = self.affine(u + v)
        un = self.proj_C(uh - v)
        vn = v - uh + un
        return un, vn

    def run(self, iters: int, u=None, v=None):
        if u is None:
            u, v = self.start()
        for _ in range(iters):
            u, v = self.step(u, v)
        return u, v

    # ---- residuals and termination ----------------------------------
    def residuals(self, u: np.ndarray, v: np.ndarray) -> dict:
        """Normalised residuals of the iterate (xi, y, z) = (u_xi, u_y, v_z)/tau."""
        nx, m = self.nx, self.m
        tau, kappa = u[-1], v[-1]
        ux, uy, vz = u[:nx], u[nx:nx + m], v[:nx]
        out = {"tau": tau, "kappa": kappa}
        by = float(self.b @ uy)
        cx = float(self.c @ ux)
        out["pinf"] = np.linalg.norm(self.At @ uy + vz) / by if by > 0 else np.inf
        out["dinf"] = np.linalg.norm(self.A @ ux) / (-cx) if cx < 0 else np.inf
        if tau > 1e-12 * (kappa + 1.0):
            xi, y, z = ux / tau, uy / tau, vz / tau
            pobj, dobj = float(self.c @ xi), float(self.b @ y)
            out["rp"] = np.linalg.norm(self.A @ xi - self.b) / (1.0 + np.linalg.norm(self.b))
            out["rd"] = np.linalg.norm(self.At @ y + z - self.c) / (1.0 + np.linalg.norm(self.c))
            out["gap"] = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
            out["pobj"], out["dobj"] = pobj, dobj
            out["res"] = max(out["rp"], out["rd"], out["gap"])
        else:
            out["res"] = np.inf
        return out


@dataclass
class Result:
    status: int
    iters: int
    u: np.ndarray
    v: np.ndarray
    res: dict
    history: List[dict] = field(default_factory=list)


def solve(cd: ConicData, tol: float, max_iter: int, k_check: int = 1,
          u0: Optional[np.ndarray] = None, v0: Optional[np.ndarray] = None,
          solver: Optional[HSDE] = None, infeas_tol: float = 1e-7) -> Result:
    """Iterate eq. (20) until max(rp, rd, gap) <= tol or an infeasibility
    certificate holds to ``infeas_tol``, checking every ``k_check``
    iterations."""
    hs = solver or HSDE(cd)
    u, v = (u0.copy(), v0.copy()) if u0 is not None else hs.start()
    hist: List[dict] = []
    res: dict = {}
    for k in range(1, max_iter + 1):
        u, v = hs.step(u, v)
        if k % k_check and k != max_iter:
            continue
        res = hs.residuals(u, v)
        res["iter"] = k
        hist.append(res)
        if not np.all(np.isfinite(u)) or not np.all(np.isfinite(v)):
            return Result(NUMERICAL, k, u, v, res, hist)
        if res["res"] <= tol:
            return Result(SOLVED, k, u, v, res, hist)
        # A nonzero solution of the embedding with tau > 0 yields an optimal
        # pair and one with kappa > 0 a certificate (the classification stated
        # with eq. (18)-(19)); the certificate tests are taken only while the
        # iterate leans towards the second case, and to their own tolerance:
        # a feasible program with b^T y* >= |c| / tol passes the primal test
        # at the residual tolerance, near its optimum or early on.
        if res["kappa"] > res["tau"]:
            if res["pinf"] <= infeas_tol:
                return Result(PRIMAL_INFEASIBLE, k, u, v, res, hist)
            if res["dinf"] <= infeas_tol:
                return Result(DUAL_INFEASIBLE, k, u, v, res, hist)
    return Result(MAX_ITER, max_iter, u, v, res, hist)
