"""Pins of the oracle's affine step (eq. (20a) through eq. (23)-(28)) against
dense linear algebra that does not use the paper's eliminations."""

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic, dense

TINY = [
    lambda: W.univariate_pop(4, 0),
    lambda: W.quartic_pop(2, 3),
    lambda: W.ball_pop(2, 1),
    lambda: W.lyapunov_linear(2, 0),
    lambda: W.lyapunov_cubic(2, 5),
]


@pytest.mark.parametrize("make", TINY)
def test_woodbury_matches_dense_inverse(make):
    cd = conic.build(make())
    hs = admm.HSDE(cd)
    A = cd.A.toarray()
    M = np.eye(cd.m) + A @ A.T
    r = np.random.default_rng(1).standard_normal(cd.m)
    ref = np.linalg.solve(M, r)
    got = hs.solve_IAAt(r)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("make", TINY)
def test_affine_step_matches_dense_lu(make):
    cd = conic.build(make())
    hs = admm.HSDE(cd)
    Q = dense.Q_matrix(cd)
    assert np.array_equal(Q, -Q.T)  # eq. (19): Q is skew
    rng = np.random.default_rng(2)
    for _ in range(3):
        om = rng.standard_normal(Q.shape[0])
        ref = np.linalg.solve(np.eye(Q.shape[0]) + Q, om)
        got = hs.affine(om)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-11 * np.abs(ref).max())


def test_affine_step_residual_midsize():
    cd = conic.build(W.ball_pop(4, 0))
    hs = admm.HSDE(cd)
    om = np.random.default_rng(3).standard_normal(hs.nx + hs.m + 1)
    u = hs.affine(om)
    nx, m = hs.nx, hs.m
    xi, y, tau = u[:nx], u[nx:nx + m], u[-1]
    Qu = np.concatenate([-(cd.A.T @ y) + cd.c * tau, cd.A @ xi - cd.b * tau,
                         [-(cd.c @ xi) + cd.b @ y]])
    assert np.linalg.norm(u + Qu - om) <= 1e-12 * np.linalg.norm(om)
