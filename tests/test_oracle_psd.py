"""Pins of the oracle's PSD projection (eq. (20b)) against properties that
characterise the Euclidean projection onto S_+."""

import numpy as np
import pytest

from oracle.admm import proj_psd


def _rand_sym(n, seed):
    a = np.random.default_rng(seed).standard_normal((n, n))
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (28, 3), (60, 4)])
def test_projection_characterisation(n, seed):
    Y = _rand_sym(n, seed)
    P = proj_psd(Y)
    R = Y - P
    tol = 1e-12 * max(1.0, np.abs(Y).max()) * n
    assert np.allclose(P, P.T, atol=tol)
    assert np.linalg.eigvalsh(P).min() >= -tol  # P(Y) is PSD
    assert np.linalg.eigvalsh(R).max() <= tol  # Y - P(Y) is NSD
    assert abs(np.sum(P * R)) <= tol * n  # complementarity <P, Y - P> = 0
    assert np.allclose(proj_psd(P), P, atol=tol)  # idempotent


def test_projection_2x2_closed_form():
    a, b, c = 0.7, -1.3, -0.4
    Y = np.array([[a, b], [b, c]])
    mid, rad = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
    lp = mid + rad  # the only positive eigenvalue here
    assert mid - rad < 0 < lp
    v = np.array([b, lp - a])
    v /= np.linalg.norm(v)
    assert np.allclose(proj_psd(Y), lp * np.outer(v, v), atol=1e-14)


def test_projection_diagonal_clamps():
    d = np.array([3.0, -1.0, 0.0, 2.5, -7.0])
    assert np.array_equal(proj_psd(np.diag(d)), np.diag(np.maximum(d, 0)))
