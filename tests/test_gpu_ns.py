"""GPU tests of the Newton-Schulz PSD projection on the tensor cores
(tcgen05, BF16 three-part split operands, FP32 accumulation), used for large
Gram blocks in the FP32-projection forms: the mixed form with it reaches the
oracle's objective within the error its tolerance allows."""

import os

import numpy as np
import pytest

from instances import workloads as W
from oracle import admm, conic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1708_04174_gb300 import build, capi as c

    if not os.path.exists(c.LIB_PATH):
        build.build()
    return c


@pytest.mark.parametrize("name,make", [("quartic_n15_N136", lambda: W.quartic_pop(15, 0)),
                                       ("config1_ball_n20_N231", lambda: W.ball_pop(20, 0))])
def test_ns_mixed_form_objective(capi, name, make):
    prog = make()
    ro = admm.solve(conic.build(prog), 1e-7, 50000, k_check=10)
    s = capi.Solver(prog, precision=capi.PREC_MIXED, k_check=10, large_method=2)
    r = s.solve(1e-4, 20000)[0]
    st = s.stats()
    s.close()
    assert r["status"] == capi.SOLVED, r
    err = abs(r["obj_primal"] - ro.res["pobj"]) / abs(ro.res["pobj"])
    assert err < 1e-3, err
    assert 5 <= st["max_sweeps"] < 60, st  # Newton-Schulz iterations of the last projection


def test_ns_iterates_track_oracle(capi):
    """40 iterations with the tensor-core projection stay within 1e-4 of the
    FP64 oracle's iterates (relative, max-norm)."""
    prog = W.quartic_pop(15, 0)
    cd = conic.build(prog)
    u, v = admm.HSDE(cd).run(40)
    uo = np.concatenate([conic.vec_to_packed(cd, u[:cd.nx]), u[cd.nx:]])
    s = capi.Solver(prog, precision=capi.PREC_MIXED, large_method=2)
    s.iterate(40)
    s.sync()
    ug, _ = s.get_iterate()
    s.close()
    assert np.abs(ug - uo).max() / np.abs(uo).max() < 1e-4


def _pack(X):
    out = []
    for j in range(X.shape[0]):
        col = X[j:, j].copy()
        col[1:] *= np.sqrt(2.0)
        out.append(col)
    return np.concatenate(out)


def _project_ns(capi, X):
    import torch

    w = torch.tensor(_pack(X), dtype=torch.float64, device="cuda")
    u = torch.empty_like(w)
    capi.psd_project_mixed(w.data_ptr(), u.data_ptr(), X.shape[0], torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return u.cpu().numpy()


# The bound, element by element: every product of the iteration carries the
# rounding of FP32 accumulation over N terms of three-part BF16 operands
# (24 significant bits, as FP32), i.e. about u32 sqrt(N) |W|_2 per entry with
# u32 = 2^-24; the bound allows four such terms (the split, the accumulation,
# the iteration's propagation of both, the closing product (W + W S) / 2).
# Measured on GB300: max |error| <= 3.3e-7 |W|_2 for N <= 496, 16x inside.
U32 = 2.0 ** -24


def _ns_bound(X):
    return 4.0 * U32 * np.sqrt(X.shape[0]) * np.linalg.norm(X, 2)


@pytest.mark.parametrize("N", [136, 231, 300, 496])
def test_ns_projection_elementwise(capi, N):
    from oracle.admm import proj_psd

    a = np.random.default_rng(N).standard_normal((N, N))
    X = 0.5 * (a + a.T)
    err = np.abs(_project_ns(capi, X) - _pack(proj_psd(X))).max()
    assert err <= _ns_bound(X), (err, _ns_bound(X))


@pytest.mark.parametrize("N", [231, 496])
def test_ns_projection_admm_like_spectrum(capi, N):
    """Many positive eigenvalues over four decades, a fifth of them negative,
    a cluster at +-1e-6 and a repeated eigenvalue."""
    from oracle.admm import proj_psd

    rng = np.random.default_rng(7 * N)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = np.exp(rng.uniform(np.log(1e-4), 0.0, N))
    lam[: N // 5] *= -1.0
    lam[N // 5: N // 5 + 3] = 1e-6
    lam[N // 5 + 3: N // 5 + 6] = -1e-6
    lam[-2:] = 0.5
    X = (Q * lam) @ Q.T
    X = 0.5 * (X + X.T)
    err = np.abs(_project_ns(capi, X) - _pack(proj_psd(X))).max()
    assert err <= _ns_bound(X), (err, _ns_bound(X))


def test_ns_config2_objective_against_stored_oracle(capi):
    """The precision form's own workload (unconstrained quartic POP n = 30,
    Gram 496): the mixed form solved to 1e-4 reaches the optimal value that
    the FP64 oracle reaches at 1e-7 (tests/golden/quartic_pop_n30_objective.txt,
    written by make_quartic_pop_n30_objective.py) within 1e-3 relative."""
    path = os.path.join(os.path.dirname(__file__), "golden", "quartic_pop_n30_objective.txt")
    ref = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        ref[k] = float(v)
    assert int(ref["status"]) == admm.SOLVED
    s = capi.Solver(W.quartic_pop(30, 0), precision=capi.PREC_MIXED, k_check=10)
    r = s.solve(1e-4, 20000, want_solution=False)[0]
    s.close()
    assert r["status"] == capi.SOLVED, r
    err = abs(r["obj_primal"] - ref["pobj"]) / abs(ref["pobj"])
    assert err < 1e-3, err
