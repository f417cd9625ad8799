"""The allocation-free projection entry point (sos_psd_project_noalloc).

It exists for callers that cannot call cudaMalloc -- e.g. code whose device
memory is owned by a pool it may not bypass, or a plugin whose host forbids
allocations after start-up.  It must give the same result as the allocating
entry point (sos_psd_project) on the same input, on consecutive calls that
share its fixed scratch array, on the shared-memory path, the tridiagonal
path and the grid path, agree with the oracle's eigen-clamp, and reject
sizes above its fixed maximum.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""

import os

import numpy as np
import pytest

from oracle.admm import proj_psd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1708_04174_gb300 import build, capi

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return torch, capi


def _pack(X):
    out = []
    for j in range(X.shape[0]):
        col = X[j:, j].copy()
        col[1:] *= np.sqrt(2.0)
        out.append(col)
    return np.concatenate(out)


def _sym(N, seed):
    a = np.random.default_rng(seed).standard_normal((N, N))
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("N", [7, 60, 96, 97, 200, 256])
def test_noalloc_matches_allocating_entry_point_twice(env, N):
    torch, capi = env
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share (and reuse) the scratch
        X = _sym(N, 1000 * N + call)
        w = torch.tensor(_pack(X), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(w)
        got = torch.empty_like(w)
        capi.psd_project(w.data_ptr(), ref.data_ptr(), N, stream)
        capi.psd_project_noalloc(w.data_ptr(), got.data_ptr(), N, stream)
        torch.cuda.synchronize()
        diff = (got - ref).abs().max().item()
        assert diff <= 1e-12 * max(1.0, float(np.abs(X).max())) * N, (call, diff)
        err = np.abs(got.cpu().numpy() - _pack(proj_psd(X))).max()
        assert err <= 1e-12 * max(1.0, float(np.abs(X).max())) * N, (call, err)
        assert torch.equal(w, torch.tensor(_pack(X), dtype=torch.float64, device="cuda"))  # input untouched


def test_noalloc_rejects_oversize(env):
    torch, capi = env
    N = capi.NOALLOC_MAX_N + 1
    w = torch.zeros(N * (N + 1) // 2, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="outside"):
        capi.psd_project_noalloc(w.data_ptr(), w.data_ptr(), N)
