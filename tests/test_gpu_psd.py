"""GPU parity of the PSD-cone projection kernels (the Gram-block part of
eq. (20b)) through sos_psd_project, against the oracle's eigen-clamp, on
random and degenerate symmetric matrices.  Sizes cover the shared-memory
path (N <= 96) and the grid path (N > 96), odd and even N, and a ragged
16-wide tile tail."""

import numpy as np
import pytest

from oracle.admm import proj_psd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import os

    import torch

    from paper_1708_04174_gb300 import build, capi

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return torch, capi


def pack(X):
    N = X.shape[0]
    out = []
    for j in range(N):
        col = X[j:, j].copy()
        col[1:] *= np.sqrt(2.0)
        out.append(col)
    return np.concatenate(out)


def project_gpu(env, X):
    torch, capi = env
    w = torch.tensor(pack(X), dtype=torch.float64, device="cuda")
    u = torch.empty_like(w)
    capi.psd_project(w.data_ptr(), u.data_ptr(), X.shape[0], torch.cuda.current_stream().cuda_stream)
    return u.cpu().numpy()


def sym(N, seed, scale=1.0):
    a = np.random.default_rng(seed).standard_normal((N, N)) * scale
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 16, 17, 28, 33, 64, 84, 96, 97, 130, 231])
def test_projection_matches_eigh(env, N):
    X = sym(N, N)
    got = project_gpu(env, X)
    want = pack(proj_psd(X))
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(X).max()) * N


@pytest.mark.parametrize("N", [5, 40, 120])
def test_projection_degenerate_inputs(env, N):
    rng = np.random.default_rng(N)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = np.zeros(N)
    lam[: N // 3] = rng.uniform(0.5, 2.0, N // 3)  # PSD, rank deficient
    lam[N // 3: N // 2] = -rng.uniform(0.5, 2.0, N // 2 - N // 3)
    lam[N // 2: N // 2 + 2] = 1.0  # repeated eigenvalue
    X = (Q * lam) @ Q.T
    X = 0.5 * (X + X.T)
    tol = 1e-12 * N
    assert np.abs(project_gpu(env, X) - pack(proj_psd(X))).max() <= tol
    P = proj_psd(X)
    assert np.abs(project_gpu(env, P) - pack(P)).max() <= tol  # PSD input is a fixed point
    assert np.abs(project_gpu(env, -P)).max() <= tol  # NSD input maps to 0
    assert np.abs(project_gpu(env, np.zeros((N, N)))).max() == 0.0


def test_projection_rejects_bad_size(env):
    torch, capi = env
    w = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        capi.psd_project(w.data_ptr(), w.data_ptr(), 0)


# ---- mixed form: FP32 Jacobi + FP64-summed refinement (sos_psd_project_mixed) ----
# The bound: the refined result carries the rounding of an FP32 product
# V' M V'^T and of V' itself, a few units of 2^-24 |W|_F per entry, so
# |error|_F <= 1e-6 |W|_F; the unrefined FP32 Jacobi misses it by ~10x
# (orthogonality loss of ~1e-5 after hundreds of rotations per column).

def project_gpu_mixed(env, X):
    torch, capi = env
    w = torch.tensor(pack(X), dtype=torch.float64, device="cuda")
    u = torch.empty_like(w)
    capi.psd_project_mixed(w.data_ptr(), u.data_ptr(), X.shape[0], torch.cuda.current_stream().cuda_stream)
    return u.cpu().numpy()


@pytest.mark.parametrize("N", [1, 2, 3, 7, 16, 17, 28, 33, 64, 66, 84, 96, 97, 112])
def test_mixed_projection_accuracy(env, N):
    X = sym(N, 1000 + N)
    got = project_gpu_mixed(env, X)
    want = pack(proj_psd(X))
    assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(pack(X))


@pytest.mark.parametrize("N", [40, 66, 112])
def test_mixed_projection_admm_like_spectrum(env, N):
    # the spectrum ADMM meets near a solution: many positive eigenvalues
    # spread over decades, a few negative ones, clusters at +-1e-6 on both
    # sides of zero, and one repeated eigenvalue
    rng = np.random.default_rng(N)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = np.exp(rng.uniform(np.log(1e-4), 0.0, N))
    lam[: N // 5] *= -1.0
    lam[N // 5: N // 5 + 3] = 1e-6
    lam[N // 5 + 3: N // 5 + 6] = -1e-6
    lam[-2:] = 0.5
    X = (Q * lam) @ Q.T
    X = 0.5 * (X + X.T)
    got = project_gpu_mixed(env, X)
    want = pack(proj_psd(X))
    assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(pack(X))
    P = proj_psd(X)
    assert np.linalg.norm(project_gpu_mixed(env, P) - pack(P)) <= 1e-6 * np.linalg.norm(pack(P))
    assert np.abs(project_gpu_mixed(env, np.zeros((N, N)))).max() == 0.0


def test_mixed_projection_rejects_oversize_block(env):
    # above MIXED_MAX_N the Newton-Schulz kernel takes the block; it needs
    # one CTA per 128 x 64 lower tile of the padded matrix, all resident, so
    # an N whose tiles outnumber the SMs is refused before any allocation
    torch, capi = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nti = 1
    while (nti + 1) * (nti + 2) <= sms:
        nti += 1
    N = 128 * nti + 1  # nti + 1 row tiles: (nti + 1)(nti + 2) CTAs > sms
    w = torch.zeros(N * (N + 1) // 2, dtype=torch.float64, device="cuda")
    u = torch.empty_like(w)
    with pytest.raises(RuntimeError, match="unsupported|SMs|UNSUPPORTED"):
        capi.psd_project_mixed(w.data_ptr(), u.data_ptr(), N)


@pytest.mark.parametrize("N", [40, 84, 97, 231])
def test_fp64_projection_admm_like_spectrum(env, N):
    # FP64 Jacobi sweeps stop below 1e-10 |W|_F and the reconstruction adds
    # the first-order correction for what is left: the error is second order
    # (|E|^2 / gap) and never above |E|, so within 2e-10 |W|_F even for
    # clusters straddling zero; small (N <= 96) and grid (N > 96) paths
    rng = np.random.default_rng(7 * N)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = np.exp(rng.uniform(np.log(1e-6), 0.0, N))
    lam[: N // 4] *= -1.0
    lam[N // 4: N // 4 + 3] = 1e-9
    lam[N // 4 + 3: N // 4 + 6] = -1e-9
    X = (Q * lam) @ Q.T
    X = 0.5 * (X + X.T)
    got = project_gpu(env, X)
    want = pack(proj_psd(X))
    assert np.linalg.norm(got - want) <= 2e-10 * np.linalg.norm(pack(X))
