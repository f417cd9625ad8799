"""GPU tests of the warm-start network kernels (tcgen05 GEMMs with BF16
operands and FP32 accumulation) against the FP64 oracle of oracle/mlp.py:
forward outputs, the loss and every gradient, on tile-aligned and ragged
shapes, and the progress of Adam training."""

import os

import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1708_04174_gb300 import build, capi

    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return torch, capi


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def _unflat(flat, n_in, n_h, n_out):
    out, pos = {}, 0
    for name, shape in (("W1", (n_h, n_in)), ("b1", (n_h,)), ("W2", (n_h, n_h)), ("b2", (n_h,)),
                        ("W3", (n_out, n_h)), ("b3", (n_out,))):
        size = int(np.prod(shape))
        out[name] = flat[pos:pos + size].reshape(shape)
        pos += size
    return out


@pytest.mark.parametrize("n_in,n_h,n_out,batch", [(16, 512, 128, 256), (16, 96, 70, 200), (5, 40, 3, 33)])
def test_gradients_match_oracle(env, n_in, n_h, n_out, batch):
    torch, capi = env
    rng = np.random.default_rng(n_h)
    p = mlp.init(n_in, n_h, n_out, rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    X = rng.standard_normal((batch, n_in)).astype(np.float32)
    Y = rng.standard_normal((batch, n_out)).astype(np.float32)
    net = capi.MLP(n_in, n_h, n_out, seed=1, stream=torch.cuda.current_stream().cuda_stream)
    net.set_params(_flat(p32))
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    loss, g = net.gradients(Xd.data_ptr(), Yd.data_ptr(), batch)
    gg = _unflat(g.astype(np.float64), n_in, n_h, n_out)
    # (1) against the same arithmetic model: operands of every product rounded
    #     to bfloat16, exact FP64 products and sums.  What remains is FP32
    #     accumulation and summation order, far below 2e-3.
    lbf, gbf = mlp.gradients(p32, X.astype(np.float64), Y.astype(np.float64), round_operands=True)
    assert abs(loss - lbf) <= 2e-3 * lbf
    for k in gbf:
        rel = np.linalg.norm(gg[k] - gbf[k]) / max(np.linalg.norm(gbf[k]), 1e-30)
        assert rel < 2e-3, ("bf16 model", k, rel)
    # (2) against plain FP64: each of the (up to) four chained products that
    #     reach W1 rounds both operands (unit roundoff 2^-8), and a rounded pre-activation
    #     near 0 can flip a ReLU mask, so the bound is 5e-2.
    lref, gref = mlp.gradients(p32, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lref) <= 1e-2 * lref
    for k in gref:
        rel = np.linalg.norm(gg[k] - gref[k]) / max(np.linalg.norm(gref[k]), 1e-30)
        assert rel < 5e-2, ("fp64", k, rel)
    out = torch.empty((batch, n_out), device="cuda")
    net.predict(Xd.data_ptr(), out.data_ptr(), batch)
    yref, _ = mlp.forward(p32, X.astype(np.float64))
    assert np.linalg.norm(out.cpu().numpy() - yref) <= 1e-2 * np.linalg.norm(yref)
    net.close()


def test_adam_training_reduces_loss(env):
    torch, capi = env
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.uniform(-1, 1, (512, 16)).astype(np.float32), device="cuda")
    W = rng.standard_normal((16, 40))
    Y = torch.tensor(np.tanh(rng.uniform(-1, 1, (512, 16)) @ W).astype(np.float32), device="cuda")
    Y = torch.tensor(np.tanh(X.cpu().numpy() @ W).astype(np.float32), device="cuda")
    net = capi.MLP(16, 256, 40, seed=5, stream=torch.cuda.current_stream().cuda_stream)
    net.fit_scaling(Y.data_ptr(), 512)
    first = net.train_step(X.data_ptr(), Y.data_ptr(), 512, 1e-3, want_loss=True)
    for _ in range(300):
        net.train_step(X.data_ptr(), Y.data_ptr(), 512, 1e-3)
    last = net.train_step(X.data_ptr(), Y.data_ptr(), 512, 1e-3, want_loss=True)
    assert last < 0.1 * first, (first, last)
    net.close()
