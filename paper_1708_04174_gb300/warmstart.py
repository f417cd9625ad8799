"""Learned warm start for a parametric family of SOS programs.

A family p(theta) = p0 + sum_k theta_k q_k of SOS programs is solved many
times.  The pipeline

1. solves a training set of members with the batched GPU solver and keeps
   their normalised solutions (xi, y, z) = (u_xi, u_y, v_z) / tau;
2. trains the network of ``capi.MLP`` (tensor-core kernels) to map theta to
   that solution vector, targets standardised per component;
3. for new members, predicts the solution and starts ADMM from
   u0 = (xi, y, 1), v0 = (z, 0, 0) (free part of z set to 0).  Any start is
   admissible: one ADMM step maps it into C x C* (u = P_C(.),
   v = u - (.) is minus the polar part), so the prediction is not projected
   first.

Only orchestration lives here; solves and training run in libsos.
"""

from __future__ import annotations

import time
from typing import List, Tuple

import numpy as np

from . import capi


def solution_vectors(results, dims) -> np.ndarray:
    """[xi; y; z] per instance from sos_solve results."""
    rows = []
    for r, d in zip(results, dims):
        rows.append(np.concatenate([r["x"], r["y"], r["s"]]))
    return np.stack(rows).astype(np.float32)


def start_points(pred: np.ndarray, dims) -> Tuple[np.ndarray, np.ndarray]:
    """Concatenated (u0, v0) for sos_set_iterate from predicted [xi; y; z]."""
    us, vs = [], []
    for row, d in zip(pred.astype(np.float64), dims):
        nx, m, t = d[0], d[1], d[2]
        xi, y, z = row[:nx], row[nx:nx + m], row[nx + m:2 * nx + m].copy()
        z[:t] = 0.0  # the dual of a free variable is 0
        us.append(np.concatenate([xi, y, [1.0]]))
        vs.append(np.concatenate([z, np.zeros(m), [0.0]]))
    return np.concatenate(us), np.concatenate(vs)


class WarmStart:
    def __init__(self, family, hidden: int = 512, seed: int = 0, precision: int = capi.PREC_MIXED,
                 k_check: int = 10, stream: int = 0):
        self.family = family
        self.hidden = hidden
        self.seed = seed
        self.precision = precision
        self.k_check = k_check
        self.stream = stream
        self.net = None
        self.n_out = None
        self.log = {}
        self.last_dims = None

    def solve(self, thetas: np.ndarray, tol: float, max_iter: int, start=None, precision=None):
        """Batched solve of the members for ``thetas`` (in this object's
        precision form unless ``precision`` is given); returns results and dims."""
        progs = self.family.programs(thetas)
        prec = self.precision if precision is None else precision
        s = capi.Solver(progs, precision=prec, k_check=self.k_check)
        if start is not None:
            s.set_iterate(*start_points(start, s.dims))
        t0 = time.perf_counter()
        res = s.solve(tol, max_iter)
        dt = time.perf_counter() - t0
        dims = s.dims
        self.last_dims = dims
        tuning = s.tuning()
        s.close()
        return res, dims, dt, tuning

    def train(self, thetas: np.ndarray, targets: np.ndarray, epochs: int = 40, batch: int = 256, lr: float = 1e-3):
        import torch

        n_in, n_out = thetas.shape[1], targets.shape[1]
        self.n_out = n_out
        self.net = capi.MLP(n_in, self.hidden, n_out, seed=self.seed, stream=self.stream)
        X = torch.tensor(thetas.astype(np.float32), device="cuda")
        Y = torch.tensor(targets.astype(np.float32), device="cuda")
        self.net.fit_scaling(Y.data_ptr(), Y.shape[0])
        rng = np.random.default_rng(self.seed)
        n = X.shape[0]
        if n == 0:
            raise ValueError("no training members")
        batch = min(batch, n)
        steps = n // batch
        losses = []
        t0 = time.perf_counter()
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device="cuda")
            Xs, Ys = X[perm].contiguous(), Y[perm].contiguous()
            for k in range(steps):
                i = k * batch
                last = k == steps - 1  # the loss of each epoch's final minibatch is recorded
                loss = self.net.train_step(Xs[i].data_ptr(), Ys[i].data_ptr(), batch, lr, want_loss=last)
                if last:
                    losses.append(loss)
        self.log["train_seconds"] = time.perf_counter() - t0
        self.log["losses"] = losses
        return losses

    def predict(self, thetas: np.ndarray) -> np.ndarray:
        import torch

        X = torch.tensor(thetas.astype(np.float32), device="cuda")
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        self.net.predict(X.data_ptr(), Y.data_ptr(), X.shape[0])
        return Y.cpu().numpy()
