"""Learned row sizing: features, the 6 -> 64 -> 64 -> 1 predictor and its
training, all through the library's CUDA kernels (argument marshalling only).

The predictor estimates log1p(n_nz) of each output row from six row
features (see ``spgemm_features`` in include/opsparse.h). Its labels are the
exact row sizes that the two-phase method itself computes; the training
loop runs forward, backward and Adam on the GPU (``spgemm_mlp_train_step``,
``spgemm_mlp_adam``).
"""

from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import CSR, Handle, _abi, _csr_in

N_PARAMS = 4673
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "predictor", "weights.npy")
MANIFEST = os.path.join(HERE, "predictor", "manifest.json")


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def features(A: CSR, B: CSR, row_begin: int = 0, row_end: int | None = None):
    """(rows, 6) float32 CUDA tensor of row features of C = A*B."""
    import torch
    row_end = A.rows if row_end is None else row_end
    n = row_end - row_begin
    X = torch.empty((max(n, 1), 6), dtype=torch.float32, device=A.rpt.device)
    ws = torch.empty(max(n, 1) * 16, dtype=torch.uint8, device=A.rpt.device)
    a, b = _csr_in(A, False), _csr_in(B, False)
    _abi.check(_abi.lib().spgemm_features(ctypes.byref(a), ctypes.byref(b), row_begin, row_end,
                                          X.data_ptr(), ws.data_ptr(), _stream()), "spgemm_features")
    return X[:n]


class Predictor:
    """Parameters, Adam moments and the GPU training step."""

    def __init__(self, theta=None, seed: int = 0):
        import torch
        if theta is None:
            import workloads
            theta = workloads.mlp_init(seed)
        self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float32)).cuda().contiguous()
        assert self.theta.numel() == N_PARAMS
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step_count = 0

    def forward(self, X):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _abi.check(_abi.lib().spgemm_mlp_forward(self.theta.data_ptr(), X.contiguous().data_ptr(),
                                                 X.shape[0], y.data_ptr(), _stream()),
                   "spgemm_mlp_forward")
        return y

    def gradient(self, X, t):
        """(loss, grad) of mean((y - t)^2) over the batch, on the GPU."""
        self.grad.zero_()
        self.loss.zero_()
        _abi.check(_abi.lib().spgemm_mlp_train_step(
            self.theta.data_ptr(), X.contiguous().data_ptr(), t.contiguous().data_ptr(),
            X.shape[0], X.shape[0], self.grad.data_ptr(), self.loss.data_ptr(), _stream()),
            "spgemm_mlp_train_step")
        return self.loss, self.grad

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        _abi.check(_abi.lib().spgemm_mlp_adam(self.theta.data_ptr(), self.grad.data_ptr(),
                                              self.m.data_ptr(), self.v.data_ptr(),
                                              self.step_count, lr, beta1, beta2, eps, _stream()),
                   "spgemm_mlp_adam")

    def fit(self, X, t, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0):
        """Mini-batch Adam on (X, t); returns the mean loss of each epoch."""
        import torch
        g = torch.Generator(device="cpu").manual_seed(seed)
        n = X.shape[0]
        history = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=g).to(X.device)
            tot = torch.zeros(1, dtype=torch.float64, device=X.device)
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                loss, _ = self.gradient(X[idx], t[idx])
                tot += loss.double() * idx.numel()
                self.adam(lr)
            history.append(float(tot.item()) / n)
        return history

    def save(self, path=WEIGHTS, manifest: dict | None = None):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        np.save(path, self.theta.cpu().numpy())
        if manifest is not None:
            with open(os.path.splitext(path)[0].replace("weights", "manifest") + ".json", "w") as f:
                json.dump(manifest, f, indent=1)

    @classmethod
    def load(cls, path=WEIGHTS):
        return cls(np.load(path))


def row_labels(A: CSR, B: CSR, handle: Handle | None = None):
    """Exact n_nz of every output row, from the two-phase method itself."""
    own = handle is None
    h = handle or Handle()
    try:
        h.symbolic(A, B)
        C = h.numeric(A, B)
        rpt = C.rpt
        return (rpt[1:] - rpt[:-1]).to(dtype=rpt.dtype)
    finally:
        if own:
            h.close()


def sample_rows(nprod_feature, k: int, seed: int):
    """Up to k row indices stratified by log1p(n_prod): equal draws from
    eight quantile strata, so the few large rows are represented."""
    import torch
    n = nprod_feature.numel()
    if n <= k:
        return torch.arange(n, device=nprod_feature.device)
    rng = np.random.default_rng(seed)
    f = nprod_feature.cpu().numpy()
    order = np.argsort(f, kind="stable")
    strata = np.array_split(order, 8)
    per = k // 8
    pick = np.concatenate([rng.choice(s, size=min(per, s.size), replace=False) for s in strata if s.size])
    return torch.as_tensor(np.sort(pick), device=nprod_feature.device)


def training_set(pairs, rows_per_matrix: int = 4096, seed: int = 0, handle: Handle | None = None):
    """Features and log1p(n_nz) labels from (A, B) pairs of CSR (device)."""
    import torch
    Xs, ts = [], []
    for i, (A, B) in enumerate(pairs):
        X = features(A, B)
        nnz = row_labels(A, B, handle)
        idx = sample_rows(X[:, 1], rows_per_matrix, seed + i)
        Xs.append(X[idx])
        ts.append(torch.log1p(nnz[idx].to(torch.float32)))
    return torch.cat(Xs), torch.cat(ts)
