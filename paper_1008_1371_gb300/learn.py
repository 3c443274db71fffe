"""Training of the learned form's skip network on sweep traces the method
itself generates (the plain blocked method writes one row per block-pair
visit: 8 features from the previous visit's record, label 1 if the visit
rotated).  Python only orchestrates: the forward/backward pass and the Adam
step run in the library's kernels (hsvd_mlp_grad, hsvd_mlp_adam).
"""
import numpy as np
import torch

from . import api


def init_params(seed=0, device="cuda"):
    """He-initialised parameter vector; the output bias starts at +2 (the
    network first predicts "rotates", i.e. skips nothing)."""
    g = torch.Generator().manual_seed(seed)
    F, H = api.HSVD_MLP_FEATURES, 64
    W1 = torch.randn(H, F, generator=g) * (2.0 / F) ** 0.5
    W2 = torch.randn(H, H, generator=g) * (2.0 / H) ** 0.5
    w3 = torch.randn(H, generator=g) * (1.0 / H) ** 0.5
    p = torch.cat([W1.ravel(), torch.zeros(H), W2.ravel(), torch.zeros(H), w3, torch.tensor([2.0])])
    assert p.numel() == api.HSVD_MLP_PARAMS
    return p.to(torch.float32).to(device).contiguous()


def collect(factors, block_w=32, max_sweeps=30, precision=api.HSVD_PRECISION_FP64, device="cuda"):
    """Training rows from plain blocked solves of (G, J) pairs (numpy).
    Returns (X, y) CUDA tensors."""
    rows = []
    for G, J in factors:
        n = G.shape[1]
        nb = -(-n // (2 * block_w)) * 2
        cap = nb * (nb // 2) * max_sweeps
        out = torch.zeros((cap, api.HSVD_MLP_FEATURES + 1), dtype=torch.float32, device=device)
        Gd = torch.from_numpy(np.asfortranarray(G)).to(device)
        Jd = torch.from_numpy(J).to(device)
        r = api.hsvd_solve_ex(Gd, Jd, api.make_opts(method=api.HSVD_METHOD_BLOCKED, block_w=block_w, sort=False,
                                                     max_sweeps=max_sweeps, precision=precision, trace_out=out),
                              compute_u=False, compute_v=False)
        rows.append(out[:r.trace_rows].clone())
    data = torch.cat(rows)
    return data[:, :api.HSVD_MLP_FEATURES].contiguous(), data[:, api.HSVD_MLP_FEATURES].contiguous()


def train(X, y, steps=400, lr=3e-3, batch=4096, seed=0, params=None):
    """Adam on the mean binary cross-entropy; minibatches drawn with a seeded
    generator.  Returns (params, losses)."""
    p = init_params(seed, X.device) if params is None else params.clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.Generator(device="cpu").manual_seed(seed + 1)
    n = X.shape[0]
    losses = []
    for t in range(1, steps + 1):
        if n > batch:
            idx = torch.randint(0, n, (batch,), generator=g).to(X.device)
            xb, yb = X[idx].contiguous(), y[idx].contiguous()
        else:
            xb, yb = X, y
        grad, loss = api.hsvd_mlp_grad(p, xb, yb)
        api.hsvd_mlp_adam(p, m, v, grad, t, lr=lr)
        if t % 50 == 0 or t == steps:
            losses.append(float(loss.item()))
    return p, losses
