"""Training data and training for the learned column scorer.

Logs come from decoding runs of the method itself: along an analytic Robust-l0 decode
(Algorithm 2, round by round through the library's round step), every candidate anchor
of every round is logged with its 16 features; its label says whether taking it would
put x_j within `tol_sigma` noise standard deviations of the true value.  Training runs
on the GPU through the library's own forward/backward kernels."""
import numpy as np
import torch

from . import (Expander, candidate_features, decode, mlp_init, mlp_train, round_step, sketch)


def decode_log_samples(A, y, k, x_true, sigma_n, max_rounds=40, tol_sigma=4.0, **params):
    """Features and labels of the candidates met along an analytic decode of (A, y).

    x_true: CUDA float32 [n], the signal the sketch came from.  Returns CUDA tensors
    (features [N, 16], labels [N])."""
    n, m = A.n, A.m
    xh = torch.zeros(n, dtype=torch.float32, device="cuda")
    rh = y.clone()
    l1h = float(rh.abs().double().sum())
    feats, labels = [], []
    xt = x_true.to(torch.float32)
    for r in range(1, max_rounds):
        f, meta, w = candidate_features(A, y, k, r, xh, rh, sigma_n=sigma_n, **params)
        if f.shape[0]:
            j = meta[:, 0].long()
            prop = xh[j] + w
            ok = ((prop - xt[j]).abs() <= tol_sigma * sigma_n) & (xt[j] != 0)
            feats.append(f.clone())
            labels.append(ok.float())
        xp, rp, _, l1 = round_step(A, y, k, r, xh, rh, want_passed=False, sigma_n=sigma_n, **params)
        if l1 < l1h:
            xh, rh, l1h = xp, rp, l1
        if l1h <= m * sigma_n * np.sqrt(2 / np.pi):
            break
    if not feats:
        return torch.empty((0, 16), device="cuda"), torch.empty(0, device="cuda")
    return torch.cat(feats), torch.cat(labels)


def train_scorer(feats, labels, epochs=8, batch=4096, lr=3e-3, seed=0):
    """Shuffle (fixed seed) and train; returns (BF16 parameter bits, FP32 parameters, loss)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(feats.shape[0], generator=g).to(feats.device)
    F = feats[perm].contiguous()
    Y = labels[perm].contiguous()
    w = mlp_init(seed)
    wb, loss = mlp_train(w, F, Y, epochs=epochs, batch=batch, lr=lr)
    return wb, w, loss
