"""Training data and training for the learned column scorer.

Logs come from decoding runs of the method itself: along an analytic Robust-l0 decode
(Algorithm 2, round by round in the library's rl0_scorer_log), every candidate anchor
of every round is logged with its 16 features; its label says whether taking it would
put x_j within `tol_sigma` noise standard deviations of the true value.  Training runs
on the GPU through the library's own forward/backward kernels."""
import torch

from . import mlp_init, mlp_train, scorer_log


def decode_log_samples(A, y, k, x_true, sigma_n, max_rounds=40, tol_sigma=4.0, **params):
    """Features and labels of the candidates met along an analytic decode of (A, y)
    (rl0_scorer_log runs the rounds, the accept test and the stop level).

    x_true: CUDA float32 [n], the signal the sketch came from.  Returns CUDA tensors
    (features [N, 16], labels [N])."""
    feats, labels, _ = scorer_log(A, y, k, x_true.to(torch.float32).contiguous(), max_rounds=max_rounds,
                                  tol_sigma=tol_sigma, sigma_n=sigma_n, **params)
    return feats, labels


def train_scorer(feats, labels, epochs=8, batch=4096, lr=3e-3, seed=0):
    """Shuffle (fixed seed) and train; returns (BF16 parameter bits, FP32 parameters, loss)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(feats.shape[0], generator=g).to(feats.device)
    F = feats[perm].contiguous()
    Y = labels[perm].contiguous()
    w = mlp_init(seed)
    wb, loss = mlp_train(w, F, Y, epochs=epochs, batch=batch, lr=lr)
    return wb, w, loss
