"""FP64 reference of the learned column scorer's network and its training loss
(TEST INFRASTRUCTURE: only the test-suite and the CPU-baseline leg may use it).

Network: 16 -> 32 -> 32 -> 1 with ReLU hidden layers; parameters in one flat vector
W1 (16x32, input-major), b1 (32), W2 (32x32), b2 (32), w3 (32), b3 (1).
Loss: mean binary cross-entropy of the logits, L = mean(softplus(o) - y o).
Gradients by the chain rule, written out layer by layer."""
import numpy as np

NF, H = 16, 32
SIZES = [("W1", NF * H), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, np.float64)
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = w[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(NF, H)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def forward(w, F):
    P = unpack(w)
    F = np.asarray(F, np.float64)
    z1 = F @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ P["w3"] + P["b3"][0]
    return o, (z1, h1, z2, h2)


def loss(w, F, y):
    o, _ = forward(w, F)
    sp = np.where(o > 0, o + np.log1p(np.exp(-np.abs(o))), np.log1p(np.exp(o)))
    return float(np.mean(sp - np.asarray(y, np.float64) * o))


def loss_and_grad(w, F, y):
    F = np.asarray(F, np.float64)
    y = np.asarray(y, np.float64)
    P = unpack(w)
    o, (z1, h1, z2, h2) = forward(w, F)
    N = F.shape[0]
    sp = np.where(o > 0, o + np.log1p(np.exp(-np.abs(o))), np.log1p(np.exp(o)))
    L = float(np.mean(sp - y * o))
    do = (1.0 / (1.0 + np.exp(-o)) - y) / N
    g_w3 = h2.T @ do
    g_b3 = np.array([do.sum()])
    dz2 = np.outer(do, P["w3"]) * (z2 > 0)
    g_W2 = h1.T @ dz2
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"].T) * (z1 > 0)
    g_W1 = F.T @ dz1
    g_b1 = dz1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])
    return L, g
