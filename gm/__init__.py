"""Seeded synthetic inputs drawn from the paper's generating model GM(n, m, k, d, mu, nu)
(Def. "Generating model", Fig. 1 of arXiv 1704.09012), with mu = N(0, sigma_s^2) and
nu = N(0, sigma_n^2).

This module only draws random numbers: the rows of A, the support and values of x,
and the noise eta.  It holds none of the decoder's arithmetic (not even the sketch
y = A x + eta), so both the FP64 oracle and the CUDA library can take their inputs
from it without sharing any of the method.

Randomness: numpy's Philox bit generator seeded with (seed, stream), one stream per
quantity, so that e.g. the noise of an instance does not change when n changes.
"""
from dataclasses import dataclass
import math

import numpy as np

STREAM_A, STREAM_SUPPORT, STREAM_VALUES, STREAM_NOISE = 1, 2, 3, 4


def _rng(seed, stream):
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, stream]))


def draw_rows(n, m, d, seed):
    """Item 1 of Def. GM: every column's support is uniform over the d-subsets of [m].

    Returns int32 (n, d), each row of the array (one column of A) sorted ascending."""
    if not (1 <= d <= m):
        raise ValueError("need 1 <= d <= m")
    rng = _rng(seed, STREAM_A)
    rows = np.sort(rng.integers(0, m, size=(n, d), dtype=np.int64), axis=1)
    while True:
        bad = np.nonzero(np.any(np.diff(rows, axis=1) == 0, axis=1))[0] if d > 1 else np.zeros(0, np.int64)
        if bad.size == 0:
            break
        rows[bad] = np.sort(rng.integers(0, m, size=(bad.size, d), dtype=np.int64), axis=1)
    return rows.astype(np.int32)


def draw_signal(n, k, sigma_s, seed):
    """Items 2-3: supp(x) uniform over the k-subsets of [n]; x_j ~ N(0, sigma_s^2) (FP32)."""
    supp = np.sort(_rng(seed, STREAM_SUPPORT).choice(n, size=k, replace=False)).astype(np.int64)
    vals = (_rng(seed, STREAM_VALUES).standard_normal(k) * sigma_s).astype(np.float32)
    x = np.zeros(n, np.float32)
    x[supp] = vals
    return x, supp


def draw_noise(m, sigma_n, seed):
    """Items 4-5: eta_i ~ N(0, sigma_n^2) i.i.d., independent of x (FP32)."""
    if sigma_n == 0:
        return np.zeros(m, np.float32)
    return (_rng(seed, STREAM_NOISE).standard_normal(m) * sigma_n).astype(np.float32)


def sigma_from_snr(d, rho, snr_db, sigma_s=1.0):
    """Noise std for a target per-measurement SNR.  E[y_i^2] = d rho sigma_s^2 under
    Def. GM (each row holds d k / m = d rho signal entries on average), so
    sigma_n = sigma_s sqrt(d rho) 10^(-SNR/20).  None means noiseless."""
    if snr_db is None:
        return 0.0
    return sigma_s * math.sqrt(d * rho) * 10.0 ** (-snr_db / 20.0)


@dataclass
class Instance:
    n: int
    m: int
    k: int
    d: int
    sigma_s: float
    sigma_n: float
    seed: int
    rows: np.ndarray      # int32 (n, d), column-major rows of A
    x: np.ndarray         # float32 (n,)
    support: np.ndarray   # int64 (k,)
    eta: np.ndarray       # float32 (m,)


def instance(n, m, k, d, sigma_n, seed, sigma_s=1.0):
    rows = draw_rows(n, m, d, seed)
    x, supp = draw_signal(n, k, sigma_s, seed)
    eta = draw_noise(m, sigma_n, seed)
    return Instance(n, m, k, d, sigma_s, sigma_n, seed, rows, x, supp, eta)


def config_small():
    """n=4096, m=1024, k=100, d=7, sigma_n=1e-3."""
    return dict(n=4096, m=1024, k=100, d=7, sigma_n=1e-3)


def config_large():
    """n=2^20, delta=0.1, rho=0.1, d=7, SNR 40 dB."""
    n = 1 << 20
    m = int(math.floor(0.1 * n))
    k = int(math.floor(0.1 * m))
    return dict(n=n, m=m, k=k, d=7, sigma_n=sigma_from_snr(7, k / m, 40.0))


def batch_shapes(count, seed=0, d=7):
    """Shapes of the batched workload: n uniform over [2^10, 2^16], delta in [0.1, 0.3],
    rho in [0.05, 0.2], SNR in [30, 60] dB.  Returns a list of dicts."""
    rng = _rng(seed, 0x42)
    out = []
    for _ in range(count):
        n = int(rng.integers(1 << 10, (1 << 16) + 1))
        delta = float(rng.uniform(0.1, 0.3))
        rho = float(rng.uniform(0.05, 0.2))
        snr = float(rng.uniform(30.0, 60.0))
        m = max(int(math.floor(delta * n)), d + 1)
        k = max(int(math.floor(rho * m)), 1)
        out.append(dict(n=n, m=m, k=k, d=d, sigma_n=sigma_from_snr(d, k / m, snr)))
    return out
