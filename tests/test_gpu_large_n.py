"""Extreme subsampling and large n (Section "Phase transitions for extreme subsampling"):
delta = 0.001, sigma = 0.001, n = 2^22 and 2^24, d = 7.

- n = 2^22: one round of the decoder from a perturbed-truth state against the oracle,
  column by column (the oracle takes ~12 s per round at this size).
- n = 2^24 (nnz = 1.17e8): the whole decode, its invariants against an FP64 residual
  recomputed by the oracle's sketch, and recovery under Eq. (success_condition_clip).
- m = 114 000 (delta = 0.1): the residual codes fill all but about 250 bytes of the
  column kernel's shared memory, so it stages at most 3 survivors per CTA there and
  lists the others in global memory; one round from a state with most of the support
  missing (thousands of survivors) against the oracle."""
import math

import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 1e-4
XTOL = 1e-5


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _problem(n, delta, rho, sigma, seed, d=7):
    m = int(delta * n)
    k = int(rho * m)
    I = gm.instance(n, m, k, d, sigma, seed)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
    return I, y.astype(np.float32)


def test_one_round_at_n_2e22_delta_1e_3_matches_oracle(rl0):
    I, y32 = _problem(1 << 22, 0.001, 0.05, 0.001, 11)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y64 = y32.astype(np.float64)
    rng = np.random.default_rng(3)
    x = I.x.astype(np.float64).copy()
    sh = rng.choice(I.support, I.k // 4, replace=False)
    x[sh] += rng.uniform(0.2, 1.0, sh.size)
    x[rng.choice(I.support, I.k // 4, replace=False)] = 0.0
    x32 = x.astype(np.float32)
    r32 = (y64 - oracle.sketch(I.rows, x32.astype(np.float64), I.m)).astype(np.float32)
    c = oracle.default_c(False, I.m / I.n, I.k / I.m)
    ridx = int(0.5 / c)
    xo, ro, updo, rec = oracle.round_step(I.rows, y64, I.k, ridx, x32.astype(np.float64), r32.astype(np.float64),
                                          sigma_n=I.sigma_n)
    xg, rg, passed, l1g = rl0.round_step(A, torch.from_numpy(y32).cuda(), I.k, ridx, torch.from_numpy(x32).cuda(),
                                         torch.from_numpy(r32).cuda(), sigma_n=I.sigma_n)
    pg = passed.cpu().numpy().astype(bool)
    po = rec["passed"].astype(bool)
    near = rec["min_margin"] < MARGIN
    assert np.array_equal(pg[~near], po[~near])
    assert po.sum() > 20 and near.sum() <= 2
    if np.array_equal(pg, po):
        xg = xg.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
        assert _rel(xg, xo) <= XTOL
        assert l1g == pytest.approx(np.abs(ro).sum(), rel=1e-6)


def test_decode_at_n_2e24_delta_1e_3(rl0):
    I, y32 = _problem(1 << 24, 0.001, 0.05, 0.001, 12)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    xg, st = rl0.decode(A, torch.from_numpy(y32).cuda(), I.k, sigma_n=I.sigma_n)
    x = xg.cpu().numpy().astype(np.float64)
    assert np.count_nonzero(x) <= I.k
    r = y32.astype(np.float64) - oracle.sketch(I.rows, x, I.m)
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)
    log = rl0.decode_log(A)
    l1 = [e["l1_hat"] for e in log]
    assert all(b <= a for a, b in zip(l1, l1[1:]))
    m, s = I.m, I.sigma_n
    xl1 = np.abs(I.x).sum()
    tol = min((m * s * math.sqrt(2 / math.pi) + math.sqrt(m * s * s * (1 - 2 / math.pi))) / xl1, 0.1)
    assert np.abs(x - I.x).sum() / xl1 <= tol
    assert st["converged"] == 1


def test_round_with_survivors_beyond_the_shared_staging(rl0):
    n, m = 1_140_000, 114_000
    I, y32 = _problem(n, 0.1, 0.1, 0.001, 14)
    assert I.m == m
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y64 = y32.astype(np.float64)
    rng = np.random.default_rng(5)
    x = I.x.astype(np.float64).copy()
    x[rng.choice(I.support, (4 * I.k) // 5, replace=False)] = 0.0       # most of the support missing
    sh = rng.choice(I.support, I.k // 10, replace=False)
    x[sh] += rng.uniform(0.2, 1.0, sh.size)
    x32 = x.astype(np.float32)
    r32 = (y64 - oracle.sketch(I.rows, x32.astype(np.float64), I.m)).astype(np.float32)
    c = oracle.default_c(False, I.m / I.n, I.k / I.m)
    ridx = int(0.5 / c)
    xo, ro, updo, rec = oracle.round_step(I.rows, y64, I.k, ridx, x32.astype(np.float64), r32.astype(np.float64),
                                          sigma_n=I.sigma_n)
    xg, rg, passed, l1g = rl0.round_step(A, torch.from_numpy(y32).cuda(), I.k, ridx, torch.from_numpy(x32).cuda(),
                                         torch.from_numpy(r32).cuda(), sigma_n=I.sigma_n)
    pg = passed.cpu().numpy().astype(bool)
    po = rec["passed"].astype(bool)
    near = rec["min_margin"] < MARGIN
    assert np.array_equal(pg[~near], po[~near])
    assert po.sum() > 152 * 10 and near.sum() <= 2 + po.size // 100000
    if np.array_equal(pg, po):
        xg = xg.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
        assert _rel(xg, xo) <= XTOL
        assert l1g == pytest.approx(np.abs(ro).sum(), rel=1e-6)
