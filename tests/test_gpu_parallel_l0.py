"""GPU Parallel-l0 (Alg. 1), run by the library's round kernels with 0/1 scores, against
the oracle's literal Alg. 1 on noiseless instances of the generating model.

Bars: identical supports after every iteration and at the end; x_hat within 1e-5
(FP32 residuals vs FP64); the same number of iterations and the same convergence; where
Alg. 1 converges, x_hat = x (Thm "convergence of Algorithm 1") in O(log k) iterations.
(Alg. 1 can stall: with d = 15 and alpha = 8 one of these instances keeps 1418 nonzero
residuals on both sides.)"""
import math

import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def _noiseless(n, m, k, d, seed):
    I = gm.instance(n, m, k, d, 0.0, seed)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), m)
    return I, y.astype(np.float32)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("cfg", [dict(n=4096, m=1024, k=60, d=7), dict(n=5003, m=1201, k=90, d=7),
                                 dict(n=20000, m=3000, k=200, d=15), dict(n=6000, m=1500, k=80, d=8)])
@pytest.mark.parametrize("seed", [0, 1])
def test_parallel_l0_matches_oracle_iterate_by_iterate(rl0, cfg, seed):
    I, y32 = _noiseless(seed=seed, **cfg)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    xg, st = rl0.parallel_l0(A, torch.from_numpy(y32).cuda(), tol=TOL)
    xg = xg.cpu().numpy().astype(np.float64)
    xo, it, hist = oracle.parallel_l0(I.rows, y32.astype(np.float64), tol=TOL, history=True)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= 1e-5
    assert st["accepted_rounds"] == it
    log = [e for e in rl0.decode_log(A) if e["updated"] > 0]
    assert [e["support"] for e in log] == [int(np.count_nonzero(h)) for h in hist]
    # converged: every |r_i| <= tol, decided on each side's own residual
    r = y32.astype(np.float64) - oracle.sketch(I.rows, xo, I.m)
    oracle_converged = bool(np.all(np.abs(r) <= TOL))
    assert st["converged"] == int(oracle_converged)
    if oracle_converged:
        np.testing.assert_allclose(xg, I.x, atol=10 * TOL)
        assert it <= 2 + 2 * math.ceil(math.log2(I.k))


def test_parallel_l0_at_full_size_recovers_x(rl0):
    cfg = gm.config_large()
    I, y32 = _noiseless(cfg["n"], cfg["m"], cfg["k"], cfg["d"], 0)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    xg, st = rl0.parallel_l0(A, torch.from_numpy(y32).cuda(), tol=TOL)
    xg = xg.cpu().numpy().astype(np.float64)
    assert st["converged"] == 1
    assert np.array_equal(np.nonzero(xg)[0], np.sort(I.support))
    np.testing.assert_allclose(xg, I.x, atol=10 * TOL)
    assert st["accepted_rounds"] <= 2 + 2 * math.ceil(math.log2(I.k))


def test_parallel_l0_arguments(rl0):
    I, y32 = _noiseless(3000, 800, 40, 8, 3)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y = torch.from_numpy(y32).cuda()
    # alpha = d/2 is allowed (the l1 test is implied); below it is not supported
    x4, st = rl0.parallel_l0(A, y, alpha=4.0, tol=TOL)
    xo, it = oracle.parallel_l0(I.rows, y32.astype(np.float64), alpha=4.0, tol=TOL)
    assert np.array_equal(np.nonzero(x4.cpu().numpy())[0], np.nonzero(xo)[0])
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.parallel_l0(A, y, alpha=3.0, tol=TOL)
    assert e.value.code == -5
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.parallel_l0(A, y, alpha=9.0, tol=TOL)
    assert e.value.code == -1
    # y = 0: nothing to do
    x0, st = rl0.parallel_l0(A, torch.zeros(I.m, device="cuda"), tol=TOL)
    assert st["rounds"] == 0 and st["converged"] == 1 and not x0.any()
    # max_iter bounds the iterations
    x1, st = rl0.parallel_l0(A, y, tol=TOL, max_iter=1)
    assert st["rounds"] == 1 and st["accepted_rounds"] == 1
    _, _, hist = oracle.parallel_l0(I.rows, y32.astype(np.float64), tol=TOL, history=True)
    assert np.array_equal(np.nonzero(x1.cpu().numpy())[0], np.nonzero(hist[0])[0])
    # a later Alg. 2 decode on the same expander is unaffected
    xa, sa = rl0.decode(A, y, I.k, sigma_n=0.0, quantised=True)
    xb, sb = rl0.decode(A, y, I.k, sigma_n=0.0, quantised=True)
    assert torch.equal(xa, xb)
