"""GPU parity of the adaptive_k variants (Alg. 2 with the adaptive_k flag; Section
"Adaptive k"; Table "variants": Robust-l0-adaptive and Robust-l0-adaptive-quantised)
against the FP64 oracle, through the C ABI.

Bars: identical final support; ||x_gpu - x_orc||_2 / ||x_orc||_2 <= 1e-5; the same
accepted rounds; per round, the posteriors' sparsity prior k0 equal to the oracle's to
1e-6 relative (the GPU sums over its FP32 x_hat, the oracle over its FP64 one)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XTOL = 1e-5


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def _A(rows, m):
    n, d = rows.shape
    return sp.csr_matrix((np.ones(n * d), (rows.ravel(), np.repeat(np.arange(n), d))), shape=(m, n))


def _problem(n, m, k, d, sigma_n, seed):
    I = gm.instance(n, m, k, d, sigma_n, seed)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
    return I, y.astype(np.float32)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _both(rl0, I, y32, **kw):
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    xg, st = rl0.decode(A, torch.from_numpy(y32).cuda(), I.k, sigma_n=I.sigma_n, adaptive_k=True, **kw)
    log = rl0.decode_log(A)
    xo, sto, logo = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, adaptive_k=True, **kw)
    return A, xg.cpu().numpy().astype(np.float64), st, log, xo, sto, logo


@pytest.mark.parametrize("quantised", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adaptive_decode_matches_oracle(rl0, quantised, seed):
    I, y32 = _problem(seed=seed, **gm.config_small())
    A, xg, st, log, xo, sto, logo = _both(rl0, I, y32, quantised=quantised)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["rounds"] == sto["rounds"]
    assert st["accepted_rounds"] == sto["accepted_rounds"]
    assert [e["accepted"] for e in log] == [e["accepted"] for e in logo]
    for e, o in zip(log, logo):
        assert e["k_prior"] == pytest.approx(o["k_prior"], rel=1e-6)
    if not quantised:
        assert any(e["k_prior"] != I.k for e in log)               # the prior did move
    r = y32.astype(np.float64) - _A(I.rows, I.m) @ xg
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)


@pytest.mark.parametrize("cfg", [dict(n=5003, m=1201, k=110, d=7, sigma_n=2e-3),
                                 dict(n=20000, m=3000, k=250, d=15, sigma_n=1e-3)])
def test_adaptive_other_shapes_match_oracle(rl0, cfg):
    I, y32 = _problem(seed=4, **cfg)
    A, xg, st, log, xo, sto, logo = _both(rl0, I, y32)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["accepted_rounds"] == sto["accepted_rounds"]


def test_noiseless_adaptive_equals_plain_bitwise(rl0):
    I, y32 = _problem(3000, 900, 60, 7, 0.0, 4)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y = torch.from_numpy(y32).cuda()
    for q in (False, True):
        x0, s0 = rl0.decode(A, y, I.k, sigma_n=0.0, quantised=q)
        x1, s1 = rl0.decode(A, y, I.k, sigma_n=0.0, quantised=q, adaptive_k=True)
        assert torch.equal(x0, x1)
        assert s0["rounds"] == s1["rounds"] and s0["final_l1"] == s1["final_l1"]


def test_adaptive_full_size_decode_properties(rl0):
    cfg = gm.config_large()
    I, y32 = _problem(seed=0, **cfg)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    xg, st = rl0.decode(A, torch.from_numpy(y32).cuda(), I.k, sigma_n=I.sigma_n, adaptive_k=True)
    x = xg.cpu().numpy().astype(np.float64)
    log = rl0.decode_log(A)
    r = y32.astype(np.float64) - _A(I.rows, I.m) @ x
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)
    assert np.count_nonzero(x) <= I.k
    l1 = [e["l1_hat"] for e in log]
    assert all(b <= a for a, b in zip(l1, l1[1:]))
    assert all(e["k_prior"] >= I.m // 100 for e in log)
    # the prior after an accepted round, from the final state of that round: checked
    # against the oracle's posterior for the first accepted round
    first = next(i for i, e in enumerate(log) if e["accepted"])
    if first + 1 < len(log):
        x1, _ = rl0.decode(A, torch.from_numpy(y32).cuda(), I.k, sigma_n=I.sigma_n, adaptive_k=True,
                           max_rounds=first + 1)
        nz = x1.cpu().numpy().astype(np.float64)
        nz = nz[nz != 0.0]
        pz = np.exp(oracle.log_posterior("z", nz, I.d, I.k / I.m, 1.0, I.sigma_n))
        k0 = max(I.k - np.sum(1.0 - pz), float(I.m // 100))
        assert log[first + 1]["k_prior"] == pytest.approx(k0, rel=1e-9)
    # success condition, C_1 = 1
    m, s = I.m, I.sigma_n
    xl1 = np.abs(I.x).sum()
    tol = min((m * s * math.sqrt(2 / math.pi) + math.sqrt(m * s * s * (1 - 2 / math.pi))) / xl1, 0.1)
    assert np.abs(x - I.x).sum() / xl1 <= tol


def test_adaptive_is_unsupported_where_no_host_step_fits(rl0):
    I, y32 = _problem(seed=1, **gm.config_small())
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y = torch.from_numpy(y32).cuda()
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_static(A, y, I.k, sigma_n=I.sigma_n, adaptive_k=True)
    assert e.value.code == -5
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_batched([A], [y], [I.k], [dict(sigma_n=I.sigma_n, adaptive_k=True)])
    assert e.value.code == -5
