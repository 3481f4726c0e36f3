"""The oracle's adaptive_k variants (Alg. 2 with the adaptive_k flag; Section "Adaptive
k"; Table "variants"), pinned against what the method fixes:

- noiseless, the posteriors are indicators that do not depend on the sparsity prior, so
  the adaptive decode must equal the plain one, and the prior it records after an
  accepted round is the closed form max(k - |supp x_hat|, floor(m/100));
- with noise, the prior recorded after an accepted round must be
  k - sum_j (1 - p_z(x_hat_j)) floored at m/100, with p_z the posterior at the prior the
  round used (evaluated through log_posterior, which the Monte-Carlo pins check against
  the model);
- the decode invariants of Alg. 2 hold and the noisy workload is recovered."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle


def _A(rows, m):
    n, d = rows.shape
    return sp.csr_matrix((np.ones(n * d), (rows.ravel(), np.repeat(np.arange(n), d))), shape=(m, n))


def _instance(cfg, seed, f32=True):
    I = gm.instance(seed=seed, **cfg)
    y = _A(I.rows, I.m) @ I.x.astype(np.float64) + I.eta.astype(np.float64)
    if f32:
        y = y.astype(np.float32).astype(np.float64)
    return I, y


@pytest.mark.parametrize("quantised", [True, False])
def test_noiseless_adaptive_equals_plain_and_prior_is_the_support_count(quantised):
    n, m, d, k = 4096, 1024, 7, 60
    for seed in range(2):
        I, y = _instance(dict(n=n, m=m, k=k, d=d, sigma_n=0.0), seed, f32=False)
        kw = dict(sigma_n=0.0, quantised=quantised, noiseless_tol=1e-9)
        x0, st0, log0 = oracle.decode(I.rows, y, I.k, **kw)
        x1, st1, log1 = oracle.decode(I.rows, y, I.k, adaptive_k=True, **kw)
        np.testing.assert_array_equal(x1, x0)
        assert [e["accepted"] for e in log1] == [e["accepted"] for e in log0]
        # p_z is the indicator of |w| <= tol: 1 - p_z(x_hat_j) counts the support
        want = float(k)
        for e in log1:
            assert e["k_prior"] == want
            if e["accepted"]:
                want = max(float(k - e["support"]), float(m // 100))
        assert log0 and all(e["k_prior"] == k for e in log0)


def test_noisy_prior_follows_the_adaptive_k_step():
    cfg = gm.config_small()
    I, y = _instance(cfg, 0)
    kw = dict(sigma_n=I.sigma_n, quantised=False, adaptive_k=True)
    _, _, full = oracle.decode(I.rows, y, I.k, **kw)
    acc = [r for r, e in enumerate(full) if e["accepted"]]
    assert len(acc) >= 2
    checked = 0
    for r in acc[:4]:
        # x_hat right after the accepted round r, and the prior round r used
        x_r, _, log_r = oracle.decode(I.rows, y, I.k, max_rounds=r + 1, **kw)
        assert log_r[r]["accepted"]
        rho_used = log_r[r]["k_prior"] / I.m
        nz = x_r[x_r != 0.0]
        pz = np.exp(oracle.log_posterior("z", nz, I.d, rho_used, 1.0, I.sigma_n))
        k0 = max(I.k - np.sum(1.0 - pz), float(I.m // 100))
        if r + 1 < len(full):
            assert full[r + 1]["k_prior"] == pytest.approx(k0, rel=1e-12, abs=1e-9)
            checked += 1
    assert checked >= 1
    # the prior only changes after accepted rounds
    for a, b in zip(full, full[1:]):
        if not a["accepted"]:
            assert b["k_prior"] == a["k_prior"]


@pytest.mark.parametrize("quantised", [False, True])
def test_adaptive_decode_invariants_and_recovery(quantised):
    cfg = gm.config_small()
    for seed in range(3):
        I, y = _instance(cfg, seed)
        x, st, log = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, quantised=quantised, adaptive_k=True)
        A = _A(I.rows, I.m)
        r = y - A @ x
        assert np.abs(r).sum() == pytest.approx(st["final_l1"], rel=1e-12)     # r_hat = y - A x_hat
        l1 = [e["l1_hat"] for e in log]
        assert all(b <= a for a, b in zip(l1, l1[1:]))                     # ||r_hat||_1 non-increasing
        assert np.count_nonzero(x) <= I.k                                   # H_k keeps the original k
        assert all(e["k_prior"] >= I.m // 100 for e in log)
        m, s = I.m, I.sigma_n
        xl1 = np.abs(I.x).sum()
        tol = min((m * s * math.sqrt(2 / math.pi) + math.sqrt(m * s * s * (1 - 2 / math.pi))) / xl1, 0.1)
        assert np.abs(x - I.x).sum() / xl1 <= tol                          # success condition, C_1 = 1


def test_adaptive_with_the_learned_scorer_is_rejected():
    I, y = _instance(gm.config_small(), 0)
    with pytest.raises(Exception):
        oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, adaptive_k=True,
                      mlp_bf16=np.zeros(1633, np.uint16))
