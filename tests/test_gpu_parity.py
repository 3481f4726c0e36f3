"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same
seeded inputs.  Inputs come from the generator module `gm` and from the oracle; nothing
the CUDA path computes is ever fed to the oracle.

Bars (from the method's arithmetic):
  - integer/index work (rows of A, supports, pass decisions) bit-exact;
  - x_hat: ||x_gpu - x_orc||_2 / ||x_orc||_2 <= 1e-5 (FP32 path vs FP64 oracle);
  - residuals: |r_gpu - r_orc| <= 4 ulp of the row's |terms| plus A |x_gpu - x_orc|;
  - a decision of the oracle whose margin is below 1e-4 may differ (FP32 scoring of the
    same FP32 inputs); such columns are counted and must be rare.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XTOL = 1e-5
MARGIN = 1e-4


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def _A(rows, m):
    n, d = rows.shape
    return sp.csr_matrix((np.ones(n * d), (rows.ravel(), np.repeat(np.arange(n), d))), shape=(m, n))


def _problem(n, m, k, d, sigma_n, seed, sigma_s=1.0):
    """Instance from the generator, y_hat computed by the oracle in FP64 and rounded to FP32."""
    I = gm.instance(n, m, k, d, sigma_n, seed, sigma_s=sigma_s)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
    return I, y.astype(np.float32)


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ------------------------------------------------------------------ expander and sketch
@pytest.mark.parametrize("n,m,d,seed", [(1000, 300, 7, 0), (4097, 1024, 7, 5), (777, 40, 15, 3),
                                        (300, 33, 32, 9), (50, 7, 7, 1), (2000, 10000, 3, 2)])
def test_make_expander_matches_oracle_philox(rl0, n, m, d, seed):
    A = rl0.Expander.random(n, m, d, seed=seed)
    got = A.rows().cpu().numpy()
    np.testing.assert_array_equal(got, oracle.make_expander(n, m, d, seed))


def test_expander_from_rows_roundtrip_and_validation(rl0):
    I = gm.instance(3000, 700, 90, 7, 0.0, 4)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    np.testing.assert_array_equal(A.rows().cpu().numpy(), I.rows)
    bad = I.rows.copy()
    bad[5, 2] = bad[5, 1]                                   # duplicate row in column 5
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.Expander.from_rows(_cuda(bad), I.m)
    assert e.value.code == -6
    bad = I.rows.copy()
    bad[7, 6] = I.m                                         # out of range
    with pytest.raises(rl0.Rl0Error):
        rl0.Expander.from_rows(_cuda(bad), I.m)
    bad = I.rows.copy()
    bad[9] = bad[9][::-1]                                   # not ascending
    with pytest.raises(rl0.Rl0Error):
        rl0.Expander.from_rows(_cuda(bad), I.m)


@pytest.mark.parametrize("sigma_n", [0.0, 1e-3, 0.05])
def test_sketch_matches_oracle(rl0, sigma_n):
    I = gm.instance(5000, 1300, 200, 7, 0.0, 11)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    y = rl0.sketch(A, _cuda(I.x), sigma_n=sigma_n, noise_seed=77).cpu().numpy()
    want = oracle.sketch(I.rows, I.x.astype(np.float64), I.m, sigma_n=sigma_n, noise_seed=77)
    # both sum in FP64 and round once: equal up to the last FP32 bit
    np.testing.assert_allclose(y, want, rtol=2 ** -23, atol=1e-30)
    assert np.mean(y == want.astype(np.float32)) > 0.999


# ------------------------------------------------------------------ one round, injected states
def _states(I, y64, rng):
    A = _A(I.rows, I.m)
    out = []
    xh, _, _ = oracle.decode(I.rows, y64, I.k, sigma_n=I.sigma_n, max_rounds=3)
    out.append(xh)
    for frac_shift, frac_drop, spur in ((0.3, 0.0, 0), (0.2, 0.3, 5), (0.0, 0.6, 0)):
        x = I.x.astype(np.float64).copy()
        s = I.support
        sh = rng.choice(s, int(frac_shift * s.size), replace=False)
        x[sh] += rng.choice([-1, 1], sh.size) * rng.uniform(0.2, 1.0, sh.size)
        x[rng.choice(s, int(frac_drop * s.size), replace=False)] = 0.0
        off = np.setdiff1d(np.arange(I.n), s)
        x[rng.choice(off, spur, replace=False)] = rng.uniform(0.3, 1.0, spur)
        out.append(x)
    states = []
    for x in out:
        x32 = x.astype(np.float32)
        r32 = (y64 - A @ x32.astype(np.float64)).astype(np.float32)
        states.append((x32, r32))
    return states


def _compare_round(rl0, A, I, y32, rows, k, ridx, x32, r32, quantised):
    """One round from (x32, r32) on both sides.  Decisions whose oracle margin is below
    MARGIN may differ; every other decision must agree, and x' and r are compared element
    by element everywhere a differing decision cannot reach: the columns that differ, the
    entries H_k kept on one side only (a differing decision can move H_k's cut), and the
    rows of those columns are left out of the comparison, everything else is checked."""
    y64 = y32.astype(np.float64)
    with oracle.openmp():
        xo, ro, updo, rec = oracle.round_step(rows, y64, k, ridx, x32.astype(np.float64), r32.astype(np.float64),
                                              sigma_n=I.sigma_n, quantised=quantised)
    xg, rg, passed, l1g = rl0.round_step(A, _cuda(y32), k, ridx, _cuda(x32), _cuda(r32), sigma_n=I.sigma_n,
                                         quantised=quantised)
    xg = xg.cpu().numpy().astype(np.float64)
    rg = rg.cpu().numpy().astype(np.float64)
    pg = passed.cpu().numpy().astype(bool)
    po = rec["passed"].astype(bool)
    near = rec["min_margin"] < MARGIN
    flip = np.nonzero(pg != po)[0]
    assert near[flip].all(), flip[~near[flip]][:10]
    # entries whose H_k outcome differs beyond the flipped columns themselves
    hk_only = np.setdiff1d(np.nonzero((xg != 0) != (xo != 0))[0], flip)
    assert hk_only.size <= 2 * flip.size, (flip.size, hk_only.size)
    out = np.union1d(flip, hk_only)
    keep = np.ones(I.n, bool)
    keep[out] = False
    assert np.array_equal(xg[keep] != 0, xo[keep] != 0)
    assert _rel(xg[keep], xo[keep]) <= XTOL
    Aabs = _A(rows, I.m)
    rows_out = np.zeros(I.m, bool)
    if out.size:
        rows_out[np.unique(rows[out].ravel())] = True
    # FP32 row sum (a few terms) plus what the FP32 consensus values in x' carry over
    scale = np.abs(y64) + Aabs @ np.abs(xo)
    ok_r = np.abs(rg - ro) <= 4 * scale * 2 ** -24 + Aabs @ np.abs(np.where(keep, xg - xo, 0.0)) + 1e-30
    assert np.all(ok_r[~rows_out])
    if flip.size == 0:
        assert l1g == pytest.approx(np.abs(ro).sum(), rel=1e-6)
    return int(near.sum()), int(po.sum()), int(near.size)


@pytest.mark.parametrize("quantised", [False, True])
@pytest.mark.parametrize("cfg", [dict(n=4096, m=1024, k=100, d=7, sigma_n=1e-3),
                                 dict(n=5000, m=1300, k=120, d=7, sigma_n=1e-2),
                                 dict(n=3001, m=900, k=60, d=15, sigma_n=5e-3)])
def test_round_step_matches_oracle(rl0, quantised, cfg):
    I, y32 = _problem(seed=21, **cfg)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    rng = np.random.default_rng(0)
    c = oracle.default_c(quantised, I.m / I.n, I.k / I.m)
    total_near = total_pass = total_cols = 0
    for x32, r32 in _states(I, y32.astype(np.float64), rng):
        for ridx in (1, int(0.3 / c), int(0.8 / c)):
            nr, np_, nc = _compare_round(rl0, A, I, y32, I.rows, I.k, ridx, x32, r32, quantised)
            total_near += nr
            total_pass += np_
            total_cols += nc
    assert total_pass > 20
    # rounding-sensitive decisions (excluded from the exact comparison) must be rare
    assert total_near <= 2 + total_cols // 1000


def test_round_step_hk_drops_with_ties(rl0):
    # a state with many equal magnitudes forces H_k to break ties by index
    I, y32 = _problem(2000, 600, 40, 7, 1e-3, 3)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    x = np.zeros(I.n, np.float32)
    x[np.arange(0, 2000, 7)] = 0.5
    x[np.arange(3, 2000, 11)] = -0.5
    r = (y32.astype(np.float64) - _A(I.rows, I.m) @ x.astype(np.float64)).astype(np.float32)
    for q in (False, True):
        _compare_round(rl0, A, I, y32, I.rows, I.k, 5, x, r, q)


# ------------------------------------------------------------------ whole decode
def _decode_both(rl0, I, y32, **kw):
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    xg, st = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n, **kw)
    xo, sto, logo = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, **kw)
    return A, xg.cpu().numpy().astype(np.float64), st, xo, sto, logo


@pytest.mark.parametrize("quantised", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_decode_small_config_matches_oracle(rl0, quantised, seed):
    I, y32 = _problem(seed=seed, **gm.config_small())
    A, xg, st, xo, sto, logo = _decode_both(rl0, I, y32, quantised=quantised)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["rounds"] == sto["rounds"]
    assert st["accepted_rounds"] == sto["accepted_rounds"]
    assert st["converged"] == sto["converged"]
    assert st["support_size"] == np.count_nonzero(xo)
    r = y32.astype(np.float64) - _A(I.rows, I.m) @ xg
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)
    log = rl0.decode_log(A)
    assert [e["accepted"] for e in log] == [e["accepted"] for e in logo]
    assert [e["updated"] for e in log] == [e["updated"] for e in logo]


@pytest.mark.parametrize("cfg", [dict(n=5003, m=1201, k=110, d=7, sigma_n=2e-3),      # ragged tail
                                 dict(n=4100, m=1100, k=90, d=6, sigma_n=1e-3),        # paired FP16 bound, d = 6
                                 dict(n=4100, m=1100, k=70, d=8, sigma_n=1e-3),        # paired FP16 bound, d = 8
                                 dict(n=20000, m=3000, k=250, d=15, sigma_n=1e-3),     # d = 15
                                 dict(n=6000, m=1500, k=100, d=20, sigma_n=1e-3),      # d > 16
                                 dict(n=3000, m=900, k=60, d=7, sigma_n=0.0)])         # noiseless
@pytest.mark.parametrize("quantised", [False, True])
def test_decode_other_shapes_match_oracle(rl0, cfg, quantised):
    I, y32 = _problem(seed=4, **cfg)
    A, xg, st, xo, sto, _ = _decode_both(rl0, I, y32, quantised=quantised)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["accepted_rounds"] == sto["accepted_rounds"]


@pytest.mark.parametrize("d", [7, 5])
@pytest.mark.parametrize("quantised", [False, True])
def test_decode_with_saturated_codes_matches_oracle(rl0, d, quantised):
    # sigma_s = 3e4: some residuals exceed the largest FP16 magnitude (65504), so the
    # column kernel cannot bound their columns from the 16-bit codes and takes every
    # anchor of such a column to the exact test (d = 7: the paired FP16 bound; d = 5:
    # the scalar one).  The decode must be the oracle's all the same.
    I, y32 = _problem(4096, 1024, 80, d, 30.0, 9, sigma_s=3e4)
    assert np.abs(y32).max() > 65504
    A, xg, st, xo, sto, _ = _decode_both(rl0, I, y32, quantised=quantised, sigma_s=3e4)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["accepted_rounds"] == sto["accepted_rounds"]
    assert st["accepted_rounds"] > 0


def test_decode_edge_cases(rl0):
    I, y32 = _problem(800, 200, 10, 5, 1e-3, 8)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    # y = 0: already converged, x_hat = 0
    x, st = rl0.decode(A, torch.zeros(I.m, device="cuda"), I.k, sigma_n=1e-3)
    assert st["rounds"] == 0 and st["converged"] == 1 and not x.any()
    # k = 1 and k = n
    for k in (1, I.n):
        xg, st = rl0.decode(A, _cuda(y32), k, sigma_n=I.sigma_n)
        xo, sto, _ = oracle.decode(I.rows, y32.astype(np.float64), k, sigma_n=I.sigma_n)
        assert np.array_equal(np.nonzero(xg.cpu().numpy())[0], np.nonzero(xo)[0])
        assert np.count_nonzero(xg.cpu().numpy()) <= k
    # invalid inputs are errors, not crashes
    with pytest.raises(rl0.Rl0Error):
        rl0.decode(A, _cuda(y32), 0, sigma_n=1e-3)
    with pytest.raises(rl0.Rl0Error):
        rl0.decode(A, _cuda(y32), I.k, sigma_n=-1.0)
    bad = y32.copy()
    bad[3] = np.nan
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode(A, _cuda(bad), I.k, sigma_n=1e-3)
    assert e.value.code == -7


def test_decode_is_deterministic_and_host_api_agrees(rl0):
    I, y32 = _problem(seed=6, **gm.config_small())
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    x1, _ = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n)
    x2, _ = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n)
    x3, _ = rl0.decode_host(A, torch.from_numpy(y32), I.k, sigma_n=I.sigma_n)
    assert torch.equal(x1, x2)
    assert torch.equal(x1.cpu(), x3)
    # a different stream gives the same bits
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x4, _ = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n, stream=s)
    s.synchronize()
    assert torch.equal(x1, x4)


# ------------------------------------------------------------------ full size (n = 2^20)
def test_full_size_round_and_decode_properties(rl0):
    cfg = gm.config_large()
    I, y32 = _problem(seed=0, **cfg)
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    y64 = y32.astype(np.float64)
    # one round from a perturbed-truth state, compared with the oracle column by column
    rng = np.random.default_rng(1)
    x = I.x.astype(np.float64).copy()
    sh = rng.choice(I.support, I.k // 4, replace=False)
    x[sh] += rng.uniform(0.2, 1.0, sh.size)
    x[rng.choice(I.support, I.k // 4, replace=False)] = 0.0
    x32 = x.astype(np.float32)
    r32 = (y64 - _A(I.rows, I.m) @ x32.astype(np.float64)).astype(np.float32)
    for q in (False, True):
        c = oracle.default_c(q, I.m / I.n, I.k / I.m)
        nr, npass, ncols = _compare_round(rl0, A, I, y32, I.rows, I.k, int(0.5 / c), x32, r32, q)
        print("\nn=2^20 round (%s): %d passing columns, %d decisions within the margin %.0e"
              % ("quantised" if q else "continuous", npass, nr, MARGIN))
        assert npass > 1000 and nr <= 2 + ncols // 1000
    # the whole decode in the benchmark's configuration: invariants at full size
    xg, st = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n)
    xg = xg.cpu().numpy().astype(np.float64)
    assert np.count_nonzero(xg) <= I.k
    r = y64 - _A(I.rows, I.m) @ xg
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)
    xl1 = np.abs(I.x).sum()
    tol = min((I.m * I.sigma_n * math.sqrt(2 / math.pi) + math.sqrt(I.m * I.sigma_n ** 2 * (1 - 2 / math.pi))) / xl1,
              0.1)
    assert np.abs(xg - I.x).sum() / xl1 <= tol


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_largest_score_anchor_rule_matches_oracle(rl0, seed):
    """The other reading of Alg. 2's per-anchor update (anchor_rule = 1: a column takes the
    passing anchor of largest n_e - n_z, ties to the lower row) against the oracle's
    best_anchor flag, quantised scores (integer n_e - n_z, so the choice is exact on both
    sides).  The batched decoder and the static entry reject it."""
    I, y32 = _problem(seed=seed, **gm.config_small())
    A = rl0.Expander.from_rows(_cuda(I.rows), I.m)
    xg, st = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n, quantised=True, anchor_rule=1)
    xo, sto, _ = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, quantised=True,
                               best_anchor=True)
    xg = xg.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert _rel(xg, xo) <= XTOL
    assert st["rounds"] == sto["rounds"] and st["accepted_rounds"] == sto["accepted_rounds"]
    # the default reading on the same expander afterwards is unaffected
    x0, _ = rl0.decode(A, _cuda(y32), I.k, sigma_n=I.sigma_n, quantised=True)
    xo0, _, _ = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, quantised=True)
    assert np.array_equal(np.nonzero(x0.cpu().numpy())[0], np.nonzero(xo0)[0])
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_batched([A], [_cuda(y32)], [I.k], [dict(sigma_n=I.sigma_n, anchor_rule=1)])
    assert e.value.code == -5
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_static(A, _cuda(y32), I.k, sigma_n=I.sigma_n, anchor_rule=1)
    assert e.value.code == -5
