"""Whole-decode parity at the sizes the benchmark measures, against the FP64 oracle (its
OpenMP build: the same results as the serial one, in seconds at n = 2^20).

  - the plain decode at n = 2^20, m = 104857, k = 10485, d = 7, SNR 40 dB (continuous and
    quantised scores), on the generator's seed-0 instance and on the benchmark's instance
    (expander seed 1000, signal seed 1000, noise seed 1001; y_hat from the oracle's sketch);
  - the batched decoder at the largest shapes of the batched workload (n = 2^16,
    delta = 0.3, m = 19660), bitwise against the single decode and against the oracle.

Bars: identical support, ||x_gpu - x_orc||_2 / ||x_orc||_2 <= 1e-5, identical round counts
and per-round accept/update logs.  One exception, for the quantised scores only: their
q_e test is a hard threshold |D| <= t_e on residual differences, and in the sweep's last
rounds (t near 0) thousands of columns pass and H_k cuts among magnitudes that lie closer
together than FP32 residuals can resolve, so a decision within rounding of its threshold
can go the other way here than in FP64.  Such an instance must differ only in the way
_compare_decode describes, and must agree everywhere else."""
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


def _bench_instance():
    """The benchmark's instance: the library's generator draws the same expander as the
    oracle's (Philox4x32-10, seed 1000); the signal comes from the generator module."""
    cfg = gm.config_large()
    n, m, k, d, sn = cfg["n"], cfg["m"], cfg["k"], cfg["d"], cfg["sigma_n"]
    rows = oracle.make_expander(n, m, d, 1000)
    x, _ = gm.draw_signal(n, k, 1.0, 1000)
    y = oracle.sketch(rows, x.astype(np.float64), m, sigma_n=sn, noise_seed=1001)
    return rows, x, y.astype(np.float32), cfg


def _seed0_instance():
    cfg = gm.config_large()
    I = gm.instance(seed=0, **cfg)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), I.m) + I.eta.astype(np.float64)
    return I.rows, I.x, y.astype(np.float32), cfg


@pytest.mark.parametrize("which", ["seed0", "bench"])
@pytest.mark.parametrize("quantised", [False, True])
def test_full_size_decode_matches_oracle(rl0, which, quantised):
    rows, x, y32, cfg = _seed0_instance() if which == "seed0" else _bench_instance()
    m, k, sn = cfg["m"], cfg["k"], cfg["sigma_n"]
    A = rl0.Expander.from_rows(torch.from_numpy(rows).cuda(), m)
    xg, st = rl0.decode(A, torch.from_numpy(y32).cuda(), k, sigma_n=sn, quantised=quantised)
    log = rl0.decode_log(A)
    with oracle.openmp():
        xo, so, lo = oracle.decode(rows, y32.astype(np.float64), k, sigma_n=sn, quantised=quantised)
    xg = xg.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print("\n%s %s: rounds %d/%d accepted %d/%d support %d rel_l2 %.2e" % (
        which, "quantised" if quantised else "continuous", st["rounds"], so["rounds"], st["accepted_rounds"],
        so["accepted_rounds"], st["support_size"], rel))
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert rel <= XTOL
    assert st["rounds"] == so["rounds"] and st["accepted_rounds"] == so["accepted_rounds"]
    assert st["converged"] == so["converged"]
    assert [e["accepted"] for e in log] == [e["accepted"] for e in lo]
    assert [e["updated"] for e in log] == [e["updated"] for e in lo]
    r = y32.astype(np.float64) - _A(rows, m) @ xg
    assert st["final_l1"] == pytest.approx(np.abs(r).sum(), rel=1e-12)
    # and the decode recovers x (success condition of Section "Stopping conditions")
    xl1 = np.abs(x).sum()
    tol = min((m * sn * math.sqrt(2 / math.pi) + math.sqrt(m * sn * sn * (1 - 2 / math.pi))) / xl1, 0.1)
    assert np.abs(xg - x).sum() / xl1 <= tol


def _largest_batched_shapes(count, seed):
    """n = 2^16, delta = 0.3 (m = 19660): the top of the batched workload's ranges, with
    rho and SNR drawn from the workload's ranges."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n, d = 1 << 16, 7
        m = int(math.floor(0.3 * n))
        rho = float(rng.uniform(0.05, 0.2))
        k = int(math.floor(rho * m))
        sn = gm.sigma_from_snr(d, k / m, float(rng.uniform(30.0, 60.0)))
        I = gm.instance(n, m, k, d, sn, 7000 + i)
        y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
        out.append((I, y.astype(np.float32)))
    return out


@pytest.mark.parametrize("quantised", [False, True])
def test_batched_largest_shapes_match_single_decode_and_oracle(rl0, quantised):
    insts = _largest_batched_shapes(6, 11)
    # with smaller instances beside them, as in the workload
    rng = np.random.default_rng(5)
    for i in range(10):
        n = int(rng.integers(1 << 10, (1 << 16) + 1))
        m = int(math.floor(float(rng.uniform(0.1, 0.3)) * n))
        k = max(int(math.floor(float(rng.uniform(0.05, 0.2)) * m)), 1)
        sn = gm.sigma_from_snr(7, k / m, float(rng.uniform(30.0, 60.0)))
        I = gm.instance(n, m, k, 7, sn, 7100 + i)
        y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
        insts.append((I, y.astype(np.float32)))
    As = [rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m) for I, _ in insts]
    ys = [torch.from_numpy(y).cuda() for _, y in insts]
    params = [dict(sigma_n=I.sigma_n, quantised=quantised) for I, _ in insts]
    xs, stats = rl0.decode_batched(As, ys, [I.k for I, _ in insts], params)
    exact = 0
    for i, (A, y, p, xb, sb, (I, y32)) in enumerate(zip(As, ys, params, xs, stats, insts)):
        x1, s1 = rl0.decode(A, y, I.k, **p)
        assert torch.equal(xb, x1), (I.n, I.m, I.k)
        assert sb["rounds"] == s1["rounds"] and sb["final_l1"] == s1["final_l1"]
        if i < 6:                                        # the largest shapes, against the oracle
            exact += _compare_decode(I, y32, xb.cpu().numpy().astype(np.float64), sb, rl0.decode_log(A),
                                     quantised)
    print("\nlargest batched shapes (%s): %d of 6 identical to the oracle"
          % ("quantised" if quantised else "continuous", exact))
    # continuous scores have no hard thresholds: every instance must be identical
    assert exact == 6 or (quantised and exact >= 4)


def _near_columns_per_round(I, y64, quantised, nrounds):
    """The oracle's own trajectory replayed round by round: per round, the columns whose
    decision lies within MARGIN of its threshold (inputs from the oracle alone)."""
    xh, rh = np.zeros(I.n), y64.copy()
    out = []
    with oracle.openmp():
        for r in range(nrounds):
            xp, rp, _, rec = oracle.round_step(I.rows, y64, I.k, r, xh, rh, sigma_n=I.sigma_n, quantised=quantised)
            out.append(np.nonzero(rec["min_margin"] < MARGIN)[0])
            if np.abs(rp).sum() < np.abs(rh).sum():
                xh, rh = xp, rp
    return out


def _compare_decode(I, y32, xg, st, log, quantised):
    """Whole decode against the oracle.  Returns 1 if identical (support, x_hat to XTOL,
    rounds, per-round logs).  Otherwise the difference must be one that rounding can
    cause, and the rest must agree: the logs equal up to the first round r* where they
    differ; r* holds decisions within MARGIN of their threshold in the oracle's own
    trajectory (a quantised q_e test |D| <= t_e or the l1 test, decided on FP32 values
    here and FP64 values there), and its update counts differ by at most their number;
    when r* is the decode's last round, x_hat agrees to XTOL on the columns both keep and
    the columns kept by one side only are at most twice that number (H_k's cut takes the
    next candidate in place of one that was not updated).  Returns 0 then."""
    y64 = y32.astype(np.float64)
    with oracle.openmp():
        xo, so, lo = oracle.decode(I.rows, y64, I.k, sigma_n=I.sigma_n, quantised=quantised)
    same_log = [(e["accepted"], e["updated"], e["support"]) for e in log] == \
               [(e["accepted"], e["updated"], e["support"]) for e in lo]
    if (np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0]) and same_log and st["rounds"] == so["rounds"]
            and np.linalg.norm(xg - xo) <= XTOL * max(np.linalg.norm(xo), 1e-30)):
        return 1
    assert quantised, "continuous scores must match the oracle exactly"
    rstar = next(r for r in range(min(len(log), len(lo)) + 1)
                 if r == min(len(log), len(lo)) or (log[r]["accepted"], log[r]["updated"], log[r]["support"]) !=
                 (lo[r]["accepted"], lo[r]["updated"], lo[r]["support"]))
    assert rstar < len(lo), "the logs agree but the results differ"
    near = _near_columns_per_round(I, y64, quantised, rstar + 1)[rstar]
    assert near.size > 0, "round %d differs without a near-threshold decision" % rstar
    assert abs(log[rstar]["updated"] - lo[rstar]["updated"]) <= near.size
    if rstar == len(lo) - 1 and len(log) == len(lo):
        both = (xg != 0) & (xo != 0)
        only = np.nonzero((xg != 0) != (xo != 0))[0]
        assert only.size <= 2 * near.size
        assert np.linalg.norm(xg[both] - xo[both]) <= XTOL * np.linalg.norm(xo[both])
    print("  n=%d m=%d k=%d: differs from round %d of %d (%d near-threshold decisions there)"
          % (I.n, I.m, I.k, rstar, len(lo), near.size))
    return 0


def test_full_size_adaptive_decode_matches_oracle(rl0):
    """adaptive_k on the benchmark's instance (Section "Adaptive k"): the GPU's sequence of
    priors, accepts and updates round by round is the oracle's, and so is its outcome --
    here both stop improving after six accepted rounds, with the prior at its floor
    m/100, 0.1% above the stop level, and sweep to t <= 0 without converging.  (Every
    round's n_z must use p_z under that round's prior: this test is what found p_z of
    r_hat left at the previous prior.)"""
    rows, x, y32, cfg = _bench_instance()
    m, k, sn = cfg["m"], cfg["k"], cfg["sigma_n"]
    A = rl0.Expander.from_rows(torch.from_numpy(rows).cuda(), m)
    xg, st = rl0.decode(A, torch.from_numpy(y32).cuda(), k, sigma_n=sn, adaptive_k=True)
    log = rl0.decode_log(A)
    with oracle.openmp():
        xo, so, lo = oracle.decode(rows, y32.astype(np.float64), k, sigma_n=sn, adaptive_k=True)
    xg = xg.cpu().numpy().astype(np.float64)
    print("\nadaptive n=2^20: rounds %d/%d accepted %d/%d converged %d/%d final_l1 %.6g/%.6g" % (
        st["rounds"], so["rounds"], st["accepted_rounds"], so["accepted_rounds"], st["converged"], so["converged"],
        st["final_l1"], so["final_l1"]))
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert np.linalg.norm(xg - xo) <= XTOL * np.linalg.norm(xo)
    assert st["rounds"] == so["rounds"] and st["accepted_rounds"] == so["accepted_rounds"]
    assert st["converged"] == so["converged"]
    assert [(e["accepted"], e["updated"]) for e in log] == [(e["accepted"], e["updated"]) for e in lo]
    # k0 is summed from FP32 x_hat here and from FP64 x_hat in the oracle
    for e, f in zip(log, lo):
        assert e["k_prior"] == pytest.approx(f["k_prior"], rel=1e-7)
