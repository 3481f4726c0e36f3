"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer values, closed forms printed in the paper, Monte-Carlo draws of
the paper's generating model, library routines, brute force and the ground-truth signal.
A plausible mistake anywhere in the oracle (a dropped term, a wrong variance, a wrong
sign or index, a transposed operand) fails at least one test here."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _A(rows, m):
    n, d = rows.shape
    return sp.csr_matrix((np.ones(n * d), (rows.ravel(), np.repeat(np.arange(n), d))), shape=(m, n))


# ---------------------------------------------------------------- generator
def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        assert list(oracle.philox(w[0:4], w[4:6])) == w[6:10]


def test_make_expander_is_uniform_d_subsets():
    n, m, d = 20000, 500, 7
    rows = oracle.make_expander(n, m, d, seed=3)
    assert rows.shape == (n, d)
    assert np.all(np.diff(rows, axis=1) > 0)            # sorted and distinct
    assert rows.min() >= 0 and rows.max() < m
    # every row index equally likely: chi-square of the row histogram
    h = np.bincount(rows.ravel(), minlength=m)
    e = n * d / m
    chi2 = ((h - e) ** 2 / e).sum()
    assert abs(chi2 - (m - 1)) < 6 * math.sqrt(2 * (m - 1))
    # pairs within a column are uniform too: P(rows 0 and 1 of a column both used)
    both = np.sum(np.any(rows == 0, axis=1) & np.any(rows == 1, axis=1))
    p = d * (d - 1) / (m * (m - 1))
    assert abs(both - n * p) < 6 * math.sqrt(n * p) + 1
    # deterministic in the seed, different across seeds
    assert np.array_equal(rows, oracle.make_expander(n, m, d, seed=3))
    assert not np.array_equal(rows, oracle.make_expander(n, m, d, seed=4))


def test_noise_l1_moments_match_paper():
    # Section "Stopping conditions": E||eta||_1 = m sigma sqrt(2/pi),
    # Var||eta||_1 = m sigma^2 (1 - 2/pi) for eta ~ N(0, sigma^2 I).
    m, sigma = 2000, 0.01
    l1 = np.array([np.abs(oracle.noise(m, sigma, seed)).sum() for seed in range(300)])
    mean = m * sigma * math.sqrt(2 / math.pi)
    var = m * sigma ** 2 * (1 - 2 / math.pi)
    assert abs(l1.mean() - mean) < 5 * math.sqrt(var / l1.size)
    assert abs(l1.var(ddof=1) / var - 1) < 0.35
    z = oracle.noise(200000, 1.0, 11)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.1                 # Gaussian kurtosis


def test_matvec_matches_sparse_library():
    I = gm.instance(3000, 700, 90, 7, 0.0, seed=5)
    x = I.x.astype(np.float64)
    np.testing.assert_allclose(oracle.matvec(I.rows, x, I.m), _A(I.rows, I.m) @ x, rtol=0, atol=1e-12)


def test_probability_of_a_zero_row():
    # Lemma "sparse sums" and Thm "distribution of y_i": P(y_i = 0) -> exp(-d rho).
    # At finite size every support column misses row i independently: (1 - d/m)^k.
    n, m, d = 1 << 16, 1 << 14, 7
    for rho in (0.05, 0.2):
        k = int(rho * m)
        zeros = 0
        for seed in range(4):
            I = gm.instance(n, m, k, d, 0.0, seed=seed)
            zeros += np.sum(oracle.matvec(I.rows, I.x.astype(np.float64), m) == 0.0)
        N = 4 * m
        p_fin = (1 - d / m) ** k
        assert abs(zeros / N - p_fin) < 5 * math.sqrt(p_fin * (1 - p_fin) / N)
        assert abs(p_fin - math.exp(-d * rho)) < 2e-3


# ---------------------------------------------------------------- posteriors
def test_tail_constants_match_their_defining_sums():
    # R(ell) = sum_{q>ell} lam^q/q!, v_tail = sum_{q>ell} w_q (q s^2 + v_n) / R(ell)
    for which, lam_mult, vmult in (("z", 1, 1), ("e", 2, 2)):
        for d, rho, ss, sn, ell in ((7, 0.1, 1.0, 1e-3, 4), (15, 0.3, 2.0, 0.05, 2), (7, 0.02, 1.0, 0.01, 1)):
            R, v = oracle.tail_constants(which, d, rho, ss, sn, ell)
            lam = lam_mult * d * rho
            w = [lam ** q / math.factorial(q) for q in range(ell + 1, 150)]
            vq = [q * ss ** 2 + vmult * sn ** 2 for q in range(ell + 1, 150)]
            R_def = math.fsum(w)
            assert R == pytest.approx(R_def, rel=1e-12)
            assert R == pytest.approx(math.exp(lam) - sum(lam ** q / math.factorial(q) for q in range(ell + 1)),
                                      rel=1e-9)
            assert v == pytest.approx(math.fsum(a * b for a, b in zip(w, vq)) / R_def, rel=1e-12)


@pytest.mark.parametrize("which", ["z", "e"])
def test_normalised_posterior_peaks_at_zero_and_is_monotone(which):
    w = np.linspace(0, 0.2, 4001)
    for sn in (1e-3, 1e-2):
        lp = oracle.log_posterior(which, w, 7, 0.1, 1.0, sn)
        assert lp[0] == 0.0
        assert np.all(np.diff(lp) <= 1e-15)
        assert np.all(lp <= 0.0)
        np.testing.assert_array_equal(lp, oracle.log_posterior(which, -w, 7, 0.1, 1.0, sn))


@pytest.mark.parametrize("which", ["z", "e"])
def test_tail_approximation_converges_to_the_full_series(which):
    w = np.linspace(-0.05, 0.05, 201)
    exact = oracle.log_posterior(which, w, 7, 0.2, 1.0, 1e-2, ell=400, exact=True)
    errs = [np.max(np.abs(oracle.log_posterior(which, w, 7, 0.2, 1.0, 1e-2, ell=l) - exact)) for l in (1, 2, 4, 8, 30)]
    assert all(b <= a + 1e-15 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12


def test_posterior_is_one_without_signal():
    # d rho -> 0: no row holds signal, so y_i = 0 and y_i1 = y_i2 for certain.
    w = np.linspace(-0.06, 0.06, 51)
    for which in ("z", "e"):
        _, raw = oracle.log_posterior(which, w, 7, 1e-40, 1.0, 1e-2, raw=True)
        np.testing.assert_allclose(raw, 0.0, atol=1e-9)


def _binned_check(obs_equal, omega, logp_raw, edges, min_count=60):
    """Empirical P(event | omega in bin) against the mean model probability in the bin."""
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (np.abs(omega) >= lo) & (np.abs(omega) < hi)
        N = int(sel.sum())
        if N < min_count:
            continue
        emp = obs_equal[sel].mean()
        pred = np.exp(logp_raw[sel]).mean()
        sd = math.sqrt(max(pred * (1 - pred), 1e-4) / N)
        assert abs(emp - pred) < 5 * sd + 0.02, (lo, hi, N, emp, pred)
        checked += 1
    return checked


@pytest.mark.parametrize("rho,sigma", [(0.1, 1e-3), (0.3, 1e-3), (0.1, 1e-2), (0.3, 1e-2)])
def test_posteriors_against_monte_carlo_of_the_model(rho, sigma):
    # The paper's own check (Section "Comparison with empirical probabilities"):
    # GM(n, 0.3 n, rho 0.3 n, 7, N(0,1), N(0, sigma^2)) against Eqs. (pz_approx), (pe_approx).
    n, d = 1 << 16, 7
    m = int(0.3 * n)
    k = int(rho * m)
    ys, yhs = [], []
    for seed in range(6):
        I = gm.instance(n, m, k, d, sigma, seed=100 + seed)
        y = _A(I.rows, m) @ I.x.astype(np.float64)
        ys.append(y)
        yhs.append(y + I.eta.astype(np.float64))
    y = np.concatenate(ys)
    yh = np.concatenate(yhs)
    edges = sigma * np.array([0, 0.5, 1, 1.5, 2, 2.5, 3, 3.5, 4, 5, 6, 8])
    _, raw_z = oracle.log_posterior("z", yh, d, k / m, 1.0, sigma, raw=True)
    assert _binned_check(y == 0.0, yh, raw_z, edges) >= 5
    rng = np.random.default_rng(0)
    i1 = rng.integers(0, y.size, 4 * y.size)
    i2 = rng.integers(0, y.size, 4 * y.size)
    keep = (i1 != i2) & (i1 // m == i2 // m)              # pairs within one instance
    i1, i2 = i1[keep], i2[keep]
    dlt = yh[i1] - yh[i2]
    _, raw_e = oracle.log_posterior("e", dlt, d, k / m, 1.0, sigma, raw=True)
    assert _binned_check(y[i1] == y[i2], dlt, raw_e, math.sqrt(2) * edges) >= 5


# ---------------------------------------------------------------- decoder pieces
def test_default_c_matches_printed_rule():
    for line in open(os.path.join(GOLDEN, "finetune_c.txt")):
        if line.startswith("#") or not line.strip():
            continue
        q, delta, rho, c = line.split()
        assert oracle.default_c(int(q), float(delta), float(rho)) == pytest.approx(float(c))


def test_number_of_rounds_of_the_sweep():
    # t = 1, 1-c, 1-2c, ... while t > 0
    for c, r in ((0.01, 100), (0.025, 40), (0.05, 20), (0.075, 14), (0.1, 10), (0.3, 4)):
        assert oracle.num_rounds(c) == r
        assert all(1 - i * c > 1e-12 for i in range(r)) and 1 - r * c <= 1e-12


def test_hard_threshold_matches_lexsort():
    rng = np.random.default_rng(1)
    for trial in range(50):
        n = int(rng.integers(1, 400))
        x = rng.standard_normal(n) * (rng.random(n) < 0.5)
        if trial % 3 == 0:                        # planted magnitude ties
            x[rng.integers(0, n, n // 3)] = rng.choice([-0.5, 0.5])
        k = int(rng.integers(1, n + 1))
        got = oracle.hard_threshold(x, k)
        nz = np.nonzero(x)[0]
        keep = nz[np.lexsort((nz, -np.abs(x[nz])))][:k]
        want = np.zeros(n)
        want[keep] = x[keep]
        np.testing.assert_array_equal(got, want)


def _instance(cfg, seed, f32=True):
    I = gm.instance(seed=seed, **cfg)
    y = _A(I.rows, I.m) @ I.x.astype(np.float64) + I.eta.astype(np.float64)
    if f32:
        y = y.astype(np.float32).astype(np.float64)
    return I, y


def test_stop_level_is_the_noise_l1_the_model_leaves():
    # Section "Stopping conditions": a decode stops once ||r_hat||_1 is at the level the
    # noise alone leaves, E||eta||_1; against the mean of ||eta||_1 over noise draws of
    # the generator (not the moment formula), within 1% (the mean's std is about 0.2%).
    cfg = gm.config_small()
    I, y = _instance(cfg, 0)
    _, st, _ = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n)
    l1 = np.mean([np.abs(gm.draw_noise(I.m, I.sigma_n, 5000 + s).astype(np.float64)).sum() for s in range(400)])
    assert st["stop_level"] == pytest.approx(l1, rel=0.01)
    assert st["converged"] == int(st["final_l1"] <= st["stop_level"])


def test_round_at_t_equal_one_updates_nothing_with_noise():
    # reading: 1 - p_z(r) >= 1 needs p_z(r) = 0, which never holds for sigma_n > 0
    I, y = _instance(gm.config_small(), 0)
    for q in (False, True):
        xp, rp, upd, rec = oracle.round_step(I.rows, y, I.k, 0, np.zeros(I.n), y, sigma_n=I.sigma_n, quantised=q)
        assert upd == 0 and not xp.any()


def test_noiseless_quantised_follows_parallel_l0_and_recovers_x():
    # Noiseless: the quantised scores become the equality/zero indicators of Alg. 1, so
    # each accepted round of Alg. 2 is one iteration of Alg. 1, and both return x exactly
    # (Thm "convergence of Algorithm 1").
    n, m, d = 4096, 1024, 7
    for seed in range(3):
        I, y = _instance(dict(n=n, m=m, k=60, d=d, sigma_n=0.0), seed, f32=False)
        xr, st, log = oracle.decode(I.rows, y, I.k, sigma_n=0.0, quantised=True, noiseless_tol=1e-9)
        xp, it, hist = oracle.parallel_l0(I.rows, y, tol=1e-9, history=True)
        np.testing.assert_allclose(xr, I.x, atol=1e-9)
        np.testing.assert_allclose(xp, I.x, atol=1e-9)
        assert st["converged"] == 1
        assert it <= 2 + 2 * math.ceil(math.log2(I.k))           # O(log k) iterations
        # accepted rounds of Alg. 2 reproduce the iterates of Alg. 1 one by one
        acc = [r for r in log if r["accepted"]]
        assert len(acc) == it
        for a, h in zip(acc, hist):
            assert a["support"] == np.count_nonzero(h)


def _brute_force_sparsest(A, y, kmax):
    n = A.shape[1]
    for s in range(0, kmax + 1):
        sols = []
        for S in itertools.combinations(range(n), s):
            if s == 0:
                if np.allclose(y, 0):
                    sols.append(np.zeros(n))
                continue
            cols = A[:, S]
            coef, *_ = np.linalg.lstsq(cols, y, rcond=None)
            if np.allclose(cols @ coef, y, atol=1e-10) and np.all(np.abs(coef) > 1e-9):
                x = np.zeros(n)
                x[list(S)] = coef
                sols.append(x)
        if sols:
            return sols
    return []


def test_noiseless_decode_finds_the_unique_sparsest_solution_on_tiny_problems():
    rng = np.random.default_rng(7)
    converged = agreed = 0
    for trial in range(150):
        n = int(rng.integers(8, 21))
        m = int(rng.integers(5, 11))
        d = int(rng.integers(2, 4))
        k = int(rng.integers(1, 3))
        I = gm.instance(n, m, k, d, 0.0, seed=1000 + trial)
        A = _A(I.rows, m).toarray()
        y = A @ I.x.astype(np.float64)
        x, st, _ = oracle.decode(I.rows, y, k, sigma_n=0.0, quantised=True, noiseless_tol=1e-9)
        sols = _brute_force_sparsest(A, y, k)
        if st["converged"]:
            converged += 1
            assert np.allclose(A @ x, y, atol=1e-9)
            assert np.count_nonzero(x) <= k
            if len(sols) == 1:
                np.testing.assert_allclose(x, sols[0], atol=1e-9)
                agreed += 1
    assert converged >= 60 and agreed >= 40


@pytest.mark.parametrize("quantised", [False, True])
def test_decode_invariants_and_recovery_on_small_config(quantised):
    cfg = gm.config_small()
    for seed in range(3):
        I, y = _instance(cfg, seed)
        x, st, log = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
        A = _A(I.rows, I.m)
        r = y - A @ x
        assert np.abs(r).sum() == pytest.approx(st["final_l1"], rel=1e-12)     # r_hat = y - A x_hat
        l1 = [e["l1_hat"] for e in log]
        assert all(b <= a for a, b in zip(l1, l1[1:]))                     # ||r_hat||_1 non-increasing
        assert np.count_nonzero(x) <= I.k                                   # |supp x_hat| <= k
        # success condition (clipped), C_1 = 1, Section "Stopping conditions"
        m, s = I.m, I.sigma_n
        xl1 = np.abs(I.x).sum()
        tol = min((m * s * math.sqrt(2 / math.pi) + math.sqrt(m * s * s * (1 - 2 / math.pi))) / xl1, 0.1)
        assert np.abs(x - I.x).sum() / xl1 <= tol


def _perturbed_states(I, y, rng):
    """Injected states (x_hat, r_hat = y - A x_hat) near the truth: some support entries
    shifted, some dropped, some spurious entries added."""
    A = _A(I.rows, I.m)
    out = []
    for frac_shift, frac_drop, n_spur in ((0.3, 0.0, 0), (0.2, 0.3, 3), (0.0, 0.5, 0)):
        xh = I.x.astype(np.float64).copy()
        supp = I.support
        sh = rng.choice(supp, max(1, int(frac_shift * supp.size)), replace=False) if frac_shift else []
        xh[sh] += rng.choice([-1, 1], len(sh)) * rng.uniform(0.2, 1.0, len(sh))
        dr = rng.choice(supp, int(frac_drop * supp.size), replace=False) if frac_drop else []
        xh[dr] = 0.0
        off = np.setdiff1d(np.arange(I.n), supp)
        xh[rng.choice(off, n_spur, replace=False)] = rng.uniform(0.3, 1.0, n_spur)
        out.append((xh, y - A @ xh))
    return out


def _python_round(I, y, xh, rh, t, quantised, alpha):
    """Alg. 2's loop body restated in plain Python for one column at a time."""
    rho = I.k / I.m
    xp = xh.copy()
    for j in range(I.n):
        rl = rh[I.rows[j]]
        lz = oracle.log_posterior("z", rl, I.d, rho, 1.0, I.sigma_n)
        qz = (lz >= math.log(1 - t)).astype(float) if quantised else np.exp(lz)
        best = None
        for s in range(I.d):
            if not lz[s] <= math.log(1 - t):
                continue
            le = oracle.log_posterior("e", rl[s] - rl, I.d, rho, 1.0, I.sigma_n)
            qe = (le >= math.log(t)).astype(float) if quantised else np.exp(le)
            ne, nzv = qe.sum(), qz.sum()
            w = (rl * qe).sum() / ne
            if np.abs(rl - w).sum() <= np.abs(rl).sum() and ne - nzv >= alpha:
                best = (ne - nzv, w)                  # the last passing anchor stands
        if best is not None:
            xp[j] = xh[j] + best[1]
    nz = np.nonzero(xp)[0]
    keep = nz[np.lexsort((nz, -np.abs(xp[nz])))][:I.k]
    xk = np.zeros_like(xp)
    xk[keep] = xp[keep]
    return xk


def test_one_round_matches_a_literal_python_round():
    # A pure-Python restatement of one round: per column, the score of every anchor from
    # the same residual (synchronous update), then H_k and r = y - A x'.  It shares only
    # log_posterior (pinned above against Monte-Carlo) with the C loop.
    cfg = dict(n=600, m=180, k=16, d=5, sigma_n=1e-2)
    I, y = _instance(cfg, 2)
    A = _A(I.rows, I.m)
    rng = np.random.default_rng(5)
    total_upd = 0
    for quantised in (False, True):
        c = oracle.default_c(quantised, I.m / I.n, I.k / I.m)
        alpha = I.d // 2 + 1 if quantised else I.d / 2
        xh0, _, _ = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, quantised=quantised, max_rounds=2)
        states = [(xh0, y - A @ xh0)] + _perturbed_states(I, y, rng)
        for xh, rh in states:
            for ridx in (1, 4, 8):
                t = 1 - ridx * c
                xp_c, rp_c, upd, rec = oracle.round_step(I.rows, y, I.k, ridx, xh, rh, sigma_n=I.sigma_n,
                                                         quantised=quantised)
                total_upd += upd
                xk = _python_round(I, y, xh, rh, t, quantised, alpha)
                np.testing.assert_allclose(xp_c, xk, rtol=1e-12, atol=1e-14)
                np.testing.assert_allclose(rp_c, y - A @ xk, rtol=0, atol=1e-12)
    assert total_upd > 50


@pytest.mark.parametrize("quantised", [False, True])
def test_one_round_corrects_shifted_entries_back_to_the_truth(quantised):
    # Ground truth: with x_hat = x except a few isolated support entries shifted by s_j,
    # the rows of such a column hold -s_j plus noise, the consensus is -s_j, and the
    # round returns x'_j = x_hat_j + w close to x_j (within a few noise std).
    n, m, k, d, sn = 4096, 1024, 24, 7, 1e-3
    I, y = _instance(dict(n=n, m=m, k=k, d=d, sigma_n=sn), 9, f32=False)
    A = _A(I.rows, m)
    rng = np.random.default_rng(3)
    supp = I.support
    # isolated: no row shared with any other support column
    cnt = np.bincount(I.rows[supp].ravel(), minlength=m)
    iso = [j for j in supp if np.all(cnt[I.rows[j]] == 1)]
    assert len(iso) >= 6
    sh = np.array(iso[:6])
    xh = I.x.astype(np.float64).copy()
    xh[sh] += rng.choice([-1, 1], sh.size) * rng.uniform(0.3, 1.0, sh.size)
    c = oracle.default_c(quantised, m / n, k / m)
    xp, rp, upd, rec = oracle.round_step(I.rows, y, k, int(round(0.5 / c)), xh, y - A @ xh,
                                         sigma_n=sn, quantised=quantised)
    np.testing.assert_allclose(xp[sh], I.x[sh], atol=6 * sn)
    others = np.setdiff1d(np.arange(n), sh)
    assert np.count_nonzero(xp[others] != xh[others]) <= 2


@pytest.mark.parametrize("quantised", [False, True])
def test_the_consensus_averages_the_rows_noise(quantised):
    # An isolated support column shifted by s_j has rows -s_j + eta_i, i in N(j).  The
    # update's value is a posterior-weighted mean of those rows (Table "scores"), so
    # x'_j - x_j carries an average of about d noise terms: rms near sigma / sqrt(d),
    # where any single row's value would leave rms sigma.
    n, m, k, d, sn = 20000, 5000, 150, 7, 1e-2
    I, y = _instance(dict(n=n, m=m, k=k, d=d, sigma_n=sn), 31, f32=False)
    A = _A(I.rows, m)
    rng = np.random.default_rng(4)
    supp = I.support
    cnt = np.bincount(I.rows[supp].ravel(), minlength=m)
    iso = np.array([j for j in supp if np.all(cnt[I.rows[j]] == 1)])
    assert iso.size >= 25
    xh = I.x.astype(np.float64).copy()
    xh[iso] += rng.choice([-1, 1], iso.size) * rng.uniform(0.3, 1.0, iso.size)
    c = oracle.default_c(quantised, m / n, k / m)
    xp, _, _, _ = oracle.round_step(I.rows, y, k, int(round(0.5 / c)), xh, y - A @ xh, sigma_n=sn,
                                    quantised=quantised)
    moved = iso[xp[iso] != xh[iso]]
    assert moved.size >= 0.8 * iso.size
    rms = math.sqrt(np.mean((xp[moved] - I.x[moved]) ** 2))
    assert rms < 0.7 * sn, rms / sn


def test_quantised_pair_test_counts_a_pair_when_its_posterior_reaches_t():
    """Table "scores", quantised: a pair (r_s, r_l) counts towards n_e when
    p_e(r_s - r_l) >= t.  Worked case: one column of d = 3 rows whose residuals are
    (a, a + D, a - D), a = 1 far above the noise (every row an anchor, no row a zero:
    p_z is below 1e-6), D where the posterior p_e (pinned against the model by Monte
    Carlo above) equals 0.5, so p_e(2 D) < 0.3.  At t = 0.3 a pair at distance D
    counts (0.5 >= 0.3) and one at 2 D does not: the last anchor in row order, a - D,
    has n_e = 2 (itself and a), n_e - n_z = 2 >= alpha = 2, the l1 test holds, and the
    column takes omega = (a + (a - D)) / 2.  At t = 0.7 no pair counts (0.5 < 0.7):
    every anchor has n_e - n_z = 1 and the column keeps x_j.  Reading the threshold as
    1 - t would give the opposite outcome in both rounds."""
    d, sigma_n = 3, 1e-2
    rows = np.array([[0, 1, 2]], np.int32)
    k, m = 1, 3
    rho = k / m
    # D with p_e(D) = 1/2, by bisection on the (Monte-Carlo-pinned) posterior
    lo, hi = 0.0, 20.0 * sigma_n
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if oracle.log_posterior("e", mid, d, rho, 1.0, sigma_n)[0] > math.log(0.5):
            lo = mid
        else:
            hi = mid
    D = 0.5 * (lo + hi)
    assert 0.5 * sigma_n < D < 10 * sigma_n
    a = 1.0
    r = np.array([a, a + D, a - D])
    assert np.exp(oracle.log_posterior("z", r, d, rho, 1.0, sigma_n)).max() < 1e-6
    assert np.exp(oracle.log_posterior("e", 2 * D, d, rho, 1.0, sigma_n))[0] < 0.3
    y = r.copy()                                         # x_hat = 0: r_hat = y
    c = 0.1
    for t, passes in ((0.3, True), (0.7, False)):
        ridx = int(round((1.0 - t) / c))
        xp, _, upd, rec = oracle.round_step(rows, y, k, ridx, np.zeros(1), r, sigma_n=sigma_n, quantised=True, c=c)
        assert bool(rec["passed"][0]) == passes, t
        if passes:
            assert rec["best_slot"][0] == 2
            assert rec["omega"][0] == pytest.approx(a - D / 2, rel=1e-12)
            assert xp[0] == rec["omega"][0]
            assert rec["score"][0] == 2.0
