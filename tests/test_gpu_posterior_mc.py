"""Monte-Carlo check of the posteriors on the GPU (Section "Comparison with empirical
probabilities", Fig. 3) through rl0_posterior_mc.

- Small instance: the GPU's integer counts (samples and events per bin) equal NumPy's
  exactly, and its sums of the FP32 posterior series equal the oracle's FP64 posteriors
  summed over the same samples (rel. 1e-5).
- The paper's settings, GM(2^20, 0.3 n, rho 0.3 n, 7, N(0,1), N(0, sigma^2)) with
  rho in {0.1, 0.3} and sigma in {1e-3, 1e-2}: the empirical frequency of y_i = 0 (rows)
  and of y_i = y_l (row pairs of a column) per bin against the mean posterior the
  decoder assigns to the bin's samples (p = p_breve p(0), p(0) from the oracle), within
  5 binomial standard deviations + 0.02, as in the oracle's own Monte-Carlo pin."""
import math

import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = 7


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def test_counts_equal_numpy_and_sums_equal_oracle(rl0):
    n, delta, rho, sigma = 1 << 14, 0.3, 0.1, 1e-3
    m = int(delta * n)
    k = int(rho * m)
    I = gm.instance(n, m, k, D, sigma, 5)
    y0_64 = oracle.sketch(I.rows, I.x.astype(np.float64), m)
    y0 = y0_64.astype(np.float32)
    yh = (y0_64 + I.eta.astype(np.float64)).astype(np.float32)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), m)
    nbins, wz, we = 64, 8 * sigma, 8 * math.sqrt(2) * sigma
    hz, he = rl0.posterior_mc(A, torch.from_numpy(y0).cuda(), torch.from_numpy(yh).cuda(), k, sigma,
                              nbins=nbins, wz_max=wz, we_max=we)
    hz, he = hz.cpu().numpy(), he.cpu().numpy()

    def want(w, event, which, wmax):
        a = np.abs(w).astype(np.float32) * np.float32(nbins / wmax)      # the kernel's FP32 binning
        sel = a < nbins
        b = a[sel].astype(np.int64)
        cnt = np.bincount(b, minlength=nbins)
        ev = np.bincount(b, weights=event[sel].astype(np.float64), minlength=nbins)
        p = np.exp(oracle.log_posterior(which, w[sel].astype(np.float64), D, k / m, 1.0, sigma))
        ps = np.bincount(b, weights=p * 2.0 ** 32, minlength=nbins)
        return cnt, ev, ps

    cnt, ev, ps = want(yh, y0 == 0.0, "z", wz)
    np.testing.assert_array_equal(hz[:, 0], cnt)
    np.testing.assert_array_equal(hz[:, 1], ev)
    np.testing.assert_allclose(hz[:, 2].astype(np.float64), ps, rtol=1e-5, atol=2.0 ** 32 * 1e-6)
    s, l = np.triu_indices(D, 1)
    i1, i2 = I.rows[:, s].ravel(), I.rows[:, l].ravel()
    dlt = yh[i1] - yh[i2]                                                  # FP32, as on the GPU
    cnt, ev, ps = want(dlt, y0[i1] == y0[i2], "e", we)
    np.testing.assert_array_equal(he[:, 0], cnt)
    np.testing.assert_array_equal(he[:, 1], ev)
    np.testing.assert_allclose(he[:, 2].astype(np.float64), ps, rtol=1e-5, atol=2.0 ** 32 * 1e-6)
    assert hz[:, 0].sum() > 1000 and he[:, 0].sum() > 10000


@pytest.mark.parametrize("rho,sigma", [(0.1, 1e-3), (0.3, 1e-3), (0.1, 1e-2), (0.3, 1e-2)])
def test_posteriors_against_gpu_monte_carlo_at_the_papers_settings(rl0, rho, sigma):
    n, delta = 1 << 20, 0.3
    m = int(delta * n)
    k = int(rho * m)
    nbins = 48
    hz = he = None
    for inst in range(4):
        A = rl0.Expander.random(n, m, D, seed=300 + inst)
        x, _ = gm.draw_signal(n, k, 1.0, 300 + inst)
        xt = torch.from_numpy(x).cuda()
        y0 = rl0.sketch(A, xt, sigma_n=0.0, noise_seed=0)
        yh = rl0.sketch(A, xt, sigma_n=sigma, noise_seed=400 + inst)
        hz, he = rl0.posterior_mc(A, y0, yh, k, sigma, nbins=nbins, hz=hz, he=he)
        A.free()
    for which, h in (("z", hz.cpu().numpy()), ("e", he.cpu().numpy())):
        _, raw0 = oracle.log_posterior(which, np.zeros(1), D, k / m, 1.0, sigma, raw=True)
        p0 = math.exp(raw0[0])
        checked = 0
        for N, E, P in h:
            if N < 2000:
                continue
            emp = E / N
            pred = p0 * (P / 2.0 ** 32) / N
            sd = math.sqrt(max(pred * (1 - pred), 1e-4) / N)
            assert abs(emp - pred) < 5 * sd + 0.02, (which, N, emp, pred)
            checked += 1
        assert checked >= 8, (which, checked)
