"""GPU learned column scorer: gradients and forward against the FP64 oracle, candidate
features against the oracle's definition, the learned rule reducing to Algorithm 2's rule
for analytic-equivalent weights, learned decodes against the oracle's learned decode, and
what a network trained on the method's own decode logs gains over the analytic rule."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_oracle_mlp import analytic_equivalent_bf16  # noqa: E402


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


def test_mlp_gradient_matches_oracle(rl0):
    rng = np.random.default_rng(0)
    N = 5000
    F = rng.standard_normal((N, 16)).astype(np.float32)
    y = (rng.random(N) < 0.3).astype(np.float32)
    w = rl0.mlp_init(seed=7)
    loss, g = rl0.mlp_grad(w, torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda())
    Lo, go = omlp.loss_and_grad(w.cpu().numpy().astype(np.float64), F.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(Lo, rel=1e-6)
    g = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - go)) <= 1e-4 * np.max(np.abs(go))
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
    # the library's gradient is deterministic
    _, g2 = rl0.mlp_grad(w, torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda())
    assert np.array_equal(g, g2.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("N", [1, 15, 37, 128, 129, 1000])
def test_mlp_gradient_at_block_edges_matches_oracle(rl0, N):
    """The tensor-core gradient with a ragged last 16-row tile and 128-sample block
    (rows past N contribute nothing)."""
    rng = np.random.default_rng(100 + N)
    F = (2.0 * rng.standard_normal((N, 16))).astype(np.float32)
    y = (rng.random(N) < 0.5).astype(np.float32)
    w = rl0.mlp_init(seed=N)
    loss, g = rl0.mlp_grad(w, torch.from_numpy(F).cuda(), torch.from_numpy(y).cuda())
    Lo, go = omlp.loss_and_grad(w.cpu().numpy().astype(np.float64), F.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(Lo, rel=1e-6)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)


def test_mlp_training_is_deterministic(rl0):
    """Two training runs from the same start give bitwise the same parameters and loss:
    every gradient reduction runs in a fixed order."""
    rng = np.random.default_rng(5)
    F = torch.from_numpy(rng.standard_normal((3001, 16)).astype(np.float32)).cuda()
    Y = torch.from_numpy((rng.random(3001) < 0.4).astype(np.float32)).cuda()
    out = []
    for _ in range(2):
        w = rl0.mlp_init(seed=9)
        wb, loss = rl0.mlp_train(w, F, Y, epochs=3, batch=500, lr=3e-3)
        out.append((w.cpu().numpy(), wb.cpu().numpy(), loss))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    w0 = rl0.mlp_init(seed=9)
    assert not np.array_equal(out[0][0], w0.cpu().numpy())          # it did train


def test_mlp_forward_at_tile_edges_matches_oracle(rl0):
    rng = np.random.default_rng(7)
    w = rl0.mlp_init(seed=11)
    wb = rl0.mlp_export(w)
    Wf = oracle.bf16_to_f64(wb.cpu().numpy().view(np.uint16))
    for N in (1, 15, 16, 17, 127, 129):
        F = rng.standard_normal((N, 16)).astype(np.float32)
        lg = rl0.mlp_forward(wb, torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
        ref = oracle.mlp_logits(Wf, F.astype(np.float64))
        assert lg.shape == (N,)
        assert np.max(np.abs(lg - ref)) <= 1e-5 * (1 + np.max(np.abs(ref)))


def test_mlp_forward_matches_oracle_with_bf16_weights(rl0):
    rng = np.random.default_rng(1)
    F = rng.standard_normal((3000, 16)).astype(np.float32)
    w = rl0.mlp_init(seed=3)
    wb = rl0.mlp_export(w)
    lg = rl0.mlp_forward(wb, torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    bits = wb.cpu().numpy().view(np.uint16)
    Wf = oracle.bf16_to_f64(bits)
    ref = oracle.mlp_logits(Wf, F.astype(np.float64))
    assert np.max(np.abs(lg - ref)) <= 1e-5 * (1 + np.max(np.abs(ref)))
    # BF16 rounding of the FP32 parameters is round-to-nearest-even
    w32 = w.cpu().numpy()
    assert np.all(np.abs(Wf - w32) <= np.abs(w32) * 2.0 ** -8)


def test_candidate_features_match_the_oracle_definition(rl0):
    I, y32 = _problem(4096, 1024, 100, 7, 1e-3, 5)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    rng = np.random.default_rng(2)
    x = I.x.astype(np.float64).copy()
    sh = rng.choice(I.support, 40, replace=False)
    x[sh] += rng.uniform(0.2, 1.0, sh.size)
    x[rng.choice(I.support, 30, replace=False)] = 0.0
    x32 = x.astype(np.float32)
    r32 = (y32.astype(np.float64) - _A(I.rows, I.m) @ x32.astype(np.float64)).astype(np.float32)
    ridx = 12
    f, meta, w = rl0.candidate_features(A, torch.from_numpy(y32).cuda(), I.k, ridx, torch.from_numpy(x32).cuda(),
                                        torch.from_numpy(r32).cuda(), sigma_n=I.sigma_n)
    f = f.cpu().numpy().astype(np.float64)
    meta = meta.cpu().numpy()
    assert f.shape[0] > 20
    c = oracle.default_c(False, I.m / I.n, I.k / I.m)
    t = 1 - ridx * c
    rho = I.k / I.m
    r = r32.astype(np.float64)
    checked = 0
    for e in range(f.shape[0]):
        j, s = int(meta[e, 0]), int(meta[e, 1])
        rl = r[I.rows[j]]
        lz = oracle.log_posterior("z", rl, I.d, rho, 1.0, I.sigma_n)
        assert lz[s] <= math.log(1 - t) + 1e-12              # an anchor
        qe = np.exp(oracle.log_posterior("e", rl[s] - rl, I.d, rho, 1.0, I.sigma_n))
        ne, nz = qe.sum(), np.exp(lz).sum()
        wv = (rl * qe).sum() / ne
        lhs, rhs = np.abs(rl - wv).sum(), np.abs(rl).sum()
        assert ne - nz >= 1.5 - 1e-4
        fo = oracle.features(rl, wv, ne, nz, lhs, rhs, I.sigma_n, t, I.d * rho)
        np.testing.assert_allclose(f[e], fo, rtol=2e-4, atol=2e-4)
        checked += 1
    assert checked == f.shape[0]


@pytest.mark.parametrize("seed", [0, 1])
def test_learned_rule_with_analytic_weights_equals_analytic_decode(rl0, seed):
    I, y32 = _problem(3000, 800, 60, 8, 2e-3, seed)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    bits = analytic_equivalent_bf16(I.d)
    wb = torch.from_numpy(bits.view(np.int16)).cuda()
    y = torch.from_numpy(y32).cuda()
    xa, sa = rl0.decode(A, y, I.k, sigma_n=I.sigma_n)
    xl, sl = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, scorer=1, mlp=wb)
    xa, xl = xa.cpu().numpy().astype(np.float64), xl.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.nonzero(xl)[0], np.nonzero(xa)[0])
    assert np.linalg.norm(xl - xa) <= 1e-5 * np.linalg.norm(xa)
    xo, so, _ = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, mlp_bf16=bits)
    assert np.array_equal(np.nonzero(xl)[0], np.nonzero(xo)[0])
    assert np.linalg.norm(xl - xo) <= 1e-5 * np.linalg.norm(xo)


def _success(x, xt, m, sn):
    xl1 = np.abs(xt).sum()
    tol = min((m * sn * math.sqrt(2 / math.pi) + math.sqrt(m * sn * sn * (1 - 2 / math.pi))) / xl1, 0.1)
    return np.abs(x - xt).sum() / xl1 <= tol


def _shape(rng, n, d):
    m = int(0.1 * n)
    rho = float(rng.uniform(0.1, 0.2))
    k = int(rho * m)
    sn = gm.sigma_from_snr(d, k / m, float(rng.uniform(30, 40)))
    return m, k, sn


def test_scorer_log_equals_the_round_loop_composed_from_round_steps(rl0):
    """rl0_scorer_log against the same loop written here from library round steps: the
    accept test ||r||_1 < ||r_hat||_1, the stop level m sigma_n sqrt(2/pi), and the label
    |x_hat_j + w - x_j| <= 4 sigma_n with x_j != 0."""
    rng = np.random.default_rng(21)
    n, d = 1 << 13, 7
    m, k, sn = _shape(rng, n, d)
    I, y32 = _problem(n, m, k, d, sn, 4242)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), m)
    y = torch.from_numpy(y32).cuda()
    xt = torch.from_numpy(I.x.astype(np.float32)).cuda()
    F, Y, rounds = rl0.scorer_log(A, y, k, xt, sigma_n=sn)
    xh = torch.zeros(n, dtype=torch.float32, device="cuda")
    rh = y.clone()
    l1h = float(np.abs(y32.astype(np.float64)).sum())
    feats, labels, ran = [], [], 0
    for r in range(1, 40):
        f, meta, w = rl0.candidate_features(A, y, k, r, xh, rh, sigma_n=sn)
        j = meta[:, 0].long()
        feats.append(f.clone())
        labels.append((((xh[j] + w) - xt[j]).abs() <= np.float32(4.0 * sn)) & (xt[j] != 0))
        xp, rp, _, l1 = rl0.round_step(A, y, k, r, xh, rh, want_passed=False, sigma_n=sn)
        ran += 1
        if l1 < l1h:
            xh, rh, l1h = xp, rp, l1
        if l1h <= m * sn * math.sqrt(2 / math.pi):
            break
    Fr, Yr = torch.cat(feats), torch.cat(labels).float()
    assert rounds == ran and F.shape == Fr.shape and F.shape[0] > 1000
    assert torch.equal(F, Fr) and torch.equal(Y, Yr)
    assert 0.05 < float(Y.mean()) < 0.95
    # a capacity below the count: the binding runs again with room for all and gets the same rows
    F2, Y2, _ = rl0.scorer_log(A, y, k, xt, cap=100, sigma_n=sn)
    assert torch.equal(F2, F) and torch.equal(Y2, Y)


@pytest.fixture(scope="module")
def trained(rl0):
    """A scorer trained on the decode logs of 12 analytic decodes (n = 2^14, d = 7,
    delta = 0.1, rho in [0.1, 0.2], SNR in [30, 40] dB)."""
    from paper_1704_09012_gb300 import learned
    rng = np.random.default_rng(11)
    n, d = 1 << 14, 7
    F, Y = [], []
    for i in range(12):
        m, k, sn = _shape(rng, n, d)
        I, y32 = _problem(n, m, k, d, sn, 500 + i)
        A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), m)
        f, lab = learned.decode_log_samples(A, torch.from_numpy(y32).cuda(), k, torch.from_numpy(I.x).cuda(), sn)
        F.append(f)
        Y.append(lab)
    F, Y = torch.cat(F), torch.cat(Y)
    wb, w, loss = learned.train_scorer(F, Y, epochs=10)
    return dict(wb=wb, bits=wb.cpu().numpy().view(np.uint16), F=F, Y=Y, loss=loss)


def test_training_reduces_the_loss(rl0, trained):
    F, Y = trained["F"], trained["Y"]
    assert F.shape[0] > 2000 and 0.05 < float(Y.mean()) < 0.95
    w0 = rl0.mlp_init(seed=0)
    l0, _ = rl0.mlp_grad(w0, F, Y)
    assert trained["loss"] < 0.7 * l0
    # the exported BF16 network separates the labels on its training logs
    lg = rl0.mlp_forward(trained["wb"], F)
    acc = float(((lg >= 0).float() == Y).float().mean())
    base = max(float(Y.mean()), 1 - float(Y.mean()))
    assert acc > base + 0.02


def test_learned_round_step_matches_oracle(rl0, trained):
    rng = np.random.default_rng(4)
    I, y32 = _problem(1 << 14, 1638, 245, 7, 0.012, 77)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    Acsr = _A(I.rows, I.m)
    near_total = dec_total = passes = 0
    for trial in range(4):
        x = I.x.astype(np.float64).copy()
        sh = rng.choice(I.support, I.k // 4, replace=False)
        x[sh] += rng.choice([-1, 1], sh.size) * rng.uniform(0.2, 1.0, sh.size)
        x[rng.choice(I.support, I.k // (2 + trial), replace=False)] = 0.0
        x32 = x.astype(np.float32)
        r32 = (y32.astype(np.float64) - Acsr @ x32.astype(np.float64)).astype(np.float32)
        for ridx in (2, 10, 25):
            xo, ro, upd, rec = oracle.round_step(I.rows, y32.astype(np.float64), I.k, ridx, x32.astype(np.float64),
                                                 r32.astype(np.float64), sigma_n=I.sigma_n, mlp_bf16=trained["bits"])
            xg, rg, passed, l1g = rl0.round_step(A, torch.from_numpy(y32).cuda(), I.k, ridx,
                                                 torch.from_numpy(x32).cuda(), torch.from_numpy(r32).cuda(),
                                                 sigma_n=I.sigma_n, scorer=1, mlp=trained["wb"])
            pg = passed.cpu().numpy().astype(bool)
            po = rec["passed"].astype(bool)
            near = rec["min_margin"] < 1e-3
            assert np.array_equal(pg[~near], po[~near])
            near_total += int(near.sum())
            dec_total += near.size
            passes += int(po.sum())
            if np.array_equal(pg, po):
                xg = xg.cpu().numpy().astype(np.float64)
                assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
                assert np.linalg.norm(xg - xo) <= 1e-5 * np.linalg.norm(xo)
    assert passes > 100
    assert near_total <= 2 + dec_total // 1000


def _analytic_restart(rl0, A, y, k, sn, x0, rounds=40):
    """A second analytic sweep of Algorithm 2 from x0 (round steps, the accept test on
    ||r||_1, the noise stop level): the control for the learned decode's analytic
    continuation."""
    xh = x0.clone()
    rh = y - rl0.sketch(A, xh, sigma_n=0.0)
    l1h = float(rh.abs().double().sum())
    for r in range(1, rounds):
        xp, rp, _, l1 = rl0.round_step(A, y, k, r, xh, rh, want_passed=False, sigma_n=sn)
        if l1 < l1h:
            xh, rh, l1h = xp, rp, l1
        if l1h <= A.m * sn * math.sqrt(2 / math.pi):
            break
    return xh


def test_trained_scorer_against_the_analytic_rule(rl0, trained):
    """Held-out instances: recovery (success condition of Section 'Stopping conditions'),
    rounds and decode time, learned vs analytic and vs the analytic rule given a second
    sweep from its own result (so that the learned decode's analytic continuation is not
    what makes the difference); and the learned decode against the oracle's learned
    decode."""
    rng = np.random.default_rng(12)
    n, d = 1 << 14, 7
    wb, bits = trained["wb"], trained["bits"]
    res, par = [], []
    for i in range(8):
        m, k, sn = _shape(rng, n, d)
        I, y32 = _problem(n, m, k, d, sn, 900 + i)
        A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), m)
        y = torch.from_numpy(y32).cuda()
        xa, sa = rl0.decode(A, y, k, sigma_n=sn)
        xl, sl = rl0.decode(A, y, k, sigma_n=sn, scorer=1, mlp=wb)
        xr = _analytic_restart(rl0, A, y, k, sn, xa)
        res.append((_success(xa.cpu().numpy(), I.x, m, sn), _success(xl.cpu().numpy(), I.x, m, sn),
                    sa["rounds"], sl["rounds"], sa["ms"], sl["ms"], sl["analytic_rounds"],
                    _success(xr.cpu().numpy(), I.x, m, sn)))
        if i < 3:
            xo, so, lo = oracle.decode(I.rows, y32.astype(np.float64), k, sigma_n=sn, mlp_bf16=bits)
            xg = xl.cpu().numpy().astype(np.float64)
            par.append((np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0]),
                        np.linalg.norm(xg - xo) / np.linalg.norm(xo), sl["rounds"], so["rounds"],
                        sl["analytic_rounds"], so["analytic_rounds"],
                        [e["updated"] for e in rl0.decode_log(A)], [e["updated"] for e in lo]))
    res = np.array(res, dtype=float)
    print("\nanalytic: success %.2f (with a second sweep %.2f) rounds %.1f ms %.3f | learned: success %.2f "
          "rounds %.1f ms %.3f (analytic continuation rounds %.1f)"
          % (res[:, 0].mean(), res[:, 7].mean(), res[:, 2].mean(), res[:, 4].mean(), res[:, 1].mean(),
             res[:, 3].mean(), res[:, 5].mean(), res[:, 6].mean()))
    for p_ in par:
        print("parity: support %s rel %.2e rounds %d/%d cont %d/%d\n  gpu %s\n  orc %s" % p_)
    # the trained network recovers strictly more held-out instances than the analytic
    # rule, with or without the analytic rule's second sweep, and loses none
    assert res[:, 1].mean() > max(res[:, 0].mean(), res[:, 7].mean())
    assert np.all(res[:, 1] >= res[:, 0])
    for p_ in par:
        assert p_[0] and p_[1] <= 1e-5


def test_learned_continuation_bounds_with_its_own_posteriors(rl0):
    """The analytic continuation of a learned decode bounds n_z with the p_z table of its own
    parameters, whatever an earlier decode on the same expander left behind.  Here an
    analytic decode at 20x the noise level runs first (a broader p_z, so larger n_z bounds);
    the learned decode that follows accepts nothing, so its continuation is Alg. 2 from
    x_hat = 0 and must equal the oracle's learned decode with the same network."""
    I, y32 = _problem(4096, 1024, 100, 7, 1e-3, 3)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y = torch.from_numpy(y32).cuda()
    rl0.decode(A, y, I.k, sigma_n=20 * I.sigma_n)
    bits = np.zeros(rl0.MLP_PARAMS, np.uint16)
    bits[-1] = 0xBF80                                     # logit -1 for every input: accept nothing
    wb = torch.from_numpy(bits.view(np.int16)).cuda()
    xl, sl = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, scorer=1, mlp=wb)
    assert sl["analytic_rounds"] > 0 and sl["accepted_rounds"] > 0
    xo, so, _ = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, mlp_bf16=bits)
    assert so["analytic_rounds"] > 0
    xg = xl.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert np.linalg.norm(xg - xo) <= 1e-5 * np.linalg.norm(xo)
    assert sl["accepted_rounds"] == so["accepted_rounds"]


def test_learned_decode_at_scale_matches_oracle(rl0, trained):
    """The learned decode at the learned workload's evaluation shape (delta = 0.1,
    rho = 0.15, SNR 30 dB, d = 7) at n = 2^20 -- the oracle's learned decode at n = 2^22
    takes too long for a test -- against the oracle's learned decode with the same BF16
    network, analytic continuation included."""
    n, d = 1 << 20, 7
    m = int(0.1 * n)
    k = int(0.15 * m)
    sn = gm.sigma_from_snr(d, k / m, 30.0)
    I, y32 = _problem(n, m, k, d, sn, 4242)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), m)
    xl, sl = rl0.decode(A, torch.from_numpy(y32).cuda(), k, sigma_n=sn, scorer=1, mlp=trained["wb"])
    with oracle.openmp():
        xo, so, _ = oracle.decode(I.rows, y32.astype(np.float64), k, sigma_n=sn, mlp_bf16=trained["bits"])
    xg = xl.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print("\nlearned n=2^20: rounds %d/%d (continuation %d/%d) accepted %d/%d rel_l2 %.2e" % (
        sl["rounds"], so["rounds"], sl["analytic_rounds"], so["analytic_rounds"], sl["accepted_rounds"],
        so["accepted_rounds"], rel))
    assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
    assert rel <= 1e-5
    assert sl["rounds"] == so["rounds"] and sl["analytic_rounds"] == so["analytic_rounds"]
    assert sl["accepted_rounds"] == so["accepted_rounds"]
