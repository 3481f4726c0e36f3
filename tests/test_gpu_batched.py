"""Batched decoding: many independent instances of uneven n, m, k, d in one persistent
launch.  Each instance must come out bitwise equal to rl0_decode on it alone (same
arithmetic, same order), and a sample is checked against the FP64 oracle."""
import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl0():
    import paper_1704_09012_gb300 as m
    m._lib()
    return m


def _instances(count, seed, d_choices=(7,), nmax=20000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(1024, nmax + 1))
        delta = float(rng.uniform(0.1, 0.3))
        rho = float(rng.uniform(0.05, 0.2))
        snr = float(rng.uniform(30, 60))
        d = int(rng.choice(d_choices))
        m = max(int(delta * n), d + 1)
        k = max(int(rho * m), 1)
        sn = gm.sigma_from_snr(d, k / m, snr)
        I = gm.instance(n, m, k, d, sn, seed * 1000 + i)
        y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
        out.append((I, y.astype(np.float32)))
    return out


def _run(rl0, insts, quantised):
    As = [rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m) for I, _ in insts]
    ys = [torch.from_numpy(y).cuda() for _, y in insts]
    ks = [I.k for I, _ in insts]
    qs = quantised if isinstance(quantised, list) else [quantised] * len(insts)
    params = [dict(sigma_n=I.sigma_n, quantised=q) for (I, _), q in zip(insts, qs)]
    xs, stats = rl0.decode_batched(As, ys, ks, params)
    return As, ys, params, xs, stats


@pytest.mark.parametrize("quantised", [False, True])
def test_batched_equals_single_decode_bitwise(rl0, quantised):
    insts = _instances(24, 1)
    As, ys, params, xs, stats = _run(rl0, insts, quantised)
    for A, y, p, xb, sb, (I, _) in zip(As, ys, params, xs, stats, insts):
        xs1, s1 = rl0.decode(A, y, I.k, **p)
        assert torch.equal(xb, xs1), (I.n, I.m, I.k)
        for f in ("rounds", "accepted_rounds", "converged", "support_size"):
            assert sb[f] == s1[f], f
        assert sb["final_l1"] == s1["final_l1"]


def test_batched_mixed_d_and_score_kinds_and_oracle_sample(rl0):
    insts = _instances(16, 2, d_choices=(5, 7, 15), nmax=12000)
    qs = [bool(i % 2) for i in range(len(insts))]
    As, ys, params, xs, stats = _run(rl0, insts, qs)
    for i, (A, y, p, xb, (I, y32)) in enumerate(zip(As, ys, params, xs, insts)):
        xs1, _ = rl0.decode(A, y, I.k, **p)
        assert torch.equal(xb, xs1)
        if i < 6:
            xo, _, _ = oracle.decode(I.rows, y32.astype(np.float64), I.k, sigma_n=I.sigma_n, quantised=qs[i])
            xg = xb.cpu().numpy().astype(np.float64)
            assert np.array_equal(np.nonzero(xg)[0], np.nonzero(xo)[0])
            assert np.linalg.norm(xg - xo) <= 1e-5 * max(np.linalg.norm(xo), 1e-30)


def test_batched_repeat_is_deterministic(rl0):
    insts = _instances(12, 3)
    As, ys, params, xs, _ = _run(rl0, insts, False)
    xs2, _ = rl0.decode_batched(As, ys, [I.k for I, _ in insts], params)
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)


def test_batched_rejects_bad_requests(rl0):
    insts = _instances(3, 4)
    As, ys, params, xs, _ = _run(rl0, insts, False)
    with pytest.raises(rl0.Rl0Error):                      # the same expander twice
        rl0.decode_batched([As[0], As[0]], [ys[0], ys[0]], [insts[0][0].k] * 2, params[:1] * 2)
    big = rl0.Expander.random(30000, 23000, 7, seed=1)
    with pytest.raises(rl0.Rl0Error) as e:                  # r_hat would not fit in shared memory
        rl0.decode_batched([big], [torch.zeros(23000, device="cuda")], [100], [dict(sigma_n=1e-3)])
    assert e.value.code == -5
