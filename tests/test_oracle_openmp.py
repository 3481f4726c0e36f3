"""The oracle's OpenMP build (the columns of a round scored by several host threads) gives
bitwise the serial build's results: every column of a round reads only r_hat and writes
only its own x'_j, so the order in which columns are scored cannot matter."""
import numpy as np

import gm
import oracle


def _y(I):
    return (oracle.sketch(I.rows, I.x.astype(np.float64), I.m) + I.eta.astype(np.float64)).astype(np.float32)


def test_openmp_decode_equals_serial():
    for quantised in (False, True):
        I = gm.instance(seed=1, **gm.config_small())
        y = _y(I).astype(np.float64)
        xs, ss, ls = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
        with oracle.openmp():
            xp, sp_, lp = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
        assert np.array_equal(xs, xp)
        assert ss == sp_ and ls == lp


def test_openmp_round_records_equal_serial():
    I = gm.instance(20000, 3000, 250, 7, 2e-3, 4)
    y = _y(I).astype(np.float64)
    rng = np.random.default_rng(0)
    x = I.x.astype(np.float64).copy()
    x[rng.choice(I.support, 60, replace=False)] += 0.4
    r = y - oracle.sketch(I.rows, x, I.m)
    a = oracle.round_step(I.rows, y, I.k, 12, x, r, sigma_n=I.sigma_n)
    with oracle.openmp():
        b = oracle.round_step(I.rows, y, I.k, 12, x, r, sigma_n=I.sigma_n)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert a[3].tobytes() == b[3].tobytes()
