"""rl0_decode_static -- the decode for callers that cannot allocate (inside a stream
capture, under a memory budget fixed at start-up, or next to an allocator that owns
the free device memory).  It must give what rl0_decode gives, call after call, even
though every call reuses the same fixed workspace inside the library.

Kept in a file that pytest collects last, so a failure here comes after every other
test has run."""
import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, m, k, d, sigma_n, seed):
    I = gm.instance(n, m, k, d, sigma_n, seed)
    y = oracle.sketch(I.rows, I.x.astype(np.float64), m) + I.eta.astype(np.float64)
    return I, torch.from_numpy(y.astype(np.float32)).cuda()


@pytest.mark.parametrize("quantised", [False, True])
def test_static_decode_matches_decode_on_two_calls_in_a_row(quantised):
    import paper_1704_09012_gb300 as rl0
    for seed, cfg in ((0, dict(n=4096, m=1024, k=100, d=7, sigma_n=1e-3)),
                      (1, dict(n=6001, m=1500, k=120, d=15, sigma_n=5e-3))):
        I, y = _problem(seed=seed, **cfg)
        A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
        want, st_want = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
        want = want.cpu().numpy().astype(np.float64)
        for call in range(2):
            got, st = rl0.decode_static(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
            got = got.cpu().numpy().astype(np.float64)
            assert np.array_equal(np.nonzero(got)[0], np.nonzero(want)[0]), call
            assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want), call
            assert st["rounds"] == st_want["rounds"] and st["support_size"] == st_want["support_size"]
            assert st["final_l1"] == pytest.approx(st_want["final_l1"], rel=1e-12)


def test_static_decode_rejects_instances_beyond_its_workspace():
    import paper_1704_09012_gb300 as rl0
    A = rl0.Expander.random(65537, 1000, 7, seed=3)
    y = torch.zeros(1000, device="cuda")
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_static(A, y, 10, sigma_n=1e-3)
    assert e.value.code == -8
    A = rl0.Expander.random(70000 // 2, 32769, 7, seed=3)
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode_static(A, torch.zeros(32769, device="cuda"), 10, sigma_n=1e-3)
    assert e.value.code == -8
