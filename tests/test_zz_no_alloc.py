"""rl0_decode_static -- the decode for callers that cannot allocate (a memory budget
fixed at start-up, or a host whose own allocator owns the free device memory).  It must
give what rl0_decode gives, call after call, even though every call reuses the same
fixed workspace inside the library, and it must not allocate device memory.

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


def _reject_all_mlp():
    """BF16 parameters of a network whose logit is -1 for every input: the learned rounds
    accept nothing, so every learned decode goes on to the analytic continuation."""
    import paper_1704_09012_gb300 as rl0
    bits = np.zeros(rl0.MLP_PARAMS, np.uint16)
    bits[-1] = 0xBF80                                     # b3 = -1.0
    return torch.from_numpy(bits.view(np.int16)).cuda()


def _same(got, want, st, st_want):
    got = got.cpu().numpy().astype(np.float64)
    want = want.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.nonzero(got)[0], np.nonzero(want)[0])
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)
    assert st["rounds"] == st_want["rounds"] and st["support_size"] == st_want["support_size"]
    assert st["accepted_rounds"] == st_want["accepted_rounds"]
    assert st["final_l1"] == pytest.approx(st_want["final_l1"], rel=1e-12)


@pytest.mark.parametrize("quantised", [False, True])
def test_static_decode_matches_decode_on_two_calls_in_a_row(quantised):
    import paper_1704_09012_gb300 as rl0
    for seed, cfg in ((0, dict(n=4096, m=1024, k=100, d=7, sigma_n=1e-3)),
                      (1, dict(n=6001, m=1500, k=120, d=15, sigma_n=5e-3))):
        I, y = _problem(seed=seed, **cfg)
        A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
        want, st_want = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
        for call in range(2):
            got, st = rl0.decode_static(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
            _same(got, want, st, st_want)


def test_static_decode_at_the_workspace_limits_allocates_nothing():
    """n = 65536 and m = 32768, the largest instance the fixed array holds: every part of
    its layout is used to the end.  A warm call leaves the device's free memory unchanged."""
    import paper_1704_09012_gb300 as rl0
    I, y = _problem(65536, 32768, 3000, 7, 2e-3, 5)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    want, st_want = rl0.decode(A, y, I.k, sigma_n=I.sigma_n)
    assert st_want["accepted_rounds"] > 0
    out = torch.empty(I.n, dtype=torch.float32, device="cuda")
    rl0.decode_static(A, y, I.k, out=out, sigma_n=I.sigma_n)        # warm (first call on this device)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        got, st = rl0.decode_static(A, y, I.k, out=out, sigma_n=I.sigma_n)
        _same(got, want, st, st_want)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_learned_decode_runs_the_analytic_continuation_like_decode():
    import paper_1704_09012_gb300 as rl0
    I, y = _problem(4096, 1024, 100, 7, 1e-3, 2)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    wb = _reject_all_mlp()
    want, st_want = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, scorer=1, mlp=wb)
    assert st_want["analytic_rounds"] > 0 and st_want["accepted_rounds"] > 0
    for call in range(2):
        got, st = rl0.decode_static(A, y, I.k, sigma_n=I.sigma_n, scorer=1, mlp=wb)
        _same(got, want, st, st_want)
        assert st["analytic_rounds"] == st_want["analytic_rounds"]
    # the static decode keeps no round log
    assert rl0.decode_log(A) == []


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
