"""Failure detection on the GPU without a GPU fault: the column kernel's bounded wait (its
bulk copy of the residual codes into shared memory) is made to give up at once through the
expander's test hook.  The kernel records RL0_ERR_TIMEOUT, waits for its copies in flight
with the built-in limit, scores nothing and returns; the decode reports the error and the
device stays usable, so the next decode on the same expander gives the normal result."""
import numpy as np
import pytest

import gm
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("quantised", [False, True])
def test_bounded_wait_runs_out_and_the_next_decode_succeeds(quantised):
    import paper_1704_09012_gb300 as rl0
    I = gm.instance(seed=3, **gm.config_small())
    y32 = (oracle.sketch(I.rows, I.x.astype(np.float64), I.m) + I.eta.astype(np.float64)).astype(np.float32)
    A = rl0.Expander.from_rows(torch.from_numpy(I.rows).cuda(), I.m)
    y = torch.from_numpy(y32).cuda()
    want, st_want = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
    assert st_want["accepted_rounds"] > 0
    rl0.set_wait_polls(A, 0)
    with pytest.raises(rl0.Rl0Error) as e:
        rl0.decode(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
    assert e.value.code == -4                             # RL0_ERR_TIMEOUT
    torch.cuda.synchronize()                              # the context is still usable
    rl0.set_wait_polls(A, -1)
    got, st = rl0.decode(A, y, I.k, sigma_n=I.sigma_n, quantised=quantised)
    assert torch.equal(got, want)
    assert st["status"] == 0 and st["rounds"] == st_want["rounds"]


def test_wait_hook_rejects_bad_arguments():
    import paper_1704_09012_gb300 as rl0
    A = rl0.Expander.random(2048, 512, 7, seed=1)
    with pytest.raises(rl0.Rl0Error):
        rl0.set_wait_polls(A, 1 << 40)
