"""Workloads for a profiler: each runs one kind of launch of the library inside an NVTX
range of its own name, so that a tool such as Nsight Compute can select it
(--nvtx --nvtx-include "<name>/").

  python -m paper_1704_09012_gb300.profile_workloads round [reps]
      one round of Algorithm 2 at n = 2^20, m = 104857, k = 10485, d = 7, SNR 40 dB
      (the benchmark's instance, expander seed 1000), from the state a decode reaches
      after three rounds, through rl0_round_step, whose column-score and rebuild
      kernels launch directly (outside the decode's conditional graph); `reps`
      repetitions (default 3), each in a range "round";
  python -m paper_1704_09012_gb300.profile_workloads batched [count]
      one rl0_decode_batched call on `count` instances of the batched workload
      (default 256; n uniform in [2^10, 2^16], delta in [0.1, 0.3], rho in [0.05, 0.2],
      d = 7, SNR 30-60 dB), after an untimed call that tunes the schedule, in a range
      "batched".

Every step of the decode runs in the CUDA library; torch only holds device memory and
subtracts A x_hat from y_hat to form the injected residual."""
import sys

import torch

import gm
import paper_1704_09012_gb300 as rl0


def round_workload(reps=3):
    cfg = gm.config_large()
    n, m, k, d, sn = cfg["n"], cfg["m"], cfg["k"], cfg["d"], cfg["sigma_n"]
    A = rl0.Expander.random(n, m, d, seed=1000)
    x, _ = gm.draw_signal(n, k, 1.0, 1000)
    y = rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sn, noise_seed=1001)
    xh, _ = rl0.decode(A, y, k, sigma_n=sn, max_rounds=3)
    rh = y - rl0.sketch(A, xh, sigma_n=0.0)          # r_hat = y_hat - A x_hat
    for _ in range(reps):
        torch.cuda.nvtx.range_push("round")
        rl0.round_step(A, y, k, 3, xh, rh, want_passed=False, sigma_n=sn)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()


def batched_workload(count=256):
    shapes = gm.batch_shapes(count, seed=0)
    As, ys, ks, ps = [], [], [], []
    for i, sh in enumerate(shapes):
        A = rl0.Expander.random(sh["n"], sh["m"], sh["d"], seed=50000 + i)
        x, _ = gm.draw_signal(sh["n"], sh["k"], 1.0, 50000 + i)
        ys.append(rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sh["sigma_n"], noise_seed=90000 + i))
        As.append(A)
        ks.append(sh["k"])
        ps.append(dict(sigma_n=sh["sigma_n"]))
    plan = rl0.BatchPlan(As, ys, ks, ps)
    plan.run()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batched")
    plan.run()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()


def main(argv):
    if not argv or argv[0] not in ("round", "batched"):
        print(__doc__)
        return 2
    torch.cuda.set_device(0)
    if argv[0] == "round":
        round_workload(int(argv[1]) if len(argv) > 1 else 3)
    else:
        batched_workload(int(argv[1]) if len(argv) > 1 else 256)
    print("%s workload done" % argv[0])
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
