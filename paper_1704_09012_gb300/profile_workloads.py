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
      "batched";
  python -m paper_1704_09012_gb300.profile_workloads learned [log2n] [reps]
      one learned-scorer round at n = 2^log2n (default 20; 22 is the learned workload's
      evaluation size), m = n/10, rho = 0.15, d = 7, SNR 30 dB, from the state the
      analytic decode reaches after three rounds, through rl0_round_step with a scorer
      trained first on the decode logs of two analytic decodes at n = 2^16 (rl0_scorer_log,
      rl0_mlp_train); `reps` repetitions (default 2), each in a range "learned".  At
      n = 2^20 the round runs on the resident-code kernel, at n = 2^22 (whose codes do not
      fit in shared memory) on the L2-gather kernel.

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


def learned_workload(log2n=20, reps=2):
    from . import learned
    d = 7
    F, Y = [], []
    for i in range(2):
        n = 1 << 16
        m = n // 10
        k = int(0.15 * m)
        sn = gm.sigma_from_snr(d, k / m, 30.0)
        A = rl0.Expander.random(n, m, d, seed=60000 + i)
        x, _ = gm.draw_signal(n, k, 1.0, 60000 + i)
        xt = torch.from_numpy(x).cuda()
        y = rl0.sketch(A, xt, sigma_n=sn, noise_seed=61000 + i)
        f, lab = learned.decode_log_samples(A, y, k, xt, sn)
        F.append(f)
        Y.append(lab)
        A.free()
    wb, _, _ = learned.train_scorer(torch.cat(F), torch.cat(Y), epochs=4)
    n = 1 << log2n
    m = n // 10
    k = int(0.15 * m)
    sn = gm.sigma_from_snr(d, k / m, 30.0)
    A = rl0.Expander.random(n, m, d, seed=62000)
    x, _ = gm.draw_signal(n, k, 1.0, 62000)
    y = rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sn, noise_seed=63000)
    xh, _ = rl0.decode(A, y, k, sigma_n=sn, max_rounds=3)
    rh = y - rl0.sketch(A, xh, sigma_n=0.0)
    for _ in range(reps):
        torch.cuda.nvtx.range_push("learned")
        rl0.round_step(A, y, k, 3, xh, rh, want_passed=False, sigma_n=sn, scorer=1, mlp=wb)
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
    if not argv or argv[0] not in ("round", "batched", "learned"):
        print(__doc__)
        return 2
    torch.cuda.set_device(0)
    if argv[0] == "round":
        round_workload(int(argv[1]) if len(argv) > 1 else 3)
    elif argv[0] == "learned":
        learned_workload(int(argv[1]) if len(argv) > 1 else 20, int(argv[2]) if len(argv) > 2 else 2)
    else:
        batched_workload(int(argv[1]) if len(argv) > 1 else 256)
    print("%s workload done" % argv[0])
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
