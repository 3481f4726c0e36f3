"""Recovery phase transitions of Robust-l0 on the GPU: the extreme-subsampling experiment of
Section "Phase transitions for extreme subsampling" (arXiv 1704.09012).

For a (delta, sigma, n) cell, rho starts at rho_step and grows by rho_step while at least
one of `problems` instances of the generating model GM(n, delta n, rho delta n, d, N(0,1),
N(0, sigma^2)) (Def. "Generating model") is recovered; an instance counts as recovered
under Eq. (success_condition_clip) with C_1 = 1.  rho* is the largest rho at which at
least half of the instances are recovered; a logistic fit of the recovery data gives the
50% point and the transition's width (fit_logistic).  Timings are the decode's own
(rl0_stats.ms).

    python -m paper_1704_09012_gb300.phase --delta 0.001 --sigma 0.001 --log2n 22

prints one JSON line per rho and a summary line.  Every decode runs in the CUDA library;
expanders, sketches and noise are drawn on the GPU by the library's generator (Philox,
Def. GM), the signal's support and values by `gm` (numpy)."""
import argparse
import json
import math
import sys

import numpy as np


def success(x_hat, x, m, sigma):
    """Eq. (success_condition_clip), C_1 = 1: ||x_hat - x||_1 / ||x||_1 is at most
    min((m sigma sqrt(2/pi) + sqrt(m sigma^2 (1 - 2/pi))) / ||x||_1, 0.1)."""
    xl1 = float(np.abs(x).sum())
    tol = min((m * sigma * math.sqrt(2 / math.pi) + math.sqrt(m * sigma * sigma * (1 - 2 / math.pi))) / xl1, 0.1)
    return float(np.abs(x_hat - x).sum()) / xl1 <= tol


def fit_logistic(rhos, recovered, problems):
    """The recovery data fitted with a logistic function (Section "Phase transitions and
    runtime", after Blanchard et al.): P(recovered | rho) = 1 / (1 + exp((rho - rho50) / w)),
    fitted by binomial maximum likelihood, w >= 1e-4.  Returns (rho50, w, width) with
    width = 2 ln(9) w, the distance in rho from 90% to 10% recovery (reading: the paper's
    transition width, whose exact definition the text does not print)."""
    from scipy.optimize import minimize
    r = np.asarray(rhos, np.float64)
    kk = np.asarray(recovered, np.float64)
    nn = np.broadcast_to(np.asarray(problems, np.float64), r.shape)

    def nll(th):
        z = (r - th[0]) / math.exp(th[1])
        # log P = -log(1 + e^z), log(1 - P) = z - log(1 + e^z)
        lse = np.logaddexp(0.0, z)
        return float(np.sum(kk * lse + (nn - kk) * (lse - z)))

    frac = kk / nn
    above = r[frac >= 0.5]
    r0 = float(above.max()) if above.size else float(r.min())
    best = None
    for w0 in (0.003, 0.01, 0.03):
        res = minimize(nll, np.array([r0, math.log(w0)]), method="L-BFGS-B",
                       bounds=[(float(r.min()) - 0.5, float(r.max()) + 0.5), (math.log(1e-4), math.log(1.0))])
        if best is None or res.fun < best.fun:
            best = res
    rho50, w = float(best.x[0]), math.exp(float(best.x[1]))
    return rho50, w, 2.0 * math.log(9.0) * w


def cell(delta, sigma, n, d=7, problems=10, rho_step=0.01, rho_max=0.5, adaptive=False, quantised=False,
         seed=0, out=None, alpha=0.0, anchor_rule=0, rho_start=None):
    """Sweep rho for one (delta, sigma, n) cell.  Returns the per-rho rows and rho*."""
    import torch
    import gm
    import paper_1704_09012_gb300 as rl0
    m = int(delta * n)
    rows = []
    rho_star = 0.0
    steps = int(round(rho_max / rho_step))
    first = 1 if rho_start is None else max(1, int(round(rho_start / rho_step)))
    A = None
    for step in range(first, steps + 1):
        rho = round(step * rho_step, 10)
        k = max(1, int(rho * m))
        ok, times, rounds = 0, [], []
        for p in range(problems):
            s = seed + 1000 * step + p
            if A is not None:
                A.free()
            A = rl0.Expander.random(n, m, d, seed=s)
            x, _ = gm.draw_signal(n, k, 1.0, s)
            y = rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sigma, noise_seed=s + 7)
            xh, st = rl0.decode(A, y, k, sigma_n=sigma, adaptive_k=adaptive, quantised=quantised, alpha=alpha,
                                anchor_rule=anchor_rule)
            if success(xh.cpu().numpy().astype(np.float64), x.astype(np.float64), m, sigma):
                ok += 1
                times.append(st["ms"])
                rounds.append(st["rounds"])
        row = {"delta": delta, "sigma": sigma, "n": n, "m": m, "d": d, "rho": rho, "k": k,
               "recovered": ok, "problems": problems,
               "ms_recovered_mean": float(np.mean(times)) if times else None,
               "rounds_recovered_mean": float(np.mean(rounds)) if rounds else None,
               "adaptive_k": int(adaptive), "quantised": int(quantised), "alpha": alpha, "anchor_rule": anchor_rule}
        rows.append(row)
        if out is not None:
            print(json.dumps(row), file=out, flush=True)
        if 2 * ok >= problems:
            rho_star = rho
        if ok == 0:
            break
    if A is not None:
        A.free()
    return rows, rho_star


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--delta", type=float, required=True)
    ap.add_argument("--sigma", type=float, required=True)
    ap.add_argument("--log2n", type=int, default=22)
    ap.add_argument("--d", type=int, default=7)
    ap.add_argument("--problems", type=int, default=10)
    ap.add_argument("--rho-step", type=float, default=0.01)
    ap.add_argument("--rho-max", type=float, default=0.5)
    ap.add_argument("--adaptive", action="store_true")
    ap.add_argument("--quantised", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--alpha", type=float, default=0.0, help="consensus threshold (0: the default reading)")
    ap.add_argument("--anchor-rule", type=int, default=0, help="0: last passing anchor; 1: largest n_e - n_z")
    ap.add_argument("--rho-start", type=float, default=None)
    a = ap.parse_args(argv)
    rows, rho_star = cell(a.delta, a.sigma, 1 << a.log2n, a.d, a.problems, a.rho_step, a.rho_max, a.adaptive,
                          a.quantised, a.seed, out=sys.stdout, alpha=a.alpha, anchor_rule=a.anchor_rule,
                          rho_start=a.rho_start)
    rho50, w, width = fit_logistic([r["rho"] for r in rows], [r["recovered"] for r in rows], a.problems)
    print(json.dumps({"summary": True, "delta": a.delta, "sigma": a.sigma, "n": 1 << a.log2n,
                      "adaptive_k": int(a.adaptive), "quantised": int(a.quantised), "alpha": a.alpha,
                      "anchor_rule": a.anchor_rule, "rho_star": rho_star,
                      "rho50_logistic": rho50, "width_90_10": width}), flush=True)


if __name__ == "__main__":
    main()
