#!/usr/bin/env python3
"""Benchmark of the Robust-l0 decoder (arXiv 1704.09012, Algorithm 2) on one GB300.

A step is one whole decode (every round of the sweep t = 1, 1-c, ... > 0, or until the
stopping level) of one synthetic instance drawn from the generating model
GM(n, m, k, d, N(0,1), N(0, sigma_n^2)) at n = 2^20, delta = m/n = 0.1, rho = k/m = 0.1,
d = 7, SNR 40 dB, continuous scores.  Instances are drawn once and stay in HBM; L2 is
flushed (a 256 MiB write) between timed steps.

Printed value: nnz(A) * rounds / s over all ranks (each rank decodes its own instance:
weak scaling).  ms_per_step is the time to recover one instance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this project has) on a
bounded sample of the same workload: each step is one full-size round.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to recover & nnz(A)*rounds/s at n=2^20,d=7; batched/learned vs plain"
UNIT = "nnz*rounds/s"
L2_FLUSH_BYTES = 256 << 20
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def workload():
    import gm
    cfg = gm.config_large()
    cfg["snr_db"] = 40.0
    return cfg


def config_dict(cfg, variant, extra=None):
    d = {
        "workload": "Robust-l0 %s decode, n=2^20, m=%d, k=%d, d=%d, SNR 40 dB (sigma_n=%.4g), "
                    "Gaussian signal, 1 instance per step per GPU" % (variant, cfg["m"], cfg["k"], cfg["d"],
                                                                   cfg["sigma_n"]),
        "n": cfg["n"], "m": cfg["m"], "k": cfg["k"], "d": cfg["d"], "sigma_n": cfg["sigma_n"],
        "scores": variant,
        "l2": "flushed between timed steps (256 MiB write)",
    }
    if extra:
        d.update(extra)
    return d


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank):
    """Each rank decodes its own instance (weak scaling: the work per GPU is fixed)."""
    return 1000 + rank


def max_over_ranks(v, ws, device):
    """The largest per-rank value over the job (the slowest rank's time); no exchange
    at one rank.  `device` is where the process group's backend keeps tensors."""
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ws, t_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return ws * units_per_rank / t_max


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # the raw samples (RL0_CLOCKS_CSV, else a temporary file); the JSON line carries their summary
        self.path = os.environ.get("RL0_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(), "rl0_clocks_bench.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        under_load = [v for v in sm if smax and v > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(under_load) if under_load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# The sources that define the column kernel (its translation unit and the
# headers it includes): the recorded DRAM traffic is reported only while these
# are unchanged since the capture.
COLUMN_KERNEL_SOURCES = ["rl0_column_res.cu", "rl0_round.cuh", "rl0_device.cuh", "rl0_common.cuh"]


def _code_only(src):
    """C/C++ source without its comments, trailing blanks and empty lines (string and
    character literals kept), so that counters stay tied to the code they measured."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in COLUMN_KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, "paper_1704_09012_gb300", "csrc", f)).read()).encode())
    h.update(_code_only(open(os.path.join(ROOT, "include", "rl0.h")).read()).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the sources still match."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC)).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def _peak_hbm():
    """(GB/s, source) of the HBM copy peak: MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        v = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"


def l2_copy_peak(torch, sizes_mib=(8, 16, 32), back_to_back=20, reps=10):
    """L2-resident copy bandwidth (GB/s, read + write bytes): `back_to_back` copies
    b.copy_(a) between one pair of CUDA events (so a short kernel's launch and ramp do
    not dominate), a and b of each size in `sizes_mib` MiB (at most 2 x 32 MiB, inside the
    129 MB L2), best over sizes and `reps` repetitions -- the L2 counterpart of the HBM
    copy figure.  Returns (GB/s, buffer MiB of the best)."""
    best = (0.0, None)
    stream = torch.cuda.current_stream()
    for mib in sizes_mib:
        n = (mib << 20) // 4
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        for _ in range(5):
            b.copy_(a)
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(back_to_back):
                b.copy_(a)
            e1.record(stream)
            torch.cuda.synchronize()
            gbs = back_to_back * 2.0 * n * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9
            if gbs > best[0]:
                best = (gbs, mib)
        del a, b
    return best


def l2_read_peak(torch, sizes_mib=(16, 32, 64), back_to_back=20, reps=10):
    """L2-resident read bandwidth (GB/s): `back_to_back` reductions a.sum() of one buffer
    of each size in `sizes_mib` MiB (inside the 129 MB L2) between one pair of CUDA
    events, best over sizes and `reps` repetitions.  The reduction writes one scalar, so
    the bytes are reads.  Returns (GB/s, buffer MiB of the best)."""
    best = (0.0, None)
    stream = torch.cuda.current_stream()
    for mib in sizes_mib:
        n = (mib << 20) // 4
        a = torch.ones(n, dtype=torch.float32, device="cuda")
        out = torch.empty((), dtype=torch.float32, device="cuda")
        for _ in range(5):
            torch.sum(a, dim=0, out=out)
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(back_to_back):
                torch.sum(a, dim=0, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            gbs = back_to_back * n * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9
            if gbs > best[0]:
                best = (gbs, mib)
        del a
    return best


def bench_batched(rl0, torch, count, steps, flush, plain=True):
    """The batched workload: `count` independent instances, n uniform over [2^10, 2^16],
    delta in [0.1, 0.3], rho in [0.05, 0.2], d = 7, SNR in [30, 60] dB, continuous scores,
    decoded in one persistent launch; the same instances decoded one by one with
    rl0_decode are timed beside it (equal work, bitwise-equal results)."""
    import numpy as np
    import gm
    shapes = gm.batch_shapes(count, seed=0)
    As, ys, ks, ps = [], [], [], []
    for i, sh in enumerate(shapes):
        A = rl0.Expander.random(sh["n"], sh["m"], sh["d"], seed=50000 + i)
        x, _ = gm.draw_signal(sh["n"], sh["k"], 1.0, 50000 + i)
        ys.append(rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sh["sigma_n"], noise_seed=90000 + i))
        As.append(A)
        ks.append(sh["k"])
        ps.append(dict(sigma_n=sh["sigma_n"]))
    outs = [torch.empty(A.n, dtype=torch.float32, device="cuda") for A in As]
    stream = torch.cuda.current_stream()
    plan = rl0.BatchPlan(As, ys, ks, ps, outs=outs)               # the call's arrays, marshalled once
    plan.run()                                                    # warm-up (and schedule tuning)
    times, stats = [], None
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, stats = plan.run(stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        stats = [s_.as_dict() for s_ in plan.S]
    nnz_rounds = sum(A.n * A.d * st["rounds"] for A, st in zip(As, stats))
    ms = sum(times) / len(times)
    kernel_ms = stats[0]["ms"]                    # the library's events around the persistent launch(es)
    alg_bytes = 4 * nnz_rounds                   # every round streams each instance's row ids once
    peak = _peak_hbm()
    res = {"workload": "%d instances, n~U[2^10,2^16], delta~U[0.1,0.3], rho~U[0.05,0.2], d=7, SNR~U[30,60] dB, "
                       "continuous scores, one persistent launch" % count,
           "ms_per_batch": ms, "value": nnz_rounds / (ms * 1e-3), "unit": UNIT,
           "kernel_ms": kernel_ms, "host_ms": ms - kernel_ms,
           "total_nnz": int(sum(A.n * A.d for A in As)), "rounds_mean": float(np.mean([s["rounds"] for s in stats])),
           "converged_frac": float(np.mean([s["converged"] for s in stats])),
           "roofline": {"bound": "hbm", "kernel": "k_decode_batched", "achieved": alg_bytes / (kernel_ms * 1e-3) / 1e9,
                        "peak": peak[0], "peak_source": peak[1], "unit": "GB/s",
                        "frac": alg_bytes / (kernel_ms * 1e-3) / 1e9 / peak[0], "alg_bytes_per_launch": alg_bytes,
                        "alg_bytes": "4 B of row ids per nonzero per round (nnz(A_i) x rounds_i summed)"}}
    if plain:
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for A, y, k, p, o in zip(As, ys, ks, ps, outs):
            rl0.decode(A, y, k, out=o, **p)
        e1.record(stream)
        torch.cuda.synchronize()
        pm = e0.elapsed_time(e1)
        res["plain_loop_ms"] = pm
        res["plain_loop_value"] = nnz_rounds / (pm * 1e-3)
        res["speedup_vs_plain_loop"] = pm / ms
    for A in As:
        A.free()
    return res


def _analytic_restart(rl0, A, y, k, sn, x0, rounds=40):
    """A second analytic sweep from x0 (round steps, accept on ||r||_1, noise stop level):
    the control for the learned decode's analytic continuation."""
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


def bench_learned(rl0, torch, flush, train_instances=4, eval_instances=10):
    """The learned column scorer: trained on the decode logs of analytic decodes at
    n=2^20, d=7, delta=0.1, rho~U[0.1,0.2], SNR~U[30,40] dB, then evaluated against the
    analytic rule (time to recover, rounds, success condition of Section 'Stopping
    conditions', relative errors) on `eval_instances` seeds at n=2^22, delta=0.1,
    rho=0.15, SNR 30 dB, with a control (the analytic rule's result given a second
    analytic sweep), and on as many seeds at n=2^20, rho=0.1, SNR 40 dB, where the
    analytic rule recovers (the learned threshold 0.9 there)."""
    import numpy as np
    import gm
    from paper_1704_09012_gb300 import learned
    rng = np.random.default_rng(2024)
    d = 7
    F, Y = [], []
    t0 = time.perf_counter()
    for i in range(train_instances):
        n = 1 << 20
        m = int(0.1 * n)
        k = int(float(rng.uniform(0.1, 0.2)) * m)
        sn = gm.sigma_from_snr(d, k / m, float(rng.uniform(30, 40)))
        A = rl0.Expander.random(n, m, d, seed=70000 + i)
        x, _ = gm.draw_signal(n, k, 1.0, 70000 + i)
        xt = torch.from_numpy(x).cuda()
        y = rl0.sketch(A, xt, sigma_n=sn, noise_seed=71000 + i)
        f, lab = learned.decode_log_samples(A, y, k, xt, sn)
        F.append(f)
        Y.append(lab)
        A.free()
    F, Y = torch.cat(F), torch.cat(Y)
    wb, _, loss = learned.train_scorer(F, Y, epochs=8)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {"workload": "train: %d analytic decodes at n=2^20 (d=7, delta=0.1, rho~U[0.1,0.2], SNR~U[30,40] dB), "
                       "%d logged candidates; evaluate: %d seeds at n=2^22, delta=0.1, rho=0.15, SNR 30 dB, and "
                       "%d at n=2^20, delta=0.1, rho=0.1, SNR 40 dB" % (train_instances, F.shape[0], eval_instances,
                                                                       eval_instances),
           "train_loss": loss, "train_s": t_train}

    def evaluate(n, rho, snr, arms, control):
        m = int(0.1 * n)
        k = int(rho * m)
        sn = gm.sigma_from_snr(d, k / m, snr)
        rows = {}
        for i in range(eval_instances):
            A = rl0.Expander.random(n, m, d, seed=80000 + i)
            x, _ = gm.draw_signal(n, k, 1.0, 80000 + i)
            y = rl0.sketch(A, torch.from_numpy(x).cuda(), sigma_n=sn, noise_seed=81000 + i)
            xl1, xl2 = np.abs(x).sum(), np.linalg.norm(x)
            tol = min((m * sn * math.sqrt(2 / math.pi) + math.sqrt(m * sn * sn * (1 - 2 / math.pi))) / xl1, 0.1)

            def score(xr):
                xr = xr.cpu().numpy().astype(np.float64)
                e1 = float(np.abs(xr - x).sum() / xl1)
                return float(e1 <= tol), e1, float(np.linalg.norm(xr - x) / xl2)

            for name, extra in arms:
                rl0.decode(A, y, k, sigma_n=sn, **extra)
                flush.zero_()
                xh, st = rl0.decode(A, y, k, sigma_n=sn, **extra)
                rows.setdefault(name, []).append((st["ms"], st["rounds"] - st["skipped_rounds"],
                                                  st["analytic_rounds"]) + score(xh))
                if control and name == "analytic":
                    rows.setdefault("analytic_second_sweep", []).append((0.0, 0.0, 0.0) + score(
                        _analytic_restart(rl0, A, y, k, sn, xh)))
            A.free()
        out = {"n": n, "m": m, "k": k, "snr_db": snr, "seeds": eval_instances}
        for name, v in rows.items():
            v = np.array(v, dtype=float)
            r = {"success_rate": float(v[:, 3].mean()), "rel_l1_err": float(v[:, 4].mean()),
                 "rel_l2_err": float(v[:, 5].mean())}
            if name != "analytic_second_sweep":
                r.update({"ms_to_recover": float(v[:, 0].mean()), "rounds_launched": float(v[:, 1].mean()),
                          "value": float(n * d * v[:, 1].mean() / (v[:, 0].mean() * 1e-3)), "unit": UNIT})
                if "learned" in name:
                    r["analytic_continuation_rounds"] = float(v[:, 2].mean())
            out[name] = r
        return out

    res["n2e22_rho0.15_snr30"] = evaluate(1 << 22, 0.15, 30.0, [("analytic", {}), ("learned", {"scorer": 1, "mlp": wb})],
                                          True)
    res["n2e20_rho0.10_snr40"] = evaluate(1 << 20, 0.10, 40.0, [
        ("analytic", {}), ("learned_threshold_0.9", {"scorer": 1, "mlp": wb, "mlp_threshold": 0.9})], False)
    # the top-level arms: the n=2^22 evaluation
    res["analytic"] = res["n2e22_rho0.15_snr30"]["analytic"]
    res["learned"] = res["n2e22_rho0.15_snr30"]["learned"]
    return res


def bench_adaptive(rl0, torch, A, y_dev, x, k, params, flush, steps):
    """The adaptive_k variant of the same decode (Table "variants"): its rounds run one
    at a time with the host's adaptive_k step after every accepted round, so it is
    timed on the device stream around the whole call, L2 flushed in between."""
    import numpy as np
    stream = torch.cuda.current_stream()
    p = dict(params, adaptive_k=True)
    rl0.decode(A, y_dev, k, **p)
    ms, st = [], None
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xh, st = rl0.decode(A, y_dev, k, **p)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    xr = xh.cpu().numpy().astype(np.float64)
    t = float(np.mean(ms))
    nnz = A.n * A.d
    return {"workload": "same instance, adaptive_k=1 (Robust-l0-adaptive%s)" % ("-quantised" if params.get("quantised") else ""),
            "ms_to_recover": t, "rounds": st["rounds"], "accepted_rounds": st["accepted_rounds"],
            "converged": st["converged"], "rel_l1_err": float(np.abs(xr - x).sum() / np.abs(x).sum()),
            "value": nnz * (st["rounds"] - st["skipped_rounds"]) / (t * 1e-3), "unit": UNIT,
            "launches": st["launches"]}


def bench_parallel_l0(rl0, torch, A, x_dev, x, flush, steps):
    """Alg. 1 (Parallel-l0) on the noiseless sketch of the bench signal, same expander."""
    import numpy as np
    y0 = rl0.sketch(A, x_dev, sigma_n=0.0, noise_seed=0)
    rl0.parallel_l0(A, y0)
    ms, st = [], None
    for _ in range(steps):
        flush.zero_()
        xh, st = rl0.parallel_l0(A, y0)
        ms.append(st["ms"])
    xr = xh.cpu().numpy().astype(np.float64)
    t = float(np.mean(ms))
    return {"workload": "same expander and signal, noiseless y = A x, tol 1e-5, alpha = floor(d/2)+1",
            "ms_to_recover": t, "iterations": st["accepted_rounds"], "converged": st["converged"],
            "max_abs_err": float(np.abs(xr - x).max()),
            "value": A.n * A.d * st["rounds"] / (t * 1e-3), "unit": UNIT}


def host_description():
    """nproc and the CPU model of this host (lscpu's 'Model name', else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def _bench_inputs(cfg, seed):
    import numpy as np
    import gm
    import oracle
    n, m, k, d, sn = cfg["n"], cfg["m"], cfg["k"], cfg["d"], cfg["sigma_n"]
    rows = oracle.make_expander(n, m, d, seed)
    x, _ = gm.draw_signal(n, k, 1.0, seed)
    y = oracle.sketch(rows, x.astype(np.float64), m, sigma_n=sn, noise_seed=seed + 1)
    return rows, y.astype(np.float32).astype(np.float64)


def cpu_baseline(cfg, seed, budget_s=20.0):
    """The FP64 oracle as it stands, on this host's cores: its OpenMP build (the columns of
    a round shared among all cores) decoding the whole n=2^20 instance, best of 3, and the
    serial build on a bounded sample (full-size rounds from x_hat = 0 until ~budget_s);
    both also decode the n=4096 workload, best of 5."""
    import numpy as np
    import gm
    import oracle
    n, k, d, sn = cfg["n"], cfg["k"], cfg["d"], cfg["sigma_n"]
    rows, y = _bench_inputs(cfg, seed)
    host = host_description()
    threads = int(os.environ.get("OMP_NUM_THREADS", host["nproc"] or 1))
    # OpenMP build: whole decodes
    best, rounds = None, 0
    with oracle.openmp():
        for _ in range(3):
            t0 = time.perf_counter()
            _, st, _ = oracle.decode(rows, y, k, sigma_n=sn)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
            rounds = st["rounds"]
    # serial build: a bounded sample of full-size rounds
    xh, rh = np.zeros(n), y.copy()
    r1, t0 = 0, time.perf_counter()
    while True:
        xp, rp, _, _ = oracle.round_step(rows, y, k, r1 + 1, xh, rh, sigma_n=sn)
        r1 += 1
        if np.abs(rp).sum() < np.abs(rh).sum():
            xh, rh = xp, rp
        if time.perf_counter() - t0 > budget_s or r1 >= 40:
            break
    dt1 = time.perf_counter() - t0
    # the n=4096 workload, both builds, best of 5 whole decodes
    small = gm.config_small()
    I = gm.instance(seed=0, **small)
    ys = (oracle.sketch(I.rows, I.x.astype(np.float64), I.m) + I.eta.astype(np.float64)).astype(np.float32)
    ys = ys.astype(np.float64)

    def best5(par):
        b = None
        for _ in range(5):
            t0_ = time.perf_counter()
            if par:
                with oracle.openmp():
                    oracle.decode(I.rows, ys, I.k, sigma_n=I.sigma_n)
            else:
                oracle.decode(I.rows, ys, I.k, sigma_n=I.sigma_n)
            b = min(b, time.perf_counter() - t0_) if b is not None else time.perf_counter() - t0_
        return b

    small_omp, small_ser = best5(True), best5(False)
    return {"value": n * d * rounds / best, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "whole n=2^20 decode (%d rounds, all columns scored each round), OpenMP build of the FP64 "
                      "oracle on %d threads, best of 3: %.2f s" % (rounds, threads, best),
            "host": host,
            "decode_s_openmp": best, "round_s_openmp": best / rounds,
            "serial": {"value": n * d * r1 / dt1, "unit": UNIT, "cores": 1, "round_s": dt1 / r1,
                       "sample": "%d full-size rounds from x_hat=0, serial build, %.1f s" % (r1, dt1)},
            "n4096_decode_s": {"openmp": small_omp, "serial": small_ser}}


def run_reference(args, cfg):
    """The reference arm: the FP64 oracle (the only reference this project has), its OpenMP
    build on all host cores, on the benchmark's instance; each step is one full-size round
    of the decode (bounded: a whole decode runs for seconds)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    n, k, d, sn = cfg["n"], cfg["k"], cfg["d"], cfg["sigma_n"]
    rows, y = _bench_inputs(cfg, rank_seed(0))
    host = host_description()
    threads = int(os.environ.get("OMP_NUM_THREADS", host["nproc"] or 1))
    xh = np.zeros(n)
    rh = y.copy()

    def one(r):
        nonlocal xh, rh
        with oracle.openmp():
            xp, rp, _, _ = oracle.round_step(rows, y, k, 1 + (r % 39), xh, rh, sigma_n=sn)
        if np.abs(rp).sum() < np.abs(rh).sum():
            xh, rh = xp, rp

    for w in range(args.warmup):
        one(w)
    t0 = time.perf_counter()
    for s in range(args.steps):
        one(args.warmup + s)
    dt = time.perf_counter() - t0
    value = n * d * args.steps / dt
    sample = ("each step: one full-size round of the n=2^20 decode (FP64 oracle, OpenMP build, %d threads)"
              % threads)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_dict(cfg, "continuous", {"reference": "FP64 CPU oracle (plain C, OpenMP)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "host": host},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quantised", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=4096, help="instances of the batched sub-measurement (0: skip)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-scorer sub-measurement")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the adaptive_k sub-measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    cfg = workload()
    if args.impl == "reference":
        return run_reference(args, cfg)

    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import gm
    import paper_1704_09012_gb300 as rl0
    from paper_1704_09012_gb300 import build as _b
    _b.build()
    n, m, k, d, sn = cfg["n"], cfg["m"], cfg["k"], cfg["d"], cfg["sigma_n"]
    nnz = n * d
    seed = rank_seed(rank)
    A = rl0.Expander.random(n, m, d, seed=seed)
    x, _ = gm.draw_signal(n, k, 1.0, seed)
    x_dev = torch.from_numpy(x).cuda()
    y_dev = rl0.sketch(A, x_dev, sigma_n=sn, noise_seed=seed + 1)
    xhat = torch.empty(n, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    params = dict(sigma_n=sn, quantised=args.quantised)
    variant = "quantised" if args.quantised else "continuous"
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        rl0.decode(A, y_dev, k, out=xhat, **params)
    # ---- timed region: K whole decodes, device-timed, L2 flushed in between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    barrier()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            _, st = rl0.decode(A, y_dev, k, out=xhat, **params)
            ev[s][1].record(stream)
            stats.append(st)
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(step_ms) / 1e3
    # throughput counts the rounds that ran kernels (the t = 1 round is only recorded)
    sweep_rounds = stats[-1]["rounds"]
    rounds = sweep_rounds - stats[-1]["skipped_rounds"]
    t_dev = max_over_ranks(t_dev, ws, "cuda")
    value = job_throughput(args.steps * nnz * rounds, ws, t_dev)
    xr = xhat.cpu().numpy().astype(np.float64)
    rel_l1 = float(np.abs(xr - x).sum() / np.abs(x).sum())

    # ---- e2e: the same decode through the host-buffer C-ABI call (copies inside the timed region)
    y_host = y_dev.cpu().pin_memory()
    x_host = torch.empty(n, dtype=torch.float32).pin_memory()
    for _ in range(2):
        rl0.decode_host(A, y_host, k, out=x_host, **params)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for s in range(args.steps):
        flush.zero_()
        ev2[s][0].record(stream)
        rl0.decode_host(A, y_host, k, out=x_host, **params)
        ev2[s][1].record(stream)
    barrier()
    t_e2e = sum(a.elapsed_time(b) for a, b in ev2) / 1e3
    t_e2e = max_over_ranks(t_e2e, ws, "cuda")
    e2e_value = job_throughput(args.steps * nnz * rounds, ws, t_e2e)

    # ---- per-kernel device time: event nodes captured around each kernel group
    prof = []
    for s in range(args.steps):
        flush.zero_()
        _, st = rl0.decode(A, y_dev, k, out=xhat, profile=True, **params)
        prof.append(st)
    launches_score = rounds * len(prof)
    ms_score = sum(p["ms_score"] for p in prof) / launches_score
    alg_bytes = 4 * nnz + 8 * m          # row ids (4 B per nonzero) + (r, p_z) of every row once
    achieved = alg_bytes / (ms_score * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    group_ms = {g: sum(p["ms_" + g] for p in prof) / len(prof) for g in ("score", "hk", "rebuild", "accept")}
    l2_peak = l2_copy_peak(torch)
    l2_read = l2_read_peak(torch)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(cfg, variant, {"rounds_per_decode": sweep_rounds, "rounds_launched_per_decode": rounds, "parallelism": "replicas" if ws > 1 else "1 GPU"}),
        "ms_to_recover": 1e3 * t_dev / args.steps,
        "recovery": {"converged": stats[-1]["converged"], "support": stats[-1]["support_size"],
                     "rel_l1_err": rel_l1, "accepted_rounds": stats[-1]["accepted_rounds"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * m, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": stats[-1]["launches"] * args.steps,
        "roofline": {"bound": "hbm", "kernel": "k_column_score_res", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic_for("k_column_score_res"), "alg_bytes_per_launch": alg_bytes,
                     "avg_launch_ms": ms_score,
                     # inside a decode the row ids stay in L2 after the first round: the same
                     # bytes against the larger of two L2-resident figures measured here, reads
                     # (reductions) and copies (read + write bytes)
                     "l2": {"peak": max(l2_read[0], l2_peak[0]), "unit": "GB/s",
                            "frac": achieved / max(l2_read[0], l2_peak[0]),
                            "peak_source": "measured: the larger of L2-resident reads (20 reductions back to back "
                                           "of %d MiB: %.0f GB/s) and copies (20 back to back, 2 x %d MiB: %.0f GB/s)"
                                           % (l2_read[1], l2_read[0], l2_peak[1], l2_peak[0]),
                            "read_peak": l2_read[0], "copy_peak": l2_peak[0]}},
        "kernel_group_ms_per_decode": group_ms,
        "clocks": clk.summary(),
        "wall_s": t_wall,
    }
    if args.batched > 0:
        line["batched"] = bench_batched(rl0, torch, args.batched, max(1, min(args.steps, 3)), flush)
    if not args.no_adaptive:
        line["adaptive"] = bench_adaptive(rl0, torch, A, y_dev, x, k, params, flush, max(1, min(args.steps, 3)))
        line["parallel_l0"] = bench_parallel_l0(rl0, torch, A, x_dev, x, flush, max(1, min(args.steps, 3)))
    if not args.no_learned:
        line["learned"] = bench_learned(rl0, torch, flush)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, seed)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
