"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of
oracle/rl0_oracle.c (a dropped or doubled term, a wrong index, a reversed test, a
swapped operand), builds the copy, and runs the oracle pin files against it through
RL0_ORACLE_LIB: at least one pin must fail, other than the restatements (the literal
Python round, the NumPy copy of the network).  The unmutated copy must pass, so that a
broken harness cannot pass for a caught mistake."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rl0_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_adaptive.py", "tests/test_oracle_mlp.py"]
# restatements are left out (the literal Python round, the NumPy copy of the
# network): a catch must come from a pin that does not retype the oracle
RESTATEMENTS = ["tests/test_oracle_pins.py::test_one_round_matches_a_literal_python_round",
                "tests/test_oracle_mlp.py::test_c_and_numpy_forward_agree"]

MUTANTS = [
    ("posterior variance counts the noise twice (Eq. pz_gaussian)",
     "S->v[q] = q * s2 + v_noise;", "S->v[q] = q * s2 + 2.0 * v_noise;"),
    ("tail variance with R(ell) in place of R(ell-1)",
     "S->v_tail = (s2 * lam * R_lm1 + v_noise * R_l) / R_l;", "S->v_tail = (s2 * lam * R_l + v_noise * R_l) / R_l;"),
    ("Poisson tail recurrence off by one",
     "term *= lam / (q + 1);", "term *= lam / (q + 2);"),
    ("p_e without the doubled noise variance (Eq. pe_gaussian)",
     "double vn = (which == 0) ? n2 : 2.0 * n2;", "double vn = (which == 0) ? n2 : n2;"),
    ("p_e with rate d rho in place of 2 d rho",
     "double lam = (which == 0) ? d * rho : 2.0 * d * rho;", "double lam = (which == 0) ? d * rho : d * rho;"),
    ("p_z and p_e swapped in the decoder",
     "int rc = orc_posterior_series(&P->pz, 0,", "int rc = orc_posterior_series(&P->pz, 1,"),
    ("n_z sums 1 - q_z",
     "nz += orc_qz(P, p->quantised, rl[l], t);", "nz += 1.0 - orc_qz(P, p->quantised, rl[l], t);"),
    ("anchor test against log t in place of log(1 - t)",
     "double lim = (t >= 1.0) ? -INFINITY : log(1.0 - t);\n    if (t <= 0.0) return 1;",
     "double lim = (t <= 0.0) ? -INFINITY : log(t);\n    if (t <= 0.0) return 1;"),
    ("consensus value from the anchor's residual",
     "num += rl[l] * q;", "num += ri * q;"),
    ("l1 test reversed",
     "} else if (lhs <= rhs && score >= p->alpha) {", "} else if (lhs >= rhs && score >= p->alpha) {"),
    ("the update overwrites x_j instead of adding omega",
     "if (best >= 0) { xp[j] = xh[j] + best_w; upd++; }", "if (best >= 0) { xp[j] = best_w; upd++; }"),
    ("H_k breaks ties towards the larger index",
     "return (u->j > v->j) - (u->j < v->j);", "return (u->j < v->j) - (u->j > v->j);"),
    ("residual with the sign reversed",
     "rp[i] = yhat[i] - rp[i];", "rp[i] = rp[i] - yhat[i];"),
    ("stop level m sigma sqrt(1/pi) in place of m sigma sqrt(2/pi)",
     "return (double)m * p->sigma_n * sqrt(2.0 / ORC_PI);", "return (double)m * p->sigma_n * sqrt(1.0 / ORC_PI);"),
    ("adaptive_k floor at m/10",
     "double floor_k = floor((double)m / 100.0);", "double floor_k = floor((double)m / 10.0);"),
    ("adaptive_k sums p_z in place of 1 - p_z",
     "if (xhat[j] != 0.0) s += 1.0 - exp(orc_log_pbreve(&P->pz, xhat[j]));",
     "if (xhat[j] != 0.0) s += exp(orc_log_pbreve(&P->pz, xhat[j]));"),
    ("one round too few in the sweep",
     "return (int)ceil(1.0 / c - 1e-9);", "return (int)ceil(1.0 / c - 1e-9) - 1;"),
    ("expander columns may repeat a row",
     "if (!dup) col[got++] = cand;", "col[got++] = cand;"),
    ("quantised q_z test reversed",
     "return (lp >= lim) ? 1.0 : 0.0;", "return (lp <= lim) ? 1.0 : 0.0;"),
    ("quantised q_e thresholded at 1 - t in place of t",
     "return (lp >= log(t)) ? 1.0 : 0.0;", "return (lp >= log(1.0 - t)) ? 1.0 : 0.0;"),
    ("learned scorer: second hidden layer without its ReLU",
     "out += (a > 0.0 ? a : 0.0) * w3[o];", "out += a * w3[o];"),
    ("learned scorer: first weight matrix read transposed",
     "for (int i = 0; i < ORC_NFEAT; ++i) a += f[i] * W1[i * ORC_HID + o];",
     "for (int i = 0; i < ORC_NFEAT; ++i) a += f[i] * W1[o * ORC_NFEAT + i];"),
    ("learned scorer: n_e and n_z features swapped",
     "f[7] = ne / d;\n    f[8] = nz / d;", "f[7] = nz / d;\n    f[8] = ne / d;"),
]


def _run_pins(tmp_path, text):
    c = tmp_path / "orc.c"
    c.write_text(text)
    so = tmp_path / "liborc.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, RL0_ORACLE_LIB=str(so))
    deselect = [a for r in RESTATEMENTS for a in ("--deselect", r)]
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS, *deselect],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    """Every copy (the unmutated one under the key None) built and run at once, one
    process per copy, as many at a time as there are cores."""
    src = open(SRC).read()
    jobs = {None: src}
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        jobs[name] = src.replace(old, new)
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        futs = {k: ex.submit(_run_pins, tmp_path_factory.mktemp("orc"), t) for k, t in jobs.items()}
        return {k: f.result() for k, f in futs.items()}


def test_the_unmutated_copy_passes_the_pins(runs):
    r = runs[None]
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(runs, name):
    r = runs[name]
    # exit code 1: collected and ran, and a pin failed (not a collection or usage error)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-2000:])
