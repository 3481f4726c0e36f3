"""FP64 CPU oracle for Robust-l0 decoding (arXiv 1704.09012) -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never uses it; the two
share no code.  The arithmetic lives in ``rl0_oracle.c`` (plain C, double
precision); this module only marshals numpy arrays through ctypes.

Function map (paper anchors):
  philox / make_expander / noise / sketch  -- Def. "Generating model GM"
  log_posterior / tail_constants           -- Eqs. (pz_gaussian), (pe_gaussian),
                                              (pz_approx), (pe_approx), (breve)
  default_c / num_rounds                   -- Eqs. (finetune_c_quant), (finetune_c_cont)
  hard_threshold                           -- H_k of Algorithm 2
  round_step / decode                      -- Algorithm 2 (Robust-l0)
  parallel_l0                              -- Algorithm 1 (Parallel-l0)
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_libs = {}
_use_openmp = False


class Params(C.Structure):
    _fields_ = [
        ("sigma_s", C.c_double),
        ("sigma_n", C.c_double),
        ("quantised", C.c_int),
        ("adaptive_k", C.c_int),
        ("c", C.c_double),
        ("alpha", C.c_double),
        ("ell", C.c_int),
        ("max_rounds", C.c_int),
        ("noiseless_tol", C.c_double),
        ("literal_ei_test", C.c_int),
        ("learned", C.c_int),
        ("mlp", C.c_void_p),
        ("mlp_threshold", C.c_double),
        ("best_anchor", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("rounds", C.c_int),
        ("accepted_rounds", C.c_int),
        ("converged", C.c_int),
        ("support_size", C.c_int64),
        ("final_l1", C.c_double),
        ("c", C.c_double),
        ("alpha", C.c_double),
        ("stop_level", C.c_double),
        ("ell", C.c_int),
        ("nrounds_max", C.c_int),
        ("analytic_rounds", C.c_int),
    ]


class RoundLog(C.Structure):
    _fields_ = [
        ("t", C.c_double),
        ("l1_candidate", C.c_double),
        ("l1_hat", C.c_double),
        ("accepted", C.c_int),
        ("updated", C.c_int64),
        ("support", C.c_int64),
        ("k_prior", C.c_double),
    ]


COLREC_DTYPE = np.dtype([
    ("passed", np.int32), ("best_slot", np.int32), ("omega", np.float64),
    ("score", np.float64), ("nz", np.float64), ("min_margin", np.float64)], align=True)


class openmp:
    """Within this context the oracle calls go to its OpenMP build (the column loop of a
    round shared among the host's cores; same results as the serial build).  Used for
    full-size checks and the multi-core CPU baseline."""

    def __enter__(self):
        global _use_openmp
        self._prev = _use_openmp
        _use_openmp = True
        return self

    def __exit__(self, *a):
        global _use_openmp
        _use_openmp = self._prev


def lib():
    key = bool(_use_openmp) and not os.environ.get("RL0_ORACLE_LIB")
    if key not in _libs:
        # RL0_ORACLE_LIB: a copy of the oracle built elsewhere (the planted-mistake
        # test runs the pins against mutated copies)
        path = os.environ.get("RL0_ORACLE_LIB") or _build.build(openmp=key)
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        i64 = C.c_int64
        L.orc_philox4x32_10.argtypes = [up, up, up]
        L.orc_make_expander.argtypes = [i64, i64, C.c_int, C.c_uint64, ip]
        L.orc_noise.argtypes = [i64, C.c_double, C.c_uint64, dp]
        L.orc_matvec.argtypes = [i64, i64, C.c_int, ip, dp, dp]
        L.orc_sketch.argtypes = [i64, i64, C.c_int, ip, dp, C.c_double, C.c_uint64, dp]
        L.orc_default_c.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_default_c.restype = C.c_double
        L.orc_num_rounds.argtypes = [C.c_double]
        L.orc_hard_threshold.argtypes = [i64, i64, dp]
        L.orc_decode.argtypes = [i64, i64, C.c_int, ip, dp, i64, C.POINTER(Params), dp,
                                 C.POINTER(Stats), C.POINTER(RoundLog), C.c_int]
        L.orc_round.argtypes = [i64, i64, C.c_int, ip, dp, i64, C.POINTER(Params), C.c_int,
                                dp, dp, dp, dp, C.POINTER(C.c_int64), C.c_void_p]
        L.orc_parallel_l0.argtypes = [i64, i64, C.c_int, ip, dp, C.c_double, C.c_double, C.c_int,
                                      dp, C.c_void_p]
        L.orc_log_posterior.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                        C.c_double, C.c_int, C.c_double, i64, dp, dp, C.c_void_p]
        L.orc_tail_constants.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_sizeof.argtypes = [C.c_int]
        L.orc_mlp_logits.argtypes = [dp, i64, dp, dp]
        L.orc_features.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_double, dp]
        assert L.orc_sizeof(0) == C.sizeof(Params)
        assert L.orc_sizeof(1) == C.sizeof(Stats)
        assert L.orc_sizeof(2) == C.sizeof(RoundLog)
        assert L.orc_sizeof(3) == COLREC_DTYPE.itemsize
        _libs[key] = L
    return _libs[key]


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle call failed with code %d" % rc)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox(counter, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (4 + 2 words)."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(counter, np.uint32),
                            np.ascontiguousarray(key, np.uint32), out)
    return out


def make_expander(n, m, d, seed):
    """Column-major (n, d) int32 rows of A, ascending per column (Def. GM item 1)."""
    rows = np.zeros((n, d), np.int32)
    _check(lib().orc_make_expander(n, m, d, seed, rows))
    return rows


def noise(m, sigma_n, seed):
    eta = np.zeros(m, np.float64)
    lib().orc_noise(m, sigma_n, seed, eta)
    return eta


def matvec(rows, x, m):
    rows = _i32(rows)
    n, d = rows.shape
    y = np.zeros(m, np.float64)
    lib().orc_matvec(n, m, d, rows, _f64(x), y)
    return y


def sketch(rows, x, m, sigma_n=0.0, noise_seed=0):
    """y_hat = A x + eta in FP64 (Def. GM item 6)."""
    rows = _i32(rows)
    n, d = rows.shape
    y = np.zeros(m, np.float64)
    lib().orc_sketch(n, m, d, rows, _f64(x), sigma_n, noise_seed, y)
    return y


def default_c(quantised, delta, rho):
    return lib().orc_default_c(int(quantised), float(delta), float(rho))


def num_rounds(c):
    return lib().orc_num_rounds(float(c))


def hard_threshold(x, k):
    x = np.array(x, dtype=np.float64, copy=True)
    _check(lib().orc_hard_threshold(x.size, k, x))
    return x


_keep = []


def make_params(sigma_s=1.0, sigma_n=0.0, quantised=False, c=0.0, alpha=0.0, ell=0,
                max_rounds=0, noiseless_tol=0.0, literal_ei_test=False, mlp_bf16=None, mlp_threshold=0.0,
                adaptive_k=False, best_anchor=False):
    """mlp_bf16: the learned scorer's parameters as a uint16 array of BF16 bit patterns
    (enables the learned rule); None keeps Algorithm 2's analytic rule."""
    ptr = None
    if mlp_bf16 is not None:
        arr = np.ascontiguousarray(mlp_bf16, dtype=np.uint16)
        _keep.append(arr)
        del _keep[:-8]
        ptr = arr.ctypes.data
    return Params(sigma_s, sigma_n, int(quantised), int(adaptive_k), c, alpha, ell, max_rounds,
                  noiseless_tol, int(literal_ei_test), int(mlp_bf16 is not None), ptr, mlp_threshold,
                  int(best_anchor))


def decode(rows, yhat, k, log_cap=256, **kw):
    """Algorithm 2.  Returns (x_hat float64[n], stats dict, per-round log list)."""
    rows = _i32(rows)
    n, d = rows.shape
    yhat = _f64(yhat)
    m = yhat.size
    p = make_params(**kw)
    x = np.zeros(n, np.float64)
    st = Stats()
    logs = (RoundLog * log_cap)()
    _check(lib().orc_decode(n, m, d, rows, yhat, k, C.byref(p), x, C.byref(st), logs, log_cap))
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    rl = [{f: getattr(logs[i], f) for f, _ in RoundLog._fields_} for i in range(min(st.rounds, log_cap))]
    return x, stats, rl


def round_step(rows, yhat, k, round_index, xh, rh, **kw):
    """One round of Algorithm 2 from the injected state (xh, rh).

    Returns (x' after H_k, r = y - A x', updated count, per-column records)."""
    rows = _i32(rows)
    n, d = rows.shape
    yhat = _f64(yhat)
    m = yhat.size
    p = make_params(**kw)
    xp = np.zeros(n, np.float64)
    rp = np.zeros(m, np.float64)
    upd = C.c_int64(0)
    rec = np.zeros(n, COLREC_DTYPE)
    _check(lib().orc_round(n, m, d, rows, yhat, k, C.byref(p), round_index, _f64(xh), _f64(rh),
                           xp, rp, C.byref(upd), rec.ctypes.data))
    return xp, rp, upd.value, rec


def parallel_l0(rows, y, alpha=None, tol=1e-9, max_iter=100, history=False):
    """Algorithm 1.  Returns (x_hat, iterations[, per-iteration x_hat])."""
    rows = _i32(rows)
    n, d = rows.shape
    y = _f64(y)
    m = y.size
    if alpha is None:
        alpha = d // 2 + 1
    x = np.zeros(n, np.float64)
    hist = np.zeros((max_iter, n), np.float64) if history else None
    it = lib().orc_parallel_l0(n, m, d, rows, y, float(alpha), float(tol), max_iter, x,
                               hist.ctypes.data if history else None)
    if it < 0:
        _check(it)
    if history:
        return x, it, hist[:it]
    return x, it


def log_posterior(which, w, d, rho, sigma_s, sigma_n, ell=4, exact=False, tol=1e-5, raw=False):
    """log p_breve (Eq. breve) of p_z (which='z') or p_e (which='e') at the points w.

    exact=False: Eq. (p*_approx) with ell explicit terms and the Gaussian tail.
    exact=True : the series of Eq. (p*_gaussian) kept to ell terms with no tail
                 (use a large ell for the untruncated series)."""
    w = _f64(np.atleast_1d(w))
    out = np.zeros_like(w)
    rawv = np.zeros_like(w) if raw else None
    _check(lib().orc_log_posterior(0 if which == "z" else 1, 1 if exact else 0, d, rho, sigma_s,
                                   sigma_n, ell, tol, w.size, w, out,
                                   rawv.ctypes.data if raw else None))
    return (out, rawv) if raw else out


def tail_constants(which, d, rho, sigma_s, sigma_n, ell):
    R = C.c_double()
    v = C.c_double()
    _check(lib().orc_tail_constants(0 if which == "z" else 1, d, rho, sigma_s, sigma_n, ell,
                                    C.byref(R), C.byref(v)))
    return R.value, v.value


def mlp_logits(W, F):
    """Logits of the learned scorer's network (FP64) for rows F (n x 16)."""
    W = _f64(W)
    F = _f64(np.atleast_2d(F))
    out = np.zeros(F.shape[0])
    lib().orc_mlp_logits(W, F.shape[0], F, out)
    return out


def features(rl, w, ne, nz, lhs, rhs, sigma_n, t, drho):
    """The learned scorer's 16 features of one candidate (FP64)."""
    rl = _f64(rl)
    f = np.zeros(16)
    lib().orc_features(rl.size, rl, w, ne, nz, lhs, rhs, sigma_n, t, drho, f)
    return f


def bf16_to_f64(bits):
    """BF16 bit patterns (uint16) -> float64, exactly."""
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
