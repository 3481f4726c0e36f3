"""GB300 (sm_103a) Robust-l0 decoding (Mendoza-Smith, Tanner, Wechsung, arXiv 1704.09012).

Thin Python binding of the C ABI declared in ``include/rl0.h``: argument marshalling
only.  Every step of the decoder runs in the CUDA library ``_build/librl0.so``; PyTorch
supplies device memory and streams.  There is no CPU fallback: if the library has not
been built (``python -m paper_1704_09012_gb300.build`` or ``__graft_entry__.build()``),
loading fails with an error.

    import torch
    import paper_1704_09012_gb300 as rl0
    A = rl0.Expander.random(n, m, d, seed=0)          # Def. "Generating model", item 1
    y = rl0.sketch(A, x, sigma_n=1e-3, noise_seed=1)   # y_hat = A x + eta
    xhat, stats = rl0.decode(A, y, k, sigma_n=1e-3)    # Algorithm 2
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librl0.so")

RL0_OK = 0
ERRORS = {
    -1: "RL0_ERR_INVALID_ARG", -2: "RL0_ERR_CUDA", -3: "RL0_ERR_ALLOC", -4: "RL0_ERR_TIMEOUT",
    -5: "RL0_ERR_UNSUPPORTED", -6: "RL0_ERR_INVALID_A", -7: "RL0_ERR_INVALID_Y", -8: "RL0_ERR_TOO_LARGE",
}

# Every symbol include/rl0.h declares.
EXPORTS = [
    "rl0_make_expander", "rl0_expander_from_rows", "rl0_expander_rows", "rl0_expander_shape",
    "rl0_free_expander", "rl0_sketch", "rl0_decode", "rl0_decode_host", "rl0_round_step",
    "rl0_decode_batched", "rl0_decode_log", "rl0_strerror", "rl0_decode_static", "rl0_expander_set_wait_polls",
    "rl0_parallel_l0",
    "rl0_posterior_mc",
    "rl0_candidate_features", "rl0_scorer_log", "rl0_mlp_init", "rl0_mlp_grad", "rl0_mlp_train", "rl0_mlp_export",
    "rl0_mlp_forward", "rl0_mlp_params",
]
MLP_PARAMS = 1633
NFEAT = 16


class Rl0Error(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%s)" % (what, ERRORS.get(code, code), _lib().rl0_strerror(code).decode()))


class Params(C.Structure):
    _fields_ = [
        ("sigma_s", C.c_double), ("sigma_n", C.c_double), ("quantised", C.c_int), ("adaptive_k", C.c_int),
        ("c", C.c_double), ("alpha", C.c_double), ("ell", C.c_int), ("scorer", C.c_int),
        ("mlp", C.c_void_p), ("mlp_threshold", C.c_double), ("max_rounds", C.c_int),
        ("noiseless_tol", C.c_double), ("profile", C.c_int), ("anchor_rule", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("rounds", C.c_int), ("accepted_rounds", C.c_int), ("converged", C.c_int), ("status", C.c_int),
        ("support_size", C.c_int64), ("final_l1", C.c_double), ("ms", C.c_float), ("hk_rounds", C.c_int),
        ("fallback_rounds", C.c_int), ("ms_score", C.c_float), ("ms_hk", C.c_float),
        ("ms_rebuild", C.c_float), ("ms_accept", C.c_float), ("launches", C.c_int),
        ("analytic_rounds", C.c_int), ("skipped_rounds", C.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RoundRecord(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("l1_candidate", C.c_double), ("l1_hat", C.c_double), ("accepted", C.c_int),
        ("updated", C.c_int), ("support", C.c_int), ("hk_dropped", C.c_int), ("k_prior", C.c_double),
    ]


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: build it with "
                               "`python -m paper_1704_09012_gb300.build` (no CPU fallback exists)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        L.rl0_make_expander.argtypes = [i64, i64, i32, C.c_uint64, vp, C.POINTER(vp)]
        L.rl0_expander_from_rows.argtypes = [i64, i64, i32, vp, vp, C.POINTER(vp)]
        L.rl0_expander_rows.argtypes = [vp, vp, vp]
        L.rl0_expander_shape.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]
        L.rl0_free_expander.argtypes = [vp]
        L.rl0_free_expander.restype = None
        L.rl0_sketch.argtypes = [vp, vp, C.c_double, C.c_uint64, vp, vp]
        L.rl0_decode.argtypes = [vp, vp, i64, C.POINTER(Params), vp, C.POINTER(Stats), vp]
        L.rl0_decode_host.argtypes = [vp, vp, i64, C.POINTER(Params), vp, C.POINTER(Stats), vp]
        L.rl0_round_step.argtypes = [vp, vp, i64, C.POINTER(Params), i32, vp, vp, vp, vp, vp,
                                     C.POINTER(C.c_double), vp]
        L.rl0_decode_batched.argtypes = [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(i64), vp,
                                         C.POINTER(vp), vp, vp]
        L.rl0_decode_log.argtypes = [vp, C.POINTER(RoundRecord), i32]
        L.rl0_decode_static.argtypes = [vp, vp, i64, C.POINTER(Params), vp, C.POINTER(Stats), vp]
        L.rl0_expander_set_wait_polls.argtypes = [vp, i64]
        L.rl0_parallel_l0.argtypes = [vp, vp, C.c_double, C.c_double, i32, vp, C.POINTER(Stats), vp]
        L.rl0_posterior_mc.argtypes = [vp, vp, vp, i64, C.c_double, C.c_double, i32, C.c_double, C.c_double,
                                       vp, vp, vp]
        L.rl0_candidate_features.argtypes = [vp, vp, i64, C.POINTER(Params), i32, vp, vp, vp, vp, vp, i32,
                                             C.POINTER(i32), vp]
        L.rl0_scorer_log.argtypes = [vp, vp, i64, C.POINTER(Params), vp, C.c_float, i32, vp, vp, i64,
                                     C.POINTER(i64), C.POINTER(i32), vp]
        L.rl0_mlp_init.argtypes = [C.c_uint64, vp, vp]
        L.rl0_mlp_grad.argtypes = [vp, vp, vp, i64, vp, C.POINTER(C.c_double), vp]
        L.rl0_mlp_train.argtypes = [vp, vp, vp, i64, i32, i32, C.c_float, vp, C.POINTER(C.c_double), vp]
        L.rl0_mlp_export.argtypes = [vp, vp, vp]
        L.rl0_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        L.rl0_mlp_params.argtypes = []
        assert L.rl0_mlp_params() == MLP_PARAMS
        L.rl0_strerror.argtypes = [i32]
        L.rl0_strerror.restype = C.c_char_p
        _L = L
    return _L


def lib_path():
    return LIB_PATH


def _check(rc, what):
    if rc != RL0_OK:
        raise Rl0Error(rc, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype, n=None, what="tensor"):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (what, dtype))
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements, has %d" % (what, n, t.numel()))
    return C.c_void_p(t.data_ptr())


def make_params(sigma_s=1.0, sigma_n=0.0, quantised=False, c=0.0, alpha=0.0, ell=0, scorer=0, mlp=None,
                mlp_threshold=0.0, max_rounds=0, noiseless_tol=0.0, adaptive_k=False, profile=False, anchor_rule=0):
    mlp_ptr = mlp.data_ptr() if isinstance(mlp, torch.Tensor) else mlp
    return Params(sigma_s, sigma_n, int(quantised), int(adaptive_k), c, alpha, ell, scorer, mlp_ptr,
                  mlp_threshold, max_rounds, noiseless_tol, int(profile), int(anchor_rule))


class Expander:
    """Device-resident expander A (Def. 1.1) plus its decode workspace."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)
        n, m, d = C.c_int64(), C.c_int64(), C.c_int()
        _check(_lib().rl0_expander_shape(self._h, C.byref(n), C.byref(m), C.byref(d)), "rl0_expander_shape")
        self.n, self.m, self.d = n.value, m.value, d.value

    @classmethod
    def random(cls, n, m, d, seed=0, stream=None):
        h = C.c_void_p()
        _check(_lib().rl0_make_expander(n, m, d, seed, _stream(stream), C.byref(h)), "rl0_make_expander")
        return cls(h.value)

    @classmethod
    def from_rows(cls, rows, m, stream=None):
        """rows: CUDA int32 (n, d), column-major row lists (each column ascending)."""
        n, d = rows.shape
        h = C.c_void_p()
        _check(_lib().rl0_expander_from_rows(n, m, d, _dev(rows, torch.int32, n * d, "rows"), _stream(stream),
                                             C.byref(h)), "rl0_expander_from_rows")
        return cls(h.value)

    def rows(self, stream=None):
        out = torch.empty((self.n, self.d), dtype=torch.int32, device="cuda")
        _check(_lib().rl0_expander_rows(self._h, C.c_void_p(out.data_ptr()), _stream(stream)), "rl0_expander_rows")
        return out

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            _lib().rl0_free_expander(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sketch(A, x, sigma_n=0.0, noise_seed=0, stream=None):
    """y_hat = A x + eta (Def. "Generating model", items 4 and 6); x CUDA float32 [n]."""
    y = torch.empty(A.m, dtype=torch.float32, device="cuda")
    _check(_lib().rl0_sketch(A.handle, _dev(x, torch.float32, A.n, "x"), float(sigma_n), int(noise_seed),
                             C.c_void_p(y.data_ptr()), _stream(stream)), "rl0_sketch")
    return y


def decode(A, y, k, out=None, stream=None, **params):
    """Algorithm 2 on one instance.  Returns (x_hat CUDA float32 [n], stats dict)."""
    p = make_params(**params)
    x = out if out is not None else torch.empty(A.n, dtype=torch.float32, device="cuda")
    st = Stats()
    _check(_lib().rl0_decode(A.handle, _dev(y, torch.float32, A.m, "y"), int(k), C.byref(p),
                             _dev(x, torch.float32, A.n, "x_hat"), C.byref(st), _stream(stream)), "rl0_decode")
    return x, st.as_dict()


def decode_static(A, y, k, out=None, stream=None, **params):
    """rl0_decode without any allocation (fixed workspace inside the library; n <= 65536,
    m <= 32768).  For callers that cannot allocate device memory while they run (a memory
    budget fixed at start-up, or an allocator of their own that owns the free memory);
    `out` lets them pass a preallocated x_hat as well.  Calls share the workspace: do not
    overlap them."""
    p = make_params(**params)
    x = out if out is not None else torch.empty(A.n, dtype=torch.float32, device="cuda")
    st = Stats()
    _check(_lib().rl0_decode_static(A.handle, _dev(y, torch.float32, A.m, "y"), int(k), C.byref(p),
                                    _dev(x, torch.float32, A.n, "x_hat"), C.byref(st), _stream(stream)),
           "rl0_decode_static")
    return x, st.as_dict()


def set_wait_polls(A, polls):
    """Failure-detection test hook (rl0_expander_set_wait_polls): polls >= 0 makes the column
    kernel's first bounded wait on A give up after that many polls (0: at once), so the next
    decode returns RL0_ERR_TIMEOUT; polls < 0 restores the built-in limit."""
    _check(_lib().rl0_expander_set_wait_polls(A.handle, int(polls)), "rl0_expander_set_wait_polls")


def parallel_l0(A, y, alpha=0.0, tol=0.0, max_iter=0, out=None, stream=None):
    """Algorithm 1 (Parallel-l0) on the noiseless model y = A x.  Returns (x_hat CUDA
    float32 [n], stats dict); stats["accepted_rounds"] counts the iterations."""
    x = out if out is not None else torch.empty(A.n, dtype=torch.float32, device="cuda")
    st = Stats()
    _check(_lib().rl0_parallel_l0(A.handle, _dev(y, torch.float32, A.m, "y"), float(alpha), float(tol),
                                  int(max_iter), _dev(x, torch.float32, A.n, "x_hat"), C.byref(st),
                                  _stream(stream)), "rl0_parallel_l0")
    return x, st.as_dict()


def posterior_mc(A, y0, yhat, k, sigma_n, sigma_s=1.0, nbins=64, wz_max=None, we_max=None, hz=None, he=None,
                 stream=None):
    """Binned Monte-Carlo counts of the posteriors (rl0_posterior_mc).  Returns the CUDA
    int64 [nbins, 3] histograms (samples, events, sum of 2^32 p_breve) for p_z (rows) and
    p_e (row pairs of each column); pass hz/he to accumulate over instances."""
    wz_max = 8.0 * sigma_n if wz_max is None else wz_max
    we_max = 8.0 * 2 ** 0.5 * sigma_n if we_max is None else we_max
    if hz is None:
        hz = torch.zeros((nbins, 3), dtype=torch.int64, device="cuda")
    if he is None:
        he = torch.zeros((nbins, 3), dtype=torch.int64, device="cuda")
    assert hz.shape == (nbins, 3) and he.shape == (nbins, 3) and hz.is_contiguous() and he.is_contiguous()
    _check(_lib().rl0_posterior_mc(A.handle, _dev(y0, torch.float32, A.m, "y0"), _dev(yhat, torch.float32, A.m, "yhat"),
                                   int(k), float(sigma_s), float(sigma_n), int(nbins), float(wz_max), float(we_max),
                                   C.c_void_p(hz.data_ptr()), C.c_void_p(he.data_ptr()), _stream(stream)),
           "rl0_posterior_mc")
    return hz, he


def decode_host(A, y_host, k, out=None, stream=None, **params):
    """Algorithm 2 with host buffers (the library copies y in and x_hat out)."""
    if y_host.is_cuda or y_host.dtype != torch.float32 or not y_host.is_contiguous() or y_host.numel() != A.m:
        raise ValueError("y_host must be a contiguous CPU float32 tensor of m elements")
    p = make_params(**params)
    x = out if out is not None else torch.empty(A.n, dtype=torch.float32, pin_memory=True)
    st = Stats()
    _check(_lib().rl0_decode_host(A.handle, C.c_void_p(y_host.data_ptr()), int(k), C.byref(p),
                                  C.c_void_p(x.data_ptr()), C.byref(st), _stream(stream)), "rl0_decode_host")
    return x, st.as_dict()


def decode_log(A, cap=1024):
    recs = (RoundRecord * cap)()
    n = _lib().rl0_decode_log(A.handle, recs, cap)
    if n < 0:
        _check(n, "rl0_decode_log")
    return [{f: getattr(recs[i], f) for f, _ in RoundRecord._fields_} for i in range(min(n, cap))]


def round_step(A, y, k, round_index, xhat, rhat, want_passed=True, stream=None, **params):
    """One round from an injected state.  Returns (x', r, passed int32 [n] or None, ||r||_1)."""
    p = make_params(**params)
    xp = torch.empty(A.n, dtype=torch.float32, device="cuda")
    rp = torch.empty(A.m, dtype=torch.float32, device="cuda")
    passed = torch.zeros(A.n, dtype=torch.int32, device="cuda") if want_passed else None
    l1 = C.c_double()
    _check(_lib().rl0_round_step(A.handle, _dev(y, torch.float32, A.m, "y"), int(k), C.byref(p), int(round_index),
                                 _dev(xhat, torch.float32, A.n, "x_hat"), _dev(rhat, torch.float32, A.m, "r_hat"),
                                 C.c_void_p(xp.data_ptr()), C.c_void_p(rp.data_ptr()),
                                 C.c_void_p(passed.data_ptr()) if want_passed else None, C.byref(l1),
                                 _stream(stream)), "rl0_round_step")
    return xp, rp, passed, l1.value


class BatchPlan:
    """The argument arrays of one rl0_decode_batched call, marshalled once: As (list of
    Expander), ys (CUDA float32 [m_i]), ks (ints), params (None, one dict for all, or one
    dict per instance), outs (CUDA float32 [n_i], or None to allocate).  run() makes the
    call and returns (list of x_hat, list of stats dicts); repeated runs reuse the arrays."""

    def __init__(self, As, ys, ks, params=None, outs=None):
        cnt = len(As)
        if not (len(ys) == len(ks) == cnt):
            raise ValueError("As, ys and ks must have the same length")
        if params is None:
            params = {}
        plist = params if isinstance(params, (list, tuple)) else [params] * cnt
        self.cnt = cnt
        self.keep = (list(As), list(ys))
        self.P = (Params * cnt)(*[make_params(**p) for p in plist])
        self.xs = outs if outs is not None else [torch.empty(A.n, dtype=torch.float32, device="cuda") for A in As]
        self.Ah = (C.c_void_p * cnt)(*[A.handle.value for A in As])
        self.Yh = (C.c_void_p * cnt)(*[_dev(y, torch.float32, A.m, "y").value for A, y in zip(As, ys)])
        self.Xh = (C.c_void_p * cnt)(*[_dev(x, torch.float32, A.n, "x_hat").value for A, x in zip(As, self.xs)])
        self.K = (C.c_int64 * cnt)(*[int(k) for k in ks])
        self.S = (Stats * cnt)()

    def run(self, stream=None, stats=True):
        _check(_lib().rl0_decode_batched(self.cnt, self.Ah, self.Yh, self.K, C.cast(self.P, C.c_void_p), self.Xh,
                                         C.cast(self.S, C.c_void_p), _stream(stream)), "rl0_decode_batched")
        return self.xs, ([s.as_dict() for s in self.S] if stats else None)


def decode_batched(As, ys, ks, params=None, outs=None, stream=None):
    """Algorithm 2 on many independent instances in one persistent launch.

    As: list of Expander; ys: list of CUDA float32 [m_i]; ks: list of int; params: None, a
    dict applied to all, or a list of dicts.  Returns (list of x_hat, list of stats dicts)."""
    return BatchPlan(As, ys, ks, params, outs).run(stream)


# ---------------------------------------------------------------------------
# Learned column scorer (an addition to the paper's method; see include/rl0.h)
# ---------------------------------------------------------------------------
def candidate_features(A, y, k, round_index, xhat, rhat, cap=None, stream=None, **params):
    """Features of every learned-scorer candidate of one round from an injected state.

    Returns (features [c, 16] float32, meta [c, 4] int32 (column, slot, analytic pass,
    l1 test), omega [c] float32), all CUDA tensors."""
    p = make_params(**params)
    if cap is None:
        cap = 4 * A.n
    feat = torch.empty((cap, NFEAT), dtype=torch.float32, device="cuda")
    meta = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    omega = torch.empty(cap, dtype=torch.float32, device="cuda")
    cnt = C.c_int()
    _check(_lib().rl0_candidate_features(A.handle, _dev(y, torch.float32, A.m, "y"), int(k), C.byref(p),
                                         int(round_index), _dev(xhat, torch.float32, A.n, "x_hat"),
                                         _dev(rhat, torch.float32, A.m, "r_hat"), C.c_void_p(feat.data_ptr()),
                                         C.c_void_p(meta.data_ptr()), C.c_void_p(omega.data_ptr()), int(cap),
                                         C.byref(cnt), _stream(stream)), "rl0_candidate_features")
    c = min(cnt.value, cap)
    return feat[:c], meta[:c], omega[:c]


def scorer_log(A, y, k, x_true, max_rounds=40, tol_sigma=4.0, cap=None, stream=None, **params):
    """Labelled candidates of an analytic decode of (A, y), for training the scorer
    (rl0_scorer_log).  x_true: CUDA float32 [n].  Returns (features [N, 16], labels [N],
    rounds run), CUDA tensors."""
    p = make_params(**params)
    if cap is None:
        cap = 8 * A.n
    xt = _dev(x_true, torch.float32, A.n, "x_true")
    yd = _dev(y, torch.float32, A.m, "y")
    while True:
        feat = torch.empty((max(cap, 1), NFEAT), dtype=torch.float32, device="cuda")
        lab = torch.empty(max(cap, 1), dtype=torch.float32, device="cuda")
        cnt, rounds = C.c_int64(), C.c_int32()
        _check(_lib().rl0_scorer_log(A.handle, yd, int(k), C.byref(p), xt, float(tol_sigma), int(max_rounds),
                                     C.c_void_p(feat.data_ptr()), C.c_void_p(lab.data_ptr()), int(cap),
                                     C.byref(cnt), C.byref(rounds), _stream(stream)), "rl0_scorer_log")
        if cnt.value <= cap:
            return feat[:cnt.value], lab[:cnt.value], rounds.value
        cap = cnt.value                        # the log is deterministic: run again with room for all


def mlp_init(seed=0, stream=None):
    w = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    _check(_lib().rl0_mlp_init(int(seed), C.c_void_p(w.data_ptr()), _stream(stream)), "rl0_mlp_init")
    return w


def mlp_grad(w, feat, label, stream=None):
    """(mean BCE loss, gradient) of the FP32 parameters on rows feat [N, 16], labels [N]."""
    N = feat.shape[0]
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = C.c_double()
    _check(_lib().rl0_mlp_grad(_dev(w, torch.float32, MLP_PARAMS, "w"), _dev(feat, torch.float32, N * NFEAT, "feat"),
                               _dev(label, torch.float32, N, "label"), N, C.c_void_p(g.data_ptr()), C.byref(loss),
                               _stream(stream)), "rl0_mlp_grad")
    return loss.value, g


def mlp_train(w, feat, label, epochs=5, batch=4096, lr=3e-3, stream=None):
    """Adam on minibatches of consecutive rows (shuffle beforehand).  Trains w in place;
    returns (BF16 parameters as a CUDA int16 tensor of bit patterns, final loss)."""
    N = feat.shape[0]
    wb = torch.empty(MLP_PARAMS, dtype=torch.int16, device="cuda")
    loss = C.c_double()
    _check(_lib().rl0_mlp_train(_dev(w, torch.float32, MLP_PARAMS, "w"), _dev(feat, torch.float32, N * NFEAT, "feat"),
                                _dev(label, torch.float32, N, "label"), N, int(epochs), int(batch), float(lr),
                                C.c_void_p(wb.data_ptr()), C.byref(loss), _stream(stream)), "rl0_mlp_train")
    return wb, loss.value


def mlp_export(w, stream=None):
    wb = torch.empty(MLP_PARAMS, dtype=torch.int16, device="cuda")
    _check(_lib().rl0_mlp_export(_dev(w, torch.float32, MLP_PARAMS, "w"), C.c_void_p(wb.data_ptr()),
                                 _stream(stream)), "rl0_mlp_export")
    return wb


def mlp_forward(wb, feat, stream=None):
    N = feat.shape[0]
    out = torch.empty(N, dtype=torch.float32, device="cuda")
    _check(_lib().rl0_mlp_forward(C.c_void_p(wb.data_ptr()), _dev(feat, torch.float32, N * NFEAT, "feat"), N,
                                  C.c_void_p(out.data_ptr()), _stream(stream)), "rl0_mlp_forward")
    return out
