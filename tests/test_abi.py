"""Host-side checks of the C ABI that need no GPU: the library builds, loads, exports
every function include/rl0.h declares, and rejects bad arguments before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "rl0.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rl0_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_09012_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_library_exports_every_declared_function(lib):
    declared = _header_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    import paper_1704_09012_gb300 as rl0
    assert sorted(rl0.EXPORTS) == _header_functions()


def test_strerror_and_argument_checks_without_gpu(lib):
    lib.rl0_strerror.restype = C.c_char_p
    assert lib.rl0_strerror(0) == b"success"
    assert b"invalid" in lib.rl0_strerror(-1)
    vp = C.c_void_p
    lib.rl0_decode.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp]
    assert lib.rl0_decode(None, None, 10, None, None, None, None) == -1
    lib.rl0_make_expander.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_uint64, vp, C.POINTER(vp)]
    h = vp()
    assert lib.rl0_make_expander(0, 10, 3, 0, None, C.byref(h)) == -1      # n < 1
    assert lib.rl0_make_expander(10, 2, 3, 0, None, C.byref(h)) == -1      # d > m
    assert lib.rl0_make_expander(10, 64, 33, 0, None, C.byref(h)) == -1    # d > 32
    lib.rl0_expander_shape.argtypes = [vp, vp, vp, vp]
    assert lib.rl0_expander_shape(None, None, None, None) == -1
    lib.rl0_decode_log.argtypes = [vp, vp, C.c_int]
    assert lib.rl0_decode_log(None, None, 0) == -1


def test_learned_and_tool_entry_points_reject_bad_arguments_without_gpu(lib):
    """Each of these returns before its first CUDA call; the dummy non-null pointers
    are never dereferenced."""
    import paper_1704_09012_gb300 as rl0
    vp, i64 = C.c_void_p, C.c_int64
    dummy = vp(256)
    lib.rl0_mlp_init.argtypes = [C.c_uint64, vp, vp]
    assert lib.rl0_mlp_init(0, None, None) == -1
    lib.rl0_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    assert lib.rl0_mlp_grad(dummy, dummy, dummy, 0, dummy, None, None) == -1           # N < 1
    lib.rl0_mlp_train.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, C.c_float, vp, vp, vp]
    assert lib.rl0_mlp_train(dummy, dummy, dummy, 10, 0, 4, 1e-3, None, None, None) == -1   # epochs < 1
    assert lib.rl0_mlp_train(dummy, dummy, dummy, 10, 1, 4, 0.0, None, None, None) == -1    # lr <= 0
    lib.rl0_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    assert lib.rl0_mlp_forward(dummy, dummy, -1, dummy, None) == -1                    # N < 0
    lib.rl0_mlp_export.argtypes = [vp, vp, vp]
    assert lib.rl0_mlp_export(None, dummy, None) == -1
    lib.rl0_round_step.argtypes = [vp, vp, i64, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp]
    assert lib.rl0_round_step(None, dummy, 10, None, 0, dummy, dummy, dummy, dummy, None, None, None) == -1
    lib.rl0_expander_set_wait_polls.argtypes = [vp, i64]
    assert lib.rl0_expander_set_wait_polls(None, 0) == -1
    lib.rl0_decode_static.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    assert lib.rl0_decode_static(None, dummy, 10, None, dummy, None, None) == -1
    # rl0_scorer_log: the analytic rule only, a positive tolerance, 2 <= max_rounds
    lib.rl0_scorer_log.argtypes = [vp, vp, i64, C.POINTER(rl0.Params), vp, C.c_float, C.c_int, vp, vp, i64,
                                   C.POINTER(i64), C.POINTER(C.c_int32), vp]
    cnt, rounds = i64(), C.c_int32()
    p = rl0.make_params(sigma_n=0.01)
    args = lambda prm, tol, mr: lib.rl0_scorer_log(dummy, dummy, 10, C.byref(prm), dummy, tol, mr, dummy, dummy,
                                                    100, C.byref(cnt), C.byref(rounds), None)
    assert args(p, 0.0, 40) == -1                                                     # tol_sigma <= 0
    assert args(p, 4.0, 1) == -1                                                      # max_rounds < 2
    assert args(rl0.make_params(sigma_n=0.01, scorer=1), 4.0, 40) == -5               # learned: unsupported
    assert args(rl0.make_params(sigma_n=0.0), 4.0, 40) == -1                          # sigma_n = 0
    assert lib.rl0_scorer_log(None, dummy, 10, C.byref(p), dummy, 4.0, 40, dummy, dummy, 100, C.byref(cnt),
                              C.byref(rounds), None) == -1


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1704_09012_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or f == "__init__.py" and \
                    "import oracle" not in src, f
                assert "import oracle" not in src and "from oracle" not in src, f
