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


def test_product_package_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_1704_09012_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or f == "__init__.py" and \
                    "import oracle" not in src, f
                assert "import oracle" not in src and "from oracle" not in src, f
