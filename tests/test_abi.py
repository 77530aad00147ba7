"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every function ``include/ttsg.h`` declares, and the binding's ctypes
prototypes name exactly those functions.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(tt_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built_lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for required in ("tt_matvec", "tt_sketch", "tt_round_rand", "tt_sgmres_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_prototypes_match_header(built_lib):
    from paper_2409_09471_gb300 import _abi
    src = open(_abi.__file__).read()
    bound = set(re.findall(r'"(tt_\w+)"\s*:', src))
    assert bound == declared_functions()


def test_version_and_error_strings(built_lib):
    built_lib.tt_version.restype = ctypes.c_char_p
    built_lib.tt_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in built_lib.tt_version()
    assert built_lib.tt_last_error() == b""


def test_argument_errors_are_caught_on_the_host(built_lib):
    # a null descriptor is rejected before any CUDA call, so this runs without a GPU
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    rc = lib.tt_dot(0, None, None, None, None, 0, None)
    assert rc == 1 and b"null descriptor" in lib.tt_last_error()
    rc = lib.tt_matvec(7, None, None, None, None, 0, None)
    assert rc == 1 and b"unknown mode" in lib.tt_last_error()


def test_workspace_queries_run_without_a_gpu(built_lib):
    # every *_workspace entry point is a dry run on the host (no CUDA call):
    # descriptors with placeholder device pointers must give a positive size
    from paper_2409_09471_gb300 import _abi
    lib = _abi.lib
    d, ns = 4, [7, 5, 8, 6]

    def desc(ranks):
        n = (ctypes.c_int64 * d)(*ns)
        r = (ctypes.c_int64 * (d + 1))(*ranks)
        p = (ctypes.c_void_p * d)(*([0x1000] * d))
        return _abi.TTVec(d, n, r, p), (n, r, p)

    x, kx = desc([1, 4, 9, 3, 1])
    y, ky = desc([1, 2, 6, 5, 1])
    for mode in (0, 1, 2):
        assert lib.tt_dot_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_dot_grad_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_local_dots_workspace(mode, ctypes.byref(x), ctypes.byref(y)) > 0
        assert lib.tt_sketch_workspace(mode, ctypes.byref(x), 40) > 0
        arr = (_abi.TTVec * 2)(x, y)
        assert lib.tt_round_rand_workspace(mode, 2, arr, 8, 4) > 0
