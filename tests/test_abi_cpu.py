"""The C-ABI library builds, loads and exports every symbol its header declares; host-side
argument checks work without a GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ebic.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1807_09932_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ebic_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("ebic_load_matrix", "ebic_free_matrix", "ebic_eval_population", "ebic_fitness",
                 "ebic_matrix_info", "ebic_matrix_ranks", "ebic_matrix_status",
                 "ebic_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header(lib):
    from paper_1807_09932_gb300 import ebic
    for n in declared_functions():
        if n in ("ebic_version",):
            continue
        assert hasattr(ebic, n), n


def test_version(lib):
    lib.ebic_version.restype = ctypes.c_int
    assert lib.ebic_version() >> 16 == 1


def _last_error(lib):
    lib.ebic_last_error.restype = ctypes.c_char_p
    return lib.ebic_last_error().decode()


def test_load_rejects_bad_arguments_before_touching_cuda(lib):
    P = ctypes.c_void_p
    f = lib.ebic_load_matrix
    f.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                  ctypes.c_float, P, ctypes.POINTER(P)]
    x = np.zeros((4, 3), np.float32)
    h = P()
    xp = x.ctypes.data
    assert f(None, 4, 3, 3, 1, 0.0, None, ctypes.byref(h)) == -1
    assert f(xp, 0, 3, 3, 1, 0.0, None, ctypes.byref(h)) == -1          # rows < 1
    assert f(xp, 2 ** 31, 3, 3, 1, 0.0, None, ctypes.byref(h)) == -1    # rows > 2^31-1
    assert f(xp, 4, 0, 3, 1, 0.0, None, ctypes.byref(h)) == -1          # cols < 1
    assert f(xp, 4, 833, 833, 1, 0.0, None, ctypes.byref(h)) == -5     # beyond the build limit
    assert f(xp, 4, 3, 2, 1, 0.0, None, ctypes.byref(h)) == -1          # ld < cols
    assert f(xp, 4, 3, 3, 8, 0.0, None, ctypes.byref(h)) == -1          # unknown flag
    assert f(xp, 4, 3, 3, 0, float("nan"), None, ctypes.byref(h)) == -1  # NaN fill
    assert "fill_value" in _last_error(lib)
    assert f(xp, 4, 3, 3, 1, 0.0, None, None) == -1


def test_calls_reject_null_matrix(lib):
    P = ctypes.c_void_p
    lib.ebic_eval_population.argtypes = [P, P, P, ctypes.c_uint32, ctypes.c_uint32, P, P, P]
    assert lib.ebic_eval_population(None, None, None, 1, 0, None, None, None) == -1
    lib.ebic_matrix_info.argtypes = [P, P, P, P, P]
    assert lib.ebic_matrix_info(None, None, None, None, None) == -1
    lib.ebic_free_matrix.argtypes = [P]
    assert lib.ebic_free_matrix(None) == 0


def test_copy_rejects_null_buffers_and_skips_empty_copies(lib):
    P = ctypes.c_void_p
    f = lib.ebic_copy_async
    f.argtypes = [P, P, ctypes.c_size_t, P]
    buf = np.zeros(4, np.uint8)
    assert f(None, buf.ctypes.data, 4, None) == -1
    assert f(buf.ctypes.data, None, 4, None) == -1
    assert "NULL" in _last_error(lib)
    assert f(None, None, 0, None) == 0  # nothing to copy: no runtime call


def test_no_device_is_reported_not_crashed(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    P = ctypes.c_void_p
    f = lib.ebic_load_matrix
    f.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                  ctypes.c_float, P, ctypes.POINTER(P)]
    x = np.zeros((4, 3), np.float32)
    h = P()
    rc = f(x.ctypes.data, 4, 3, 3, 1, 0.0, None, ctypes.byref(h))
    assert rc in (-6, -3), rc
    assert not h.value


def test_c_marshalling_matches_ctypes_marshalling(lib):
    """The C module that converts the per-generation calls' arguments gives the same statuses,
    messages and argument errors as the ctypes path (both call the same library functions)."""
    import torch
    from paper_1807_09932_gb300 import ebic
    fast = ebic._fast
    if fast is None:
        pytest.skip("the interpreter's headers are not installed: the binding uses ctypes only")
    cols = np.zeros(6, np.uint16)
    offs = np.array([0, 3, 6], np.uint32)
    cnt = torch.zeros(2, dtype=torch.int32)
    fit = torch.zeros(2, dtype=torch.int64)
    calls = [
        ("ebic_eval_fitness", lambda: fast.eval_fitness(None, cols, offs, 2, 0, None, None, None, 0,
                                                        cnt, None, fit, None, 0),
         lambda: ebic._lib_eval_fitness(None, cols.ctypes.data, offs.ctypes.data, 2, 0, None, None,
                                        None, 0, cnt.data_ptr(), None, fit.data_ptr(), None, None)),
        ("ebic_eval_population", lambda: fast.eval_population(ctypes.c_void_p(), cols, offs, 2, 0,
                                                              cnt, None, 0),
         lambda: ebic._lib_eval(None, cols.ctypes.data, offs.ctypes.data, 2, 0, cnt.data_ptr(),
                                None, None)),
        ("ebic_fitness", lambda: fast.fitness(0, cols, offs, 2, cnt, None, None, None, None, 0, 0,
                                              fit, None, None),
         lambda: ebic._lib_fitness(None, cols.ctypes.data, offs.ctypes.data, 2, cnt.data_ptr(),
                                   None, None, None, None, 0, 0, fit.data_ptr(), None, None)),
    ]
    for name, via_c, via_ctypes in calls:
        rc_c = via_c()
        msg_c = ebic.ebic_last_error()
        rc_t = via_ctypes()
        msg_t = ebic.ebic_last_error()
        assert rc_c == rc_t == ebic.EBIC_ERR_INVALID_ARG, name
        assert msg_c == msg_t and "NULL" in msg_c, (name, msg_c, msg_t)
    # argument errors are raised before the library is called
    with pytest.raises(ValueError):
        fast.eval_fitness(None, np.zeros((3, 4), np.uint16)[:, 1], offs, 2, 0, None, None, None, 0,
                          cnt, None, fit, None, 0)
    with pytest.raises(ValueError):
        fast.eval_fitness(None, cols, offs, 2, 0, None, None, None, 0,
                          torch.zeros(4, dtype=torch.int32)[::2], None, fit, None, 0)
    with pytest.raises(TypeError):
        fast.eval_fitness(None, "cols", offs, 2, 0, None, None, None, 0, cnt, None, fit, None, 0)
    with pytest.raises(TypeError):
        fast.eval_fitness(None, cols, offs, 2)
    with pytest.raises(OverflowError):
        fast.eval_fitness(None, cols, offs, 1 << 32, 0, None, None, None, 0, cnt, None, fit,
                          None, 0)
    # the module links to the library the binding loaded: one copy of its state
    maps = {l.split()[-1] for l in open("/proc/self/maps") if "libebic_gb300" in l}
    assert len(maps) == 1, maps
