"""Python binding of the EBIC GB300 C ABI (``include/ebic.h``): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels. This module converts arguments
(numpy arrays as host buffers, torch tensors as device buffers, torch streams as cudaStream_t)
and raises ``EbicError`` on a non-zero status. There is no fallback of any kind: if the compiled
library is missing, importing this module raises.

The functions keep the C names (``ebic_load_matrix``, ``ebic_eval_population``, ...). ``Matrix``,
``eval_population`` and ``fitness`` are conveniences over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libebic_gb300.so")

EBIC_OK = 0
EBIC_ERR_INVALID_ARG = -1
EBIC_ERR_OOM = -2
EBIC_ERR_CUDA = -3
EBIC_ERR_DEVICE_TIMEOUT = -4
EBIC_ERR_UNSUPPORTED = -5
EBIC_ERR_NO_DEVICE = -6
EBIC_EXCLUDE_MISSING = 0x1
EBIC_NEGATIVE_TRENDS = 0x1
EBIC_EVAL_DIRECT = 0x2
EBIC_RUN_ON_DEVICE = 0x2  # ebic_params.flags
EBIC_MAX_COLS = 832
EBIC_MAX_CANDIDATE_LEN = 64

if not os.path.exists(LIB_PATH):
    raise ImportError(f"the EBIC CUDA library is not built ({LIB_PATH} is missing); "
                      "run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)


def _load_fast():
    """The C marshalling module for the per-generation calls, when it was built (it links to the
    library loaded above; the calls and their results are the same either way)."""
    import importlib.util
    import sysconfig
    path = os.path.join(_PKG, "lib", "_ebic_fast" + (sysconfig.get_config_var("EXT_SUFFIX") or ".so"))
    if not os.path.exists(path) or os.environ.get("EBIC_CTYPES_ONLY"):
        return None
    spec = importlib.util.spec_from_file_location("_ebic_fast", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


_fast = _load_fast()
_P = ctypes.c_void_p
_I32, _I64, _U32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_lib_load = _sig("ebic_load_matrix", [_P, _I64, _I32, _I64, _U32, ctypes.c_float, _P,
                                      ctypes.POINTER(_P)])
_lib_free = _sig("ebic_free_matrix", [_P])
_lib_info = _sig("ebic_matrix_info", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                                      ctypes.POINTER(_I64), ctypes.POINTER(_I32)])
_lib_ranks = _sig("ebic_matrix_ranks", [_P, _P, _P])
_lib_eval = _sig("ebic_eval_population", [_P, _P, _P, _U32, _U32, _P, _P, _P])
_lib_eval_noalloc = _sig("ebic_eval_population_noalloc", [_P, _P, _P, _U32, _U32, _P, _P, _P])
_lib_fitness = _sig("ebic_fitness", [_P, _P, _P, _U32, _P, _P, _P, _P, _P, _U32, _U32, _P, _P,
                                     _P])
_lib_eval_fitness = _sig("ebic_eval_fitness", [_P, _P, _P, _U32, _U32, _P, _P, _P, _U32, _P,
                                               _P, _P, _P, _P])
_lib_load_shard = _sig("ebic_load_matrix_shard", [_P, _I64, _I32, _I64, _I64, _I64, _U32,
                                                  ctypes.c_float, _P, ctypes.POINTER(_P)])
_lib_shard = _sig("ebic_matrix_shard", [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                        ctypes.POINTER(_I64)])
_lib_eval_partials = _sig("ebic_eval_partials", [_P, _P, _P, _U32, _U32, _P, _P, _P, _U32, _P,
                                                 _P, _P, _P, _P])
_lib_fitness_reduced = _sig("ebic_fitness_reduced", [_P, _P, _P, _U32, _P, _P, _P, _P, _P, _U32,
                                                     _U32, _P, _P])
_lib_status = _sig("ebic_matrix_status", [_P, _P])
_lib_set_tile = _sig("ebic_matrix_set_tile", [_P, _I32])
_lib_get_tile = _sig("ebic_matrix_get_tile", [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)])
_lib_set_chunk = _sig("ebic_matrix_set_chunk_cols", [_P, _I32])
_lib_build_pairs = _sig("ebic_matrix_build_pairs", [_P, ctypes.c_uint64, _P,
                                                    ctypes.POINTER(ctypes.c_uint64)])
_lib_drop_pairs = _sig("ebic_matrix_drop_pairs", [_P])
_lib_last_error = _sig("ebic_last_error", [], ctypes.c_char_p)
_lib_launch_count = _sig("ebic_launch_count", [], ctypes.c_int64)
_lib_copy_async = _sig("ebic_copy_async", [_P, _P, ctypes.c_size_t, _P])
_lib_timing_enable = _sig("ebic_timing_enable", [ctypes.c_int])
_lib_timing_read = _sig("ebic_timing_read", [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(_I64)])
_lib_version = _sig("ebic_version", [])
_lib_selftest = _sig("ebic_selftest_wait_timeout", [ctypes.c_uint64, _P])


class EbicParams(ctypes.Structure):
    _fields_ = [("population", ctypes.c_uint32), ("generations", ctypes.c_uint32),
                ("archive_size", ctypes.c_uint32), ("elite", ctypes.c_uint32),
                ("tournament", ctypes.c_uint32), ("min_len", ctypes.c_uint32),
                ("max_init_len", ctypes.c_uint32), ("max_len", ctypes.c_uint32),
                ("p_crossover", ctypes.c_float), ("p_mutation", ctypes.c_float),
                ("overlap_threshold", ctypes.c_float), ("tabu_retries", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class EbicResult(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("cols", ctypes.POINTER(ctypes.c_uint16)),
                ("offsets", ctypes.POINTER(ctypes.c_uint32)),
                ("counts", ctypes.POINTER(ctypes.c_uint32)),
                ("quality", ctypes.POINTER(ctypes.c_uint64)),
                ("bitmaps", ctypes.POINTER(ctypes.c_uint32)), ("words", ctypes.c_int64),
                ("generations_run", ctypes.c_uint32), ("candidates_evaluated", ctypes.c_uint64)]


class EbicTextMatrix(ctypes.Structure):
    _fields_ = [("values", ctypes.POINTER(ctypes.c_float)), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int32), ("row_names", ctypes.POINTER(ctypes.c_char_p)),
                ("col_names", ctypes.POINTER(ctypes.c_char_p))]


EVALUATE_FN = ctypes.CFUNCTYPE(ctypes.c_int, _P, ctypes.POINTER(ctypes.c_uint16),
                               ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                               ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint32))
PAIR_FN = ctypes.CFUNCTYPE(ctypes.c_int, _P, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                           ctypes.POINTER(ctypes.c_uint32))
SET_ARCHIVE_FN = ctypes.CFUNCTYPE(ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.c_uint32)


class EbicEvaluator(ctypes.Structure):
    _fields_ = [("user", _P), ("evaluate", EVALUATE_FN), ("pair_overlaps", PAIR_FN),
                ("set_archive", SET_ARCHIVE_FN)]


class EbicEvalRequest(ctypes.Structure):
    _fields_ = [("m", _P), ("cols", _P), ("offsets", _P), ("n_cand", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("counts", _P), ("bitmaps", _P),
                ("arch_cols", _P), ("arch_offsets", _P), ("arch_bitmaps", _P),
                ("n_arch", ctypes.c_uint32), ("fitness", _P)]


_lib_eval_batch = _sig("ebic_eval_batch", [ctypes.POINTER(EbicEvalRequest), _U32, _P])
_lib_batch_create = _sig("ebic_batch_create", [_U32, ctypes.POINTER(_P)])
_lib_batch_run = _sig("ebic_batch_run", [_P, ctypes.POINTER(EbicEvalRequest), _U32, _P])
_lib_batch_status = _sig("ebic_batch_status", [_P, ctypes.POINTER(ctypes.c_uint32), _U32, _P])
_lib_batch_free = _sig("ebic_batch_free", [_P])
_lib_params_default = _sig("ebic_params_default", [ctypes.POINTER(EbicParams)])
_lib_run = _sig("ebic_run", [_P, ctypes.POINTER(EbicParams), _P,
                             ctypes.POINTER(ctypes.POINTER(EbicResult))])
_lib_run_custom = _sig("ebic_run_custom", [_I64, _I32, ctypes.POINTER(EbicParams),
                                           ctypes.POINTER(EbicEvaluator),
                                           ctypes.POINTER(ctypes.POINTER(EbicResult))])
_lib_free_result = _sig("ebic_free_result", [ctypes.POINTER(EbicResult)])
_lib_read_text = _sig("ebic_read_matrix_text", [ctypes.c_char_p, ctypes.c_char, ctypes.c_char_p,
                                                ctypes.POINTER(ctypes.POINTER(EbicTextMatrix))])
_lib_free_text = _sig("ebic_free_text_matrix", [ctypes.POINTER(EbicTextMatrix)])
_lib_write_bic = _sig("ebic_write_biclusters", [ctypes.c_char_p, ctypes.c_char_p,
                                                ctypes.POINTER(EbicResult),
                                                ctypes.POINTER(EbicTextMatrix)])


class EbicError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _check(code, where):
    if code != EBIC_OK:
        raise EbicError(code, where)


_TENSOR = None  # torch.Tensor, once one has been seen (torch is not imported here)


def _ptr(x):
    """Raw address of a numpy array (host) or torch tensor (its device or host memory)."""
    global _TENSOR
    if x is None:
        return None
    if type(x) is _TENSOR:  # the common case first: a plain torch tensor
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if type(x).__name__ == "Tensor" and type(x).__module__ == "torch":
            _TENSOR = type(x)
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def version():
    return int(_lib_version())


# ---- thin C-named wrappers --------------------------------------------------------------------

def ebic_load_matrix(x, rows, cols, ld, flags, fill_value, stream=None):
    h = _P()
    _check(_lib_load(_ptr(x), rows, cols, ld, flags, fill_value, _stream(stream),
                     ctypes.byref(h)), "ebic_load_matrix")
    return h


def ebic_load_matrix_shard(x, rows, cols, ld, row_offset, total_rows, flags, fill_value,
                           stream=None):
    h = _P()
    _check(_lib_load_shard(_ptr(x), rows, cols, ld, row_offset, total_rows, flags, fill_value,
                           _stream(stream), ctypes.byref(h)), "ebic_load_matrix_shard")
    return h


def ebic_matrix_shard(h):
    r, t, w = _I64(), _I64(), _I64()
    _check(_lib_shard(h, ctypes.byref(r), ctypes.byref(t), ctypes.byref(w)), "ebic_matrix_shard")
    return r.value, t.value, w.value


def ebic_eval_partials(h, cols, offsets, n_cand, flags, arch_cols, arch_offsets, arch_bitmaps,
                       n_arch, counts, overlaps, arch_counts, bitmaps, stream=None):
    return _lib_eval_partials(h, _ptr(cols), _ptr(offsets), n_cand, flags, _ptr(arch_cols),
                              _ptr(arch_offsets), _ptr(arch_bitmaps), n_arch, _ptr(counts),
                              _ptr(overlaps), _ptr(arch_counts), _ptr(bitmaps), _stream(stream))


def ebic_fitness_reduced(h, cols, offsets, n_cand, counts, overlaps, arch_cols, arch_offsets,
                         arch_counts, n_arch, flags, fitness, stream=None):
    return _lib_fitness_reduced(h, _ptr(cols), _ptr(offsets), n_cand, _ptr(counts),
                                _ptr(overlaps), _ptr(arch_cols), _ptr(arch_offsets),
                                _ptr(arch_counts), n_arch, flags, _ptr(fitness),
                                _stream(stream))


def ebic_free_matrix(h):
    _check(_lib_free(h), "ebic_free_matrix")


def ebic_matrix_info(h):
    r, c, w, b = _I64(), _I32(), _I64(), _I32()
    _check(_lib_info(h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(w), ctypes.byref(b)),
           "ebic_matrix_info")
    return r.value, c.value, w.value, b.value


def ebic_matrix_ranks(h, out, stream=None):
    _check(_lib_ranks(h, _ptr(out), _stream(stream)), "ebic_matrix_ranks")


def ebic_eval_population(h, cols, offsets, n_cand, flags, counts, bitmaps, stream=None):
    if _fast is not None:
        return _fast.eval_population(h, cols, offsets, n_cand, flags, counts, bitmaps,
                                     stream if stream is not None else _stream(None))
    return _lib_eval(h, _ptr(cols), _ptr(offsets), n_cand, flags, _ptr(counts), _ptr(bitmaps),
                     _stream(stream))


def ebic_eval_population_noalloc(h, cols, offsets, n_cand, flags, counts, bitmaps, stream=None):
    """Allocation-free evaluation (outputs must be device buffers); see include/ebic.h."""
    return _lib_eval_noalloc(h, _ptr(cols), _ptr(offsets), n_cand, flags, _ptr(counts),
                             _ptr(bitmaps), _stream(stream))


def ebic_fitness(h, cols, offsets, n_cand, counts, bitmaps, arch_cols, arch_offsets,
                 arch_bitmaps, n_arch, flags, fitness, overlaps, stream=None):
    if _fast is not None:
        return _fast.fitness(h, cols, offsets, n_cand, counts, bitmaps, arch_cols, arch_offsets,
                             arch_bitmaps, n_arch, flags, fitness, overlaps,
                             stream if stream is not None else _stream(None))
    return _lib_fitness(h, _ptr(cols), _ptr(offsets), n_cand, _ptr(counts), _ptr(bitmaps),
                        _ptr(arch_cols), _ptr(arch_offsets), _ptr(arch_bitmaps), n_arch, flags,
                        _ptr(fitness), _ptr(overlaps), _stream(stream))


def ebic_eval_fitness(h, cols, offsets, n_cand, flags, arch_cols, arch_offsets, arch_bitmaps,
                      n_arch, counts, bitmaps, fitness, overlaps, stream=None):
    if _fast is not None:
        return _fast.eval_fitness(h, cols, offsets, n_cand, flags, arch_cols, arch_offsets,
                                  arch_bitmaps, n_arch, counts, bitmaps, fitness, overlaps,
                                  stream if stream is not None else _stream(None))
    return _lib_eval_fitness(h, _ptr(cols), _ptr(offsets), n_cand, flags, _ptr(arch_cols),
                             _ptr(arch_offsets), _ptr(arch_bitmaps), n_arch, _ptr(counts),
                             _ptr(bitmaps), _ptr(fitness), _ptr(overlaps), _stream(stream))


def ebic_matrix_status(h, stream=None):
    return _lib_status(h, _stream(stream))


def ebic_matrix_set_tile(h, tile_slabs):
    _check(_lib_set_tile(h, tile_slabs), "ebic_matrix_set_tile")


def ebic_matrix_set_chunk_cols(h, chunk_cols):
    _check(_lib_set_chunk(h, chunk_cols), "ebic_matrix_set_chunk_cols")


def ebic_matrix_build_pairs(h, max_bytes, stream=None):
    """Build the matrix's pair table if it fits max_bytes; returns its size in bytes."""
    n = ctypes.c_uint64()
    _check(_lib_build_pairs(h, max_bytes, _stream(stream), ctypes.byref(n)),
           "ebic_matrix_build_pairs")
    return n.value


def ebic_matrix_drop_pairs(h):
    _check(_lib_drop_pairs(h), "ebic_matrix_drop_pairs")


def ebic_matrix_get_tile(h):
    t, r = _I32(), _I32()
    _check(_lib_get_tile(h, ctypes.byref(t), ctypes.byref(r)), "ebic_matrix_get_tile")
    return t.value, r.value


EBIC_TIMING_RANK_TRANSFORM, EBIC_TIMING_PREPARE, EBIC_TIMING_EVALUATE = 0, 1, 2
EBIC_TIMING_OVERLAP, EBIC_TIMING_FITNESS, EBIC_TIMING_PAIR_EVALUATE = 3, 4, 5
EBIC_TIMING_KINDS = 6


def ebic_launch_count():
    return int(_lib_launch_count())


def ebic_copy_async(dst, src, nbytes, stream=None):
    """A stream-ordered copy of nbytes bytes between any two buffers (addresses, arrays or
    tensors); see include/ebic.h."""
    return _lib_copy_async(_ptr(dst), _ptr(src), nbytes, _stream(stream))


def ebic_timing_enable(on):
    _check(_lib_timing_enable(1 if on else 0), "ebic_timing_enable")


def ebic_timing_read(kind):
    ms, n = ctypes.c_double(), _I64()
    _check(_lib_timing_read(kind, ctypes.byref(ms), ctypes.byref(n)), "ebic_timing_read")
    return ms.value, n.value


def make_requests(items):
    """items: (handle, cols, offsets, n_cand, flags, counts, bitmaps) tuples, optionally followed
    by (arch_cols, arch_offsets, arch_bitmaps, n_arch, fitness) -> ctypes array."""
    arr = (EbicEvalRequest * max(len(items), 1))()
    for i, it in enumerate(items):
        h, c, o, n, f, cnt, bm = it[:7]
        ac, ao, ab, k, fit = it[7:] if len(it) > 7 else (None, None, None, 0, None)
        arr[i] = EbicEvalRequest(h, _ptr(c), _ptr(o), n, f, _ptr(cnt), _ptr(bm), _ptr(ac),
                                 _ptr(ao), _ptr(ab), k, _ptr(fit))
    return arr


def ebic_eval_batch(reqs, n_req, stream=None):
    return _lib_eval_batch(reqs, n_req, _stream(stream))


def ebic_batch_create(max_requests):
    b = _P()
    _check(_lib_batch_create(max_requests, ctypes.byref(b)), "ebic_batch_create")
    return b


def ebic_batch_run(b, reqs, n_req, stream=None):
    return _lib_batch_run(b, reqs, n_req, _stream(stream))


def ebic_batch_status(b, n, stream=None):
    out = (ctypes.c_uint32 * max(n, 1))()
    rc = _lib_batch_status(b, out, n, _stream(stream))
    return rc, list(out)[:n]


def ebic_batch_free(b):
    _check(_lib_batch_free(b), "ebic_batch_free")


def ebic_params_default(**overrides):
    p = EbicParams()
    _check(_lib_params_default(ctypes.byref(p)), "ebic_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _take_result(rp):
    r = rp.contents
    n = r.n
    offs = np.ctypeslib.as_array(r.offsets, (n + 1,)).copy()
    out = {"offsets": offs,
           "cols": np.ctypeslib.as_array(r.cols, (max(int(offs[-1]), 1),))[: int(offs[-1])].copy(),
           "counts": np.ctypeslib.as_array(r.counts, (max(n, 1),))[:n].copy(),
           "quality": np.ctypeslib.as_array(r.quality, (max(n, 1),))[:n].copy(),
           "generations_run": r.generations_run,
           "candidates_evaluated": r.candidates_evaluated,
           "bitmaps": None}
    if bool(r.bitmaps):
        out["bitmaps"] = np.ctypeslib.as_array(r.bitmaps, (n * r.words + 1,))[: n * r.words] \
            .reshape(n, r.words).copy()
    _lib_free_result(rp)
    out["members"] = [out["cols"][offs[i]:offs[i + 1]].tolist() for i in range(n)]
    return out


def ebic_run(h, params, stream=None):
    """Run the EBIC generation loop on a loaded matrix; returns the archive as a dict."""
    rp = ctypes.POINTER(EbicResult)()
    _check(_lib_run(h, ctypes.byref(params), _stream(stream), ctypes.byref(rp)), "ebic_run")
    return _take_result(rp)


def ebic_run_custom(rows, cols, params, evaluator):
    """The same loop over an EbicEvaluator of Python callbacks (host buffers)."""
    rp = ctypes.POINTER(EbicResult)()
    _check(_lib_run_custom(rows, cols, ctypes.byref(params), ctypes.byref(evaluator),
                           ctypes.byref(rp)), "ebic_run_custom")
    return _take_result(rp)


def ebic_free_result(rp):
    _check(_lib_free_result(rp), "ebic_free_result")


def ebic_selftest_wait_timeout(timeout_ns, stream=None):
    return _lib_selftest(timeout_ns, _stream(stream))


def ebic_last_error():
    return _lib_last_error().decode(errors="replace")


# ---- conveniences -------------------------------------------------------------------------------

def words(rows):
    return (rows + 31) // 32


class Matrix:
    """A loaded matrix: its device-resident rank matrix stays on the GPU until ``close()``."""

    def __init__(self, X, *, exclude_missing=True, fill_value=0.0, stream=None, row_offset=None,
                 total_rows=None):
        """With row_offset / total_rows: X holds rows [row_offset, row_offset + len(X)) of a
        matrix of total_rows rows (a row shard, ebic_load_matrix_shard)."""
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float32)
        rows, cols = X.shape
        flags = EBIC_EXCLUDE_MISSING if exclude_missing else 0
        if row_offset is None and total_rows is None:
            self.handle = ebic_load_matrix(X, rows, cols, cols, flags, float(fill_value), stream)
        else:
            self.handle = ebic_load_matrix_shard(
                X, rows, cols, cols, int(row_offset or 0),
                int(rows if total_rows is None else total_rows), flags, float(fill_value), stream)
        self.rows, self.cols, self.words, self.rank_bits = ebic_matrix_info(self.handle)
        self.row_offset, self.total_rows, self.word_offset = ebic_matrix_shard(self.handle)
        self.exclude_missing = exclude_missing

    def close(self):
        if self.handle:
            ebic_free_matrix(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def ranks(self):
        out = np.zeros((self.rows, self.cols), dtype=np.uint16)
        ebic_matrix_ranks(self.handle, out)
        return out

    @property
    def tile(self):
        return ebic_matrix_get_tile(self.handle)

    def set_tile(self, tile_slabs):
        ebic_matrix_set_tile(self.handle, tile_slabs)

    def build_pairs(self, max_bytes=1 << 34, stream=None):
        return ebic_matrix_build_pairs(self.handle, max_bytes, stream)

    def drop_pairs(self):
        ebic_matrix_drop_pairs(self.handle)

    def set_chunk_cols(self, chunk_cols):
        ebic_matrix_set_chunk_cols(self.handle, chunk_cols)

    def status(self, stream=None):
        return ebic_matrix_status(self.handle, stream)


def eval_population(m: Matrix, cols, offsets, *, negative=False, want_bitmaps=True, counts=None,
                    bitmaps=None, stream=None, direct=False):
    """Counts and bitmaps. Host numpy inputs give host numpy outputs unless buffers are given."""
    n = len(offsets) - 1
    if counts is None:
        counts = np.zeros(n, dtype=np.uint32)
    if want_bitmaps and bitmaps is None:
        bitmaps = np.zeros((n, m.words), dtype=np.uint32)
    if not want_bitmaps:
        bitmaps = None
    flags = (EBIC_NEGATIVE_TRENDS if negative else 0) | (EBIC_EVAL_DIRECT if direct else 0)
    rc = ebic_eval_population(m.handle, cols, offsets, n, flags, counts, bitmaps, stream)
    _check(rc, "ebic_eval_population")
    return counts, bitmaps


def fitness(m: Matrix, cols, offsets, counts, bitmaps, arch_cols, arch_offsets, arch_bitmaps, *,
            fitness_out=None, overlaps=None, want_overlaps=True, stream=None):
    n = len(offsets) - 1
    k = len(arch_offsets) - 1
    if fitness_out is None:
        fitness_out = np.zeros(n, dtype=np.uint64)
    if want_overlaps and overlaps is None:
        overlaps = np.zeros((n, k), dtype=np.uint32)
    rc = ebic_fitness(m.handle, cols, offsets, n, counts, bitmaps, arch_cols, arch_offsets,
                      arch_bitmaps, k, 0, fitness_out, overlaps if want_overlaps else None,
                      stream)
    _check(rc, "ebic_fitness")
    return fitness_out, overlaps


def eval_fitness(m: Matrix, cols, offsets, arch_cols, arch_offsets, arch_bitmaps, *,
                 negative=False, direct=False, want_bitmaps=False, want_overlaps=False,
                 stream=None):
    """One generation's scoring (ebic_eval_fitness): counts, bitmaps or None, fitness, overlaps
    or None, as host numpy arrays."""
    n = len(offsets) - 1
    k = len(arch_offsets) - 1
    counts = np.zeros(n, dtype=np.uint32)
    bitmaps = np.zeros((n, m.words), dtype=np.uint32) if want_bitmaps else None
    fit = np.zeros(n, dtype=np.uint64)
    overlaps = np.zeros((n, k), dtype=np.uint32) if want_overlaps and k else None
    flags = (EBIC_NEGATIVE_TRENDS if negative else 0) | (EBIC_EVAL_DIRECT if direct else 0)
    rc = ebic_eval_fitness(m.handle, cols, offsets, n, flags, arch_cols, arch_offsets,
                           arch_bitmaps, k, counts, bitmaps, fit, overlaps, stream)
    _check(rc, "ebic_eval_fitness")
    return counts, bitmaps, fit, overlaps


def eval_partials(m: Matrix, cols, offsets, arch_cols, arch_offsets, arch_bitmaps, *,
                  negative=False, want_bitmaps=False, stream=None):
    """One row shard's share of a generation's scoring (ebic_eval_partials): counts, overlaps
    (or None without an archive), archive counts (or None) and bitmaps (or None), as host numpy
    arrays. arch_bitmaps are the members' bitmaps over the shard's rows."""
    n = len(offsets) - 1
    k = len(arch_offsets) - 1
    counts = np.zeros(n, dtype=np.uint32)
    overlaps = np.zeros((n, k), dtype=np.uint32) if k else None
    acounts = np.zeros(k, dtype=np.uint32) if k else None
    bitmaps = np.zeros((n, m.words), dtype=np.uint32) if want_bitmaps else None
    rc = ebic_eval_partials(m.handle, cols, offsets, n, EBIC_NEGATIVE_TRENDS if negative else 0,
                            arch_cols, arch_offsets, arch_bitmaps, k, counts, overlaps, acounts,
                            bitmaps, stream)
    _check(rc, "ebic_eval_partials")
    return counts, overlaps, acounts, bitmaps


def fitness_reduced(m: Matrix, cols, offsets, counts, overlaps, arch_cols, arch_offsets,
                    arch_counts, stream=None):
    """The fitness from whole-matrix sums of the shards' partials (ebic_fitness_reduced)."""
    n = len(offsets) - 1
    k = len(arch_offsets) - 1
    fit = np.zeros(n, dtype=np.uint64)
    rc = ebic_fitness_reduced(m.handle, cols, offsets, n, counts, overlaps if k else None,
                              arch_cols, arch_offsets, arch_counts if k else None, k, 0, fit,
                              stream)
    _check(rc, "ebic_fitness_reduced")
    return fit


# ---- text input and bicluster output ------------------------------------------------------------

def ebic_read_matrix_text(path, delimiter, missing, out):
    """out: a ctypes.POINTER(EbicTextMatrix) receiving the matrix (see TextMatrix)."""
    return _lib_read_text(path, delimiter, missing, ctypes.byref(out))


def ebic_free_text_matrix(m):
    return _lib_free_text(m)


def ebic_write_biclusters(path, title, result, names):
    """result: an EbicResult (by pointer or byref); names: a POINTER(EbicTextMatrix) or None."""
    return _lib_write_bic(path, title, result, names)


class TextMatrix:
    """A matrix read by ebic_read_matrix_text: values (float32 numpy [rows][cols], NaN where
    missing), row_names and col_names (lists of str, or None). Keep it open while writing results
    with its names; close() (or a with-block) frees the library's copy."""

    def __init__(self, path, delimiter=None, missing=None):
        self._p = None
        d = b"\0" if delimiter is None else str(delimiter).encode()
        if len(d) != 1:
            raise ValueError("delimiter must be one character")
        self._p = ctypes.POINTER(EbicTextMatrix)()
        _check(_lib_read_text(os.fsencode(path), d,
                              None if missing is None else str(missing).encode(),
                              ctypes.byref(self._p)), "ebic_read_matrix_text")
        t = self._p.contents
        self.rows, self.cols = int(t.rows), int(t.cols)
        self.values = np.ctypeslib.as_array(t.values, (self.rows * self.cols,)) \
            .reshape(self.rows, self.cols).copy()
        self.row_names = [t.row_names[i].decode() for i in range(self.rows)] \
            if bool(t.row_names) else None
        self.col_names = [t.col_names[i].decode() for i in range(self.cols)] \
            if bool(t.col_names) else None

    def close(self):
        if getattr(self, "_p", None):
            _lib_free_text(self._p)
            self._p = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()


def read_matrix_text(path, delimiter=None, missing=None):
    """(values, row_names, col_names) of a delimited text matrix; see ebic_read_matrix_text."""
    with TextMatrix(path, delimiter, missing) as t:
        return t.values, t.row_names, t.col_names


def write_biclusters(path, result, rows, names=None, title="EBIC"):
    """Write an ebic_run result dict (members, counts, bitmaps) in the biclust result-file
    layout; `rows` is the matrix's row count, `names` an open TextMatrix or None."""
    n = len(result["members"])
    W = words(rows)
    cols = np.ascontiguousarray(result["cols"], dtype=np.uint16) if n else np.zeros(1, np.uint16)
    offs = np.ascontiguousarray(result["offsets"], dtype=np.uint32)
    counts = np.ascontiguousarray(result["counts"], dtype=np.uint32) if n else np.zeros(1, np.uint32)
    qual = np.ascontiguousarray(result["quality"], dtype=np.uint64) if n else np.zeros(1, np.uint64)
    bm = np.ascontiguousarray(result["bitmaps"], dtype=np.uint32).reshape(-1) if n \
        else np.zeros(1, np.uint32)
    r = EbicResult()
    r.n = n
    r.cols = cols.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))
    r.offsets = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    r.counts = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    r.quality = qual.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    r.bitmaps = bm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    r.words = W
    nm = names._p if names is not None else None
    _check(_lib_write_bic(os.fsencode(path), title.encode(), ctypes.byref(r), nm),
           "ebic_write_biclusters")
