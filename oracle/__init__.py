"""EBIC population-evaluation oracle -- TEST INFRASTRUCTURE ONLY.

A plain CPU restatement (``ebic_oracle.c``) of what the EBIC hot path computes, written from
arXiv 1807.09932, Methods, "Handling missing values" (rows are counted; a row follows a
candidate when its values obey the "greater or equal" relation along the candidate's column
order; missing values no longer count), plus the project's readings for the points the paper
leaves open (negative trends, bitmap layout, overlap-penalised fitness).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package. It shares no code with the CUDA library and never imports it.

The C source is compiled on first use with the system C compiler (``-O2``, no fast-math, OpenMP
when the compiler has it) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libebic_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's shared library (gcc, -O2, no fast-math). Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _open(path):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_eval.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                ctypes.c_int, ctypes.c_float, P, P, ctypes.c_uint32,
                                ctypes.c_int, P, P, ctypes.c_int]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_fitness.argtypes = [ctypes.c_int64, P, P, ctypes.c_uint32, P, P, P, P, P,
                                   ctypes.c_uint32, P, P, ctypes.c_int]
    lib.oracle_fitness.restype = ctypes.c_int
    lib.oracle_dense_ranks.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_float, P]
    lib.oracle_dense_ranks.restype = None
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(build())
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def words(rows: int) -> int:
    """Bitmap words per candidate: one LSB-first uint32 per 32 rows."""
    return (rows + 31) // 32


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def eval_population(X, cols, offsets, *, exclude_missing=True, fill_value=0.0, negative=False,
                    want_bitmaps=True, nthreads=0):
    """Counts (uint32[P]) and bitmaps (uint32[P, W] or None) of every candidate on every row.

    ``X`` is a C-contiguous float32 [R, C] array; ``cols``/``offsets`` the population in CSR
    form (uint16 columns, uint32 offsets with offsets[0] == 0).
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    cols = np.ascontiguousarray(cols, dtype=np.uint16)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    R, C = X.shape
    P = len(offsets) - 1
    counts = np.zeros(P, dtype=np.uint32)
    bitmaps = np.zeros((P, words(R)), dtype=np.uint32) if want_bitmaps else None
    rc = _load().oracle_eval(_ptr(X), R, C, C, int(exclude_missing), float(fill_value),
                             _ptr(cols), _ptr(offsets), P, int(negative), _ptr(counts),
                             _ptr(bitmaps), int(nthreads))
    if rc != 0:
        raise ValueError("invalid candidate (length 0 or > 64, column out of range, or repeat)")
    return counts, bitmaps


def fitness(R, cols, offsets, counts, bitmaps, arch_cols, arch_offsets, arch_bitmaps,
            want_overlaps=True, nthreads=0):
    """Overlap-penalised fitness (uint64[P]) and overlaps (uint32[P, K] or None)."""
    cols = np.ascontiguousarray(cols, dtype=np.uint16)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint32)
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    bitmaps = np.ascontiguousarray(bitmaps, dtype=np.uint32)
    arch_cols = np.ascontiguousarray(arch_cols, dtype=np.uint16)
    arch_offsets = np.ascontiguousarray(arch_offsets, dtype=np.uint32)
    K = len(arch_offsets) - 1
    arch_bitmaps = np.ascontiguousarray(arch_bitmaps, dtype=np.uint32).reshape(K, words(R))
    P = len(offsets) - 1
    fit = np.zeros(P, dtype=np.uint64)
    ov = np.zeros((P, K), dtype=np.uint32) if want_overlaps else None
    _load().oracle_fitness(R, _ptr(cols), _ptr(offsets), P, _ptr(counts), _ptr(bitmaps),
                           _ptr(arch_cols), _ptr(arch_offsets), _ptr(arch_bitmaps), K,
                           _ptr(fit), _ptr(ov), int(nthreads))
    return fit, ov


def dense_ranks(X, *, exclude_missing=True, fill_value=0.0):
    """Row-major uint16 dense ranks; 0xFFFF marks a missing value (exclusion on)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    R, C = X.shape
    out = np.zeros((R, C), dtype=np.uint16)
    _load().oracle_dense_ranks(_ptr(X), R, C, C, int(exclude_missing), float(fill_value),
                               _ptr(out))
    return out


def fitness_from_overlaps(cols, offsets, counts, overlaps, arch_cols, arch_offsets, arch_counts):
    """D9 from row counts and overlaps alone (no bitmaps): the quantities a row-sharded run
    sums over its shards. q(x) = n_x << (min(L_x, 33) - 1); p_c = n_c minus the largest
    overlaps[c][a] over members a whose column set meets c's and with q(a) >= q(c), 0 if none;
    F_c = p_c << (min(L_c, 33) - 1). Plain Python over candidates and members."""
    P = len(offsets) - 1
    K = len(arch_offsets) - 1
    fit = np.zeros(P, dtype=np.uint64)
    asets = [set(int(x) for x in arch_cols[arch_offsets[a]:arch_offsets[a + 1]])
             for a in range(K)]
    aq = [int(arch_counts[a]) << (min(int(arch_offsets[a + 1] - arch_offsets[a]), 33) - 1)
          for a in range(K)]
    for c in range(P):
        cset = [int(x) for x in cols[offsets[c]:offsets[c + 1]]]
        L = len(cset)
        n = int(counts[c])
        qc = n << (min(L, 33) - 1)
        worst = 0
        for a in range(K):
            if aq[a] >= qc and asets[a] & set(cset):
                worst = max(worst, int(overlaps[c][a]))
        fit[c] = (n - worst) << (min(L, 33) - 1)
    return fit
