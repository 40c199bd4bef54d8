"""Autotuner of the evaluator's tile shapes: row-tile height (slabs per shared-memory stage) and
candidate-tile size (candidate columns staged per chunk).

Neither knob changes results (the tests check every tile against the oracle); both change speed.
Which is best depends on the matrix's rank layout and column count, its row count, and the
population's size and length mix. The tuner times every allowed (tile, chunk) pair on a real
population with CUDA events, keeps the fastest, and remembers it in a JSON cache keyed by that
shape class. The next matrix of the same class is configured from the cache without timing.

The timing itself is injected (``measure(tile, chunk) -> ms``), so the cache and selection logic
run on the CPU in tests; ``gpu_measure`` builds the real one over the C ABI.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

CHUNKS = (0, 256, 1024, 4096, 16384)   # 0 = the library's built-in choice
TILES = (1, 2, 4)


def default_cache_path():
    return os.environ.get("EBIC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ebic_gb300",
                                       "autotune.json"))


def shape_key(rank_bits, cols, rows, n_cand, mean_len, negative):
    """The shape class a tuning result is valid for."""
    return (f"w{rank_bits}-c{cols}-r{int(round(math.log2(max(rows, 1))))}"
            f"-p{int(round(math.log2(max(n_cand, 1))))}-l{int(round(mean_len))}"
            f"-n{int(bool(negative))}")


class Cache:
    def __init__(self, path=None):
        self.path = path or default_cache_path()
        self._lock = threading.Lock()
        self.entries = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.entries = json.load(f)
            except (OSError, ValueError):
                self.entries = {}

    def get(self, key):
        return self.entries.get(key)

    def put(self, key, value):
        with self._lock:
            self.entries[key] = value
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            tmp = f"{self.path}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def select(measure, tiles, chunks):
    """Time every (tile, chunk) and return (best_tile, best_chunk, best_ms, table)."""
    table = {}
    for t in tiles:
        for c in chunks:
            table[(t, c)] = measure(t, c)
    (bt, bc), bms = min(table.items(), key=lambda kv: (kv[1], kv[0]))
    return bt, bc, bms, table


def tune(key, measure, tiles, chunks=CHUNKS, cache=None, force=False):
    """Look ``key`` up in the cache, else time all pairs and store the winner."""
    if cache is not None and not force:
        hit = cache.get(key)
        if hit is not None:
            return hit["tile"], hit["chunk"], hit["ms"], True
    bt, bc, bms, table = select(measure, tiles, chunks)
    if cache is not None:
        cache.put(key, {"tile": bt, "chunk": bc, "ms": bms,
                        "table": {f"{t},{c}": v for (t, c), v in table.items()}})
    return bt, bc, bms, False


# ---- GPU side -----------------------------------------------------------------------------------

def allowed_tiles(m):
    """Tile heights whose shared-memory stage fits for this matrix."""
    from . import ebic
    out = []
    for t in TILES:
        try:
            m.set_tile(t)
            out.append(t)
        except ebic.EbicError:
            pass
    m.set_tile(0)
    return out


def gpu_measure(m, dcols, doffs, n_cand, counts, bitmaps, negative=False, iters=5):
    """measure(tile, chunk) over ebic_eval_population on device buffers, timed with CUDA events
    on the current stream (median of ``iters`` after one warm-up)."""
    import torch

    from . import ebic
    stream = torch.cuda.current_stream()
    flags = ebic.EBIC_NEGATIVE_TRENDS if negative else 0

    def measure(tile, chunk):
        m.set_tile(tile)
        m.set_chunk_cols(chunk)
        times = []
        for i in range(iters + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = ebic.ebic_eval_population(m.handle, dcols, doffs, n_cand, flags, counts, bitmaps,
                                           stream.cuda_stream)
            b.record(stream)
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_population")
            b.synchronize()
            if i:
                times.append(a.elapsed_time(b))
        return statistics.median(times)

    return measure


def tune_matrix(m, dcols, doffs, n_cand, mean_len, counts, bitmaps, negative=False, cache=None,
                force=False, iters=5):
    """Tune (or configure from the cache) matrix ``m`` for populations like the one given.
    Leaves the winning tile and chunk set on ``m``; returns (tile, chunk, ms, from_cache)."""
    key = shape_key(m.rank_bits, m.cols, m.rows, n_cand, mean_len, negative)
    tiles = allowed_tiles(m)
    measure = gpu_measure(m, dcols, doffs, n_cand, counts, bitmaps, negative, iters)
    tile, chunk, ms, hit = tune(key, measure, tiles, CHUNKS, cache, force)
    m.set_tile(tile)
    m.set_chunk_cols(chunk)
    return tile, chunk, ms, hit
