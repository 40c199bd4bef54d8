"""Row-sharded scoring: one matrix spread over several GPUs by rows, one all-reduce per generation.

The paper's multi-GPU support spreads the rows of one matrix over up to 8 GPUs (Abstract;
Methods, "Support for Big Data"; Results, Table 1 and Fig. 1). Rows are independent, so a
candidate's row count, its overlaps with the archive members and the members' own row counts
are sums over row ranges; only the fitness needs the whole sums. A generation on N shards:

  1. every rank: ebic_eval_partials on its shard, into one packed uint32 buffer
     [counts (P) | overlaps (P x K) | archive counts (K)];
  2. one all-reduce (sum) of that buffer over the ranks (P + P*K + K values);
  3. every rank: ebic_fitness_reduced on the sums, the same fitness everywhere.

Sums fit in 32 bits (each is at most the total row count, below 2^31), so the buffer travels as
int32 and the sum is exact.

``shard_ranges`` splits the rows so that every shard starts on a multiple of 32 rows (a shard's
bitmap word w is then the whole matrix's word row_offset/32 + w). ``ShardedScorer`` runs the
three steps on device buffers, with the collective given as a function (torch.distributed's
all_reduce under torchrun; any exact sum in tests).
"""
from __future__ import annotations

import numpy as np


def shard_ranges(total_rows: int, n_shards: int, align: int = 32):
    """(row_offset, rows) of each of n_shards shards: contiguous, covering [0, total_rows),
    offsets multiples of `align`, sizes as equal as that allows (the last takes the rest)."""
    if n_shards < 1 or total_rows < 1:
        raise ValueError("need at least one shard and one row")
    units = -(-total_rows // align)
    out, start = [], 0
    for k in range(n_shards):
        end_units = (units * (k + 1)) // n_shards
        end = min(total_rows, end_units * align)
        out.append((start, end - start))
        start = end
    if any(r <= 0 for _, r in out):
        raise ValueError(f"{total_rows} rows are too few for {n_shards} shards of {align}-row "
                         "units")
    return out


def packed_size(P: int, K: int) -> int:
    return P + P * K + K


def views(buf, P: int, K: int):
    """counts [P], overlaps [P, K] and archive counts [K] as views of one packed buffer
    (a torch tensor or a numpy array)."""
    counts = buf[:P]
    overlaps = buf[P:P + P * K].reshape(P, K) if K else None
    acounts = buf[P + P * K:P + P * K + K] if K else None
    return counts, overlaps, acounts


def reduce_sum(dist):
    """The collective of step 2 under torch.distributed: an in-place sum over the ranks."""
    def f(buf):
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    return f


class ShardedScorer:
    """One rank's share of sharded generations on its shard matrix (device-resident inputs).

    ``score`` runs partials -> all-reduce -> fitness for a population (device int16/int32
    tensors holding uint16 columns / uint32 offsets) against an archive whose bitmaps are this
    shard's rows of the members' bitmaps. Returns the device fitness tensor (int64 holding
    uint64) and the reduced packed buffer (int32 holding uint32)."""

    def __init__(self, m, max_cand: int, max_arch: int, allreduce, device, stream=None):
        import torch
        from . import ebic
        self.torch, self.ebic = torch, ebic
        self.m = m
        self.allreduce = allreduce
        self.stream = stream
        self.buf = torch.zeros(packed_size(max_cand, max_arch), dtype=torch.int32, device=device)
        self.fit = torch.zeros(max_cand, dtype=torch.int64, device=device)

    def score(self, cols, offsets, n_cand, arch_cols, arch_offsets, arch_bitmaps, n_arch,
              negative=False):
        ebic = self.ebic
        P, K = n_cand, n_arch
        buf = self.buf[:packed_size(P, K)]
        counts, overlaps, acounts = views(buf, P, K)
        sp = None if self.stream is None else self.stream.cuda_stream
        rc = ebic.ebic_eval_partials(self.m.handle, cols, offsets, P,
                                     ebic.EBIC_NEGATIVE_TRENDS if negative else 0,
                                     arch_cols if K else None, arch_offsets if K else None,
                                     arch_bitmaps if K else None, K, counts, overlaps, acounts,
                                     None, sp)
        if rc:
            raise ebic.EbicError(rc, "ebic_eval_partials")
        self.allreduce(buf)
        fit = self.fit[:P]
        rc = ebic.ebic_fitness_reduced(self.m.handle, cols, offsets, P, counts, overlaps,
                                       arch_cols if K else None, arch_offsets if K else None,
                                       acounts, K, 0, fit, sp)
        if rc:
            raise ebic.EbicError(rc, "ebic_fitness_reduced")
        return fit, buf


def combine_bitmaps(parts, word_offsets, total_words):
    """The whole matrix's bitmaps from the shards' [n][W_s] bitmaps (numpy), by word offset."""
    n = parts[0].shape[0]
    out = np.zeros((n, total_words), dtype=np.uint32)
    for b, w0 in zip(parts, word_offsets):
        out[:, w0:w0 + b.shape[1]] = b
    return out
