"""Row-sharded scoring on the CPU: the shard split, the packed reduction over two gloo ranks, and
the fitness after the sum (the paper's multi-GPU layout: rows of one matrix spread over GPUs,
Abstract; Methods, "Support for Big Data").

Each rank computes its shard's partials (row counts, overlaps with the archive, the members' row
counts) with the CPU oracle on its rows, packs them into one buffer with the package's packing,
and sums it with the package's collective over gloo. The sums must equal the oracle's values on
the whole matrix, and the fitness from the sums (D9 from counts and overlaps) the oracle's
fitness on the whole matrix.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import shard, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_the_rows_on_word_boundaries():
    for R, n in ((1, 1), (31, 1), (33, 2), (1000, 3), (436444, 8), (4096, 4), (65, 3)):
        rs = shard.shard_ranges(R, n)
        assert len(rs) == n
        assert rs[0][0] == 0 and sum(r for _, r in rs) == R
        for (o, r), (o2, _) in zip(rs, rs[1:]):
            assert o + r == o2 and o % 32 == 0 and r % 32 == 0
        assert rs[-1][0] % 32 == 0
        sizes = [r for _, r in rs]
        assert max(sizes) - min(sizes) <= 64
    with pytest.raises(ValueError):
        shard.shard_ranges(40, 3)      # two 32-row units cannot make three shards


def test_views_of_the_packed_buffer():
    P, K = 5, 3
    buf = np.arange(shard.packed_size(P, K))
    c, o, a = shard.views(buf, P, K)
    assert list(c) == [0, 1, 2, 3, 4] and o.shape == (5, 3) and o[1, 0] == 8
    assert list(a) == [20, 21, 22]
    c, o, a = shard.views(np.arange(4), 4, 0)
    assert o is None and a is None


def _problem(seed=3, R=3001, C=24):
    ds = synth.make_dataset(seed, R, C, planted=[(400, 6, False), (300, 5, True)], nan_frac=0.02)
    cols, offs = synth.make_population(seed + 1, 90, C, 1, 9)
    acols, aoffs = synth.make_population(seed + 2, 7, C, 2, 6)
    return ds.X, cols, offs, acols, aoffs


def test_fitness_from_overlaps_is_the_fitness():
    """Pin of the oracle's count-and-overlap form of D9 against its bitmap form (itself pinned
    against Python sets in tests/pins.py), archives of 0 to 7 members, both trend options."""
    X, cols, offs, acols, aoffs = _problem()
    R = X.shape[0]
    for neg in (False, True):
        c, b = oracle.eval_population(X, cols, offs, negative=neg)
        _, ab = oracle.eval_population(X, acols, aoffs, negative=neg)
        for k in (0, 1, 7):
            ac, ao = acols[:aoffs[k]], aoffs[:k + 1]
            f, ov = oracle.fitness(R, cols, offs, c, b, ac, ao, ab[:k])
            an = np.array([int(np.unpackbits(ab[a].view(np.uint8)).sum()) for a in range(k)])
            g = oracle.fitness_from_overlaps(cols, offs, c, ov if k else np.zeros((len(c), 0)),
                                             ac, ao, an)
            assert np.array_equal(f, g)


def _partials(X, rows, cols, offs, acols, aoffs, negative):
    """One shard's partials by the oracle: counts, overlaps and member counts over its rows."""
    o, r = rows
    Xs = X[o:o + r]
    c, b = oracle.eval_population(Xs, cols, offs, negative=negative)
    _, ab = oracle.eval_population(Xs, acols, aoffs, negative=negative)
    _, ov = oracle.fitness(r, cols, offs, c, b, acols, aoffs, ab)
    an = np.array([int(np.unpackbits(ab[a].view(np.uint8)).sum()) for a in range(len(aoffs) - 1)],
                  dtype=np.uint32)
    return c, ov, an, b


def _rank_main(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        X, cols, offs, acols, aoffs = _problem()
        P, K = len(offs) - 1, len(aoffs) - 1
        out = {}
        for neg in (False, True):
            rows = shard.shard_ranges(X.shape[0], ws)[rank]
            c, ov, an, _ = _partials(X, rows, cols, offs, acols, aoffs, neg)
            buf = torch.zeros(shard.packed_size(P, K), dtype=torch.int32)
            bc, bo, ba = shard.views(buf, P, K)
            bc.copy_(torch.from_numpy(c.astype(np.int32)))
            bo.copy_(torch.from_numpy(ov.astype(np.int32)))
            ba.copy_(torch.from_numpy(an.astype(np.int32)))
            shard.reduce_sum(dist)(buf)
            out[str(neg)] = buf.numpy().astype(np.int64).tolist()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(out, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_whole_matrix(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    X, cols, offs, acols, aoffs = _problem()
    R = X.shape[0]
    P, K = len(offs) - 1, len(aoffs) - 1
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for neg in (False, True):
        assert got[0][str(neg)] == got[1][str(neg)]        # every rank holds the same sums
        c, o, a = shard.views(np.array(got[0][str(neg)], dtype=np.int64), P, K)
        ec, eb = oracle.eval_population(X, cols, offs, negative=neg)
        _, eab = oracle.eval_population(X, acols, aoffs, negative=neg)
        ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, eab)
        ean = [int(np.unpackbits(eab[i].view(np.uint8)).sum()) for i in range(K)]
        assert np.array_equal(c, ec) and np.array_equal(o, eov) and list(a) == ean
        f = oracle.fitness_from_overlaps(cols, offs, c, o, acols, aoffs, a)
        assert np.array_equal(f, ef)
        # and the shards' bitmaps, placed by word offset, are the whole matrix's
        parts, w0 = [], []
        for rows in shard.shard_ranges(R, ws):
            parts.append(_partials(X, rows, cols, offs, acols, aoffs, neg)[3])
            w0.append(rows[0] // 32)
        assert np.array_equal(shard.combine_bitmaps(parts, w0, eb.shape[1]), eb)
