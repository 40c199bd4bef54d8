"""Row shards of one matrix on one GPU, combined, against the unsharded call and the oracle.

The paper spreads the rows of one matrix over several GPUs (Abstract; Methods, "Support for Big
Data"; Results, Fig. 1). Here every shard of a split is loaded with ebic_load_matrix_shard on
the one GPU, each gives its partials (ebic_eval_partials: counts, overlaps, the archive members'
counts, bitmaps), the partials are summed, and ebic_fitness_reduced turns the sums into the
fitness. Everything must equal ebic_eval_fitness on the whole matrix and the oracle, bit for bit:
counts, fitness, the overlaps of members sharing a column, and the bitmaps placed by word offset.
The collective itself is covered by the two-rank gloo test on the CPU.
"""
import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ebic():
    import torch
    torch.cuda.init()
    from paper_1807_09932_gb300 import ebic as e
    return e


def _share_mask(cols, offs, acols, aoffs):
    P, K = len(offs) - 1, len(aoffs) - 1
    sets = [set(cols[offs[i]:offs[i + 1]].tolist()) for i in range(P)]
    asets = [set(acols[aoffs[a]:aoffs[a + 1]].tolist()) for a in range(K)]
    return np.array([[bool(sets[i] & asets[a]) for a in range(K)] for i in range(P)],
                    dtype=bool).reshape(P, K)


def _run_split(ebic, X, splits, cols, offs, acols, aoffs, abm_whole, negative, pairs):
    """Partials of every shard, summed; returns (counts, overlaps, arch counts, bitmaps,
    fitness from the sums)."""
    R = X.shape[0]
    P, K = len(offs) - 1, len(aoffs) - 1
    tot_c = np.zeros(P, np.int64)
    tot_o = np.zeros((P, K), np.int64)
    tot_a = np.zeros(K, np.int64)
    parts, w0s, mats = [], [], []
    try:
        for o, r in splits:
            m = ebic.Matrix(X[o:o + r], row_offset=o, total_rows=R)
            mats.append(m)
            assert (m.row_offset, m.total_rows, m.word_offset) == (o, R, o // 32)
            if pairs:
                m.build_pairs()
            w0 = o // 32
            abm = np.ascontiguousarray(abm_whole[:, w0:w0 + m.words]) if K else abm_whole
            c, ov, an, b = ebic.eval_partials(m, cols, offs, acols, aoffs, abm,
                                              negative=negative, want_bitmaps=True)
            tot_c += c
            if K:
                tot_o += ov
                tot_a += an
            parts.append(b)
            w0s.append(w0)
        counts = tot_c.astype(np.uint32)
        ov = tot_o.astype(np.uint32)
        acnt = tot_a.astype(np.uint32)
        fit = ebic.fitness_reduced(mats[0], cols, offs, counts, ov, acols, aoffs, acnt)
        bms = shard.combine_bitmaps(parts, w0s, (R + 31) // 32)
    finally:
        for m in mats:
            m.close()
    return counts, ov, acnt, bms, fit


SPLITS = {
    "one shard": lambda R: [(0, R)],
    "two": lambda R: shard.shard_ranges(R, 2),
    "three uneven": lambda R: [(0, 64), (64, (R - 64 - 33) // 32 * 32),
                               (64 + (R - 64 - 33) // 32 * 32, R - 64 - (R - 64 - 33) // 32 * 32)],
    "eight": lambda R: shard.shard_ranges(R, 8),
}


@pytest.mark.parametrize("pairs", [True, False])
@pytest.mark.parametrize("K", [0, 7, 20, 33, 70])
@pytest.mark.parametrize("split", sorted(SPLITS))
def test_shards_sum_to_the_whole_matrix(ebic, split, K, pairs):
    R, C = 20011, 40
    ds = synth.make_dataset(31, R, C, kind="beta",
                            planted=[(3000, 8, False), (2000, 6, True), (500, 12, False)],
                            nan_frac=0.01)
    X = ds.X
    cols, offs = synth.make_population(32, 300, C, 1, 14)
    lists = [list(p.cols) for p in ds.planted]
    lists += [list(cols[offs[i]:offs[i + 1]]) for i in range(0, 3 * max(K - 3, 0), 3)]
    acols, aoffs = synth.population_from_lists(lists[:K]) if K else (
        np.zeros(0, np.uint16), np.zeros(1, np.uint32))
    for neg in (False, True):
        ec, eb = oracle.eval_population(X, cols, offs, negative=neg)
        if K:
            _, eab = oracle.eval_population(X, acols, aoffs, negative=neg)
        else:
            eab = np.zeros((0, (R + 31) // 32), np.uint32)
        ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, eab)
        c, ov, acnt, bms, fit = _run_split(ebic, X, SPLITS[split](R), cols, offs, acols, aoffs,
                                           eab, neg, pairs)
        assert np.array_equal(c, ec)
        assert np.array_equal(bms, eb)
        assert np.array_equal(fit, ef)
        if K:
            share = _share_mask(cols, offs, acols, aoffs)
            assert np.array_equal(ov[share], eov[share])
            ean = [int(np.unpackbits(eab[a].view(np.uint8)).sum()) for a in range(K)]
            assert list(acnt) == ean
        # the unsharded call agrees
        with ebic.Matrix(X) as m:
            if pairs:
                m.build_pairs()
            uc, _, uf, _ = ebic.eval_fitness(m, cols, offs, acols, aoffs, eab, negative=neg)
        assert np.array_equal(uc, ec) and np.array_equal(uf, ef)


def test_methylation_workload_on_four_shards(ebic):
    """436,444 x 64, 1,600 candidates, the bench's 20-member archive form, four shards with pair
    tables, device buffers and the packed reduction buffer of ShardedScorer (the sum taken on the
    device over the four shards' buffers)."""
    import torch
    ds, cols, offs = synth.config3()
    X = ds.X
    R = X.shape[0]
    P = len(offs) - 1
    ec, eb = oracle.eval_population(X, cols, offs)
    top = np.argsort(-ec.astype(np.int64), kind="stable")[:10]
    acols, aoffs = synth.population_from_lists([list(p.cols) for p in ds.planted] +
                                               [list(cols[offs[i]:offs[i + 1]]) for i in top])
    K = len(aoffs) - 1
    _, eab = oracle.eval_population(X, acols, aoffs)
    ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, eab, want_overlaps=False)

    def d(a):
        view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
        return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()

    dc, do, dac, dao = d(cols), d(offs), d(acols), d(aoffs)
    splits = shard.shard_ranges(R, 4)
    mats, scorers, bufs = [], [], []
    total = None
    try:
        for k, (o, r) in enumerate(splits):
            m = ebic.Matrix(torch.from_numpy(X[o:o + r]).cuda(), row_offset=o, total_rows=R)
            mats.append(m)
            m.build_pairs()
            abm = d(np.ascontiguousarray(eab[:, o // 32:o // 32 + m.words]))
            bufs.append(abm)
        # step 1 on every shard into its own packed buffer; step 2 on the device: the sum of the
        # buffers, handed to each shard's scorer as its all-reduce; step 3 on every shard
        packed = []
        for m, abm in zip(mats, bufs):
            sc = shard.ShardedScorer(m, P, K, allreduce=lambda b: None, device="cuda")
            _, buf = sc.score(dc, do, P, dac, dao, abm, K)
            packed.append(buf.clone())
        total = torch.stack(packed).sum(dim=0, dtype=torch.int64).to(torch.int32)

        def set_total(b):
            b.copy_(total)
        fits = []
        for m, abm in zip(mats, bufs):
            sc = shard.ShardedScorer(m, P, K, allreduce=set_total, device="cuda")
            fit, buf = sc.score(dc, do, P, dac, dao, abm, K)
            fits.append(fit.cpu().numpy().view(np.uint64).copy())
            assert m.status() == ebic.EBIC_OK
    finally:
        for m in mats:
            m.close()
    c, _, _ = shard.views(total.cpu().numpy().view(np.uint32), P, K)
    assert np.array_equal(c, ec)
    for f in fits:
        assert np.array_equal(f, ef)


def test_shard_rules(ebic):
    X = np.random.default_rng(1).standard_normal((200, 6)).astype(np.float32)
    for o, r, R in ((16, 64, 200), (0, 40, 200), (192, 16, 200), (0, 201, 200), (-32, 64, 200)):
        with pytest.raises(ebic.EbicError) as ei:
            ebic.Matrix(X[:max(r, 1)] if r <= 200 else np.zeros((r, 6), np.float32),
                        row_offset=o, total_rows=R)
        assert ei.value.code == ebic.EBIC_ERR_INVALID_ARG
    # a shard that is not the whole matrix cannot run the generation loop
    with ebic.Matrix(X[:64], row_offset=64, total_rows=200) as m:
        with pytest.raises(ebic.EbicError) as ei:
            ebic.ebic_run(m.handle, ebic.ebic_params_default(population=20, generations=2))
        assert ei.value.code == ebic.EBIC_ERR_UNSUPPORTED
    # the last shard may be ragged; a whole-matrix "shard" runs ebic_run
    with ebic.Matrix(X[192:], row_offset=192, total_rows=200) as m:
        assert m.rows == 8 and m.word_offset == 6
    with ebic.Matrix(X, row_offset=0, total_rows=200) as m:
        res = ebic.ebic_run(m.handle, ebic.ebic_params_default(population=20, generations=2,
                                                               max_len=6))
        assert res["generations_run"] == 2
