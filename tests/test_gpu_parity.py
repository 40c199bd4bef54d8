"""CUDA path vs the oracle, element by element, through the C ABI (bit-exact: all results are
integers). Sizes span several row tiles with a ragged tail; the full-size methylation-shaped
workload is checked on sampled candidates the oracle computes one by one."""
import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ebic():
    import torch
    torch.cuda.init()
    from paper_1807_09932_gb300 import ebic as e
    return e


def dev_tensor(a):
    """numpy (uint16/uint32) -> torch device tensor with the same bytes."""
    import torch
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32,
            np.dtype(np.float32): np.float32, np.dtype(np.uint64): np.int64}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def check_eval(ebic, X, cols, offs, *, exclude=True, fill=0.0, negative=False, device=False,
               tile=None):
    with ebic.Matrix(X, exclude_missing=exclude, fill_value=fill) as m:
        if tile is not None:
            m.set_tile(tile)
        n = len(offs) - 1
        if device:
            import torch
            cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
            bm = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
            ebic.eval_population(m, dev_tensor(cols), dev_tensor(offs), negative=negative,
                                 counts=cnt, bitmaps=bm)
            assert m.status() == ebic.EBIC_OK
            got_c, got_b = host(cnt, np.uint32), host(bm, np.uint32)
        else:
            got_c, got_b = ebic.eval_population(m, cols, offs, negative=negative)
        exp_c, exp_b = oracle.eval_population(X, cols, offs, exclude_missing=exclude,
                                              fill_value=fill, negative=negative)
        assert np.array_equal(got_c, exp_c), np.nonzero(got_c != exp_c)[0][:10]
        assert np.array_equal(got_b, exp_b)
        # counts-only mode gives the same counts
        c2, _ = ebic.eval_population(m, cols, offs, negative=negative, want_bitmaps=False)
        assert np.array_equal(c2, exp_c)
        return exp_c, exp_b


@pytest.mark.parametrize("negative", [False, True])
def test_config1_small(ebic, negative):
    ds, cols, offs = synth.config1()
    check_eval(ebic, ds.X, cols, offs, negative=negative)


@pytest.mark.parametrize("negative", [False, True])
def test_config2_expression_shaped(ebic, negative):
    ds, cols, offs = synth.config2()
    check_eval(ebic, ds.X, cols, offs, negative=negative, device=True)


def test_config3_reduced_rows(ebic):
    ds, cols, offs = synth.config3(rows=60001)
    check_eval(ebic, ds.X, cols, offs)


@pytest.mark.parametrize("R,C", [(1, 1), (1, 5), (31, 3), (33, 2), (127, 127), (129, 128),
                                 (700, 200), (1000, 208), (513, 209), (300, 416), (257, 417),
                                 (200, 832), (5000, 64), (65537, 7)])
def test_shapes_and_ragged_tails(ebic, R, C):
    rng = np.random.default_rng(R * 1000 + C)
    X = rng.standard_normal((R, C)).astype(np.float32)
    X[rng.random((R, C)) < 0.03] = np.nan
    lmax = min(C, 12)
    cols, offs = synth.make_population(R + C, 40, C, 1, lmax)
    for neg in (False, True):
        check_eval(ebic, X, cols, offs, negative=neg)


def test_edge_values_ties_and_fill(ebic):
    from pins import tiny_matrix, all_candidates
    X = tiny_matrix(3, 600, 5, nan_frac=0.15)
    cols, offs = synth.population_from_lists(all_candidates(5, 4))
    for exclude in (True, False):
        for fill in (0.0, 999.0, -np.inf):
            for neg in (False, True):
                check_eval(ebic, X, cols, offs, exclude=exclude, fill=fill, negative=neg)


def test_long_candidates_and_many_columns(ebic):
    rng = np.random.default_rng(9)
    R, C = 3000, 100
    X = rng.standard_normal((R, C)).astype(np.float32)
    order = rng.permutation(C)[:64]
    rows = rng.choice(R, 400, replace=False)
    X[np.ix_(rows, order)] = np.sort(X[np.ix_(rows, order)], axis=1)
    cands = [list(order[:k]) for k in (1, 2, 32, 33, 63, 64)] + [list(order[::-1])]
    cols, offs = synth.population_from_lists(cands)
    c, _ = check_eval(ebic, X, cols, offs, negative=True)
    assert c[5] >= 400


@pytest.mark.parametrize("C,tile", [(50, 1), (50, 2), (50, 4), (100, 1), (100, 2), (150, 1),
                                    (300, 1), (600, 1)])
def test_tile_choice_never_changes_results(ebic, tile, C):
    ds = synth.make_dataset(77 + C, 20011, C, kind="beta", planted=[(2000, 8, False)],
                            nan_frac=0.01)
    cols, offs = synth.make_population(78, 300, C, 2, 16)
    check_eval(ebic, ds.X, cols, offs, tile=tile, negative=True)


def test_tile_that_does_not_fit_is_rejected(ebic):
    X = np.zeros((5000, 64), np.float32)
    with ebic.Matrix(X) as m:
        with pytest.raises(ebic.EbicError) as ei:
            m.set_tile(4)  # 64 columns x 4 slabs x 512 B = 128 KB > one pipeline stage
        assert ei.value.code == ebic.EBIC_ERR_UNSUPPORTED
        m.set_tile(2)
        assert m.tile == (2, 512)


def test_rank_export_matches_dense_ranks(ebic):
    from pins import tiny_matrix
    for C in (1, 2, 5, 31, 32, 33, 63, 64, 65, 127, 128, 300):
        X = tiny_matrix(C, 700, C, nan_frac=0.1)
        rng = np.random.default_rng(C)
        X[:, : C // 2] += rng.standard_normal((700, C // 2)).astype(np.float32)
        for exclude in (True, False):
            with ebic.Matrix(X, exclude_missing=exclude, fill_value=1.0) as m:
                got = m.ranks()
            want = oracle.dense_ranks(X, exclude_missing=exclude, fill_value=1.0)
            assert np.array_equal(got, want)


def test_rank_export_matches_dense_ranks_past_one_round_of_slabs(ebic):
    """Matrices of more 512-row slabs than the GPU has SMs: several rounds of slabs per CTA, a
    partial last round, a ragged last slab and one almost all padding; rows on 16-byte
    boundaries (the staged form) and not."""
    from pins import tiny_matrix
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cases = [(sms * 512 + 44 * 512 + 37, 64, True),     # a short last round
             (sms * 512 + 130 * 512 + 3, 32, True),     # a long last round
             (sms * 512 + 130 * 512 + 3, 64, False),
             (2 * sms * 512 + 1, 36, True),             # one padding chunk, mostly empty
             (sms * 512 + 77 * 512, 61, True)]          # rows not on 16-byte boundaries
    for R, C, exclude in cases:
        X = tiny_matrix(R + C, R, C, nan_frac=0.02)
        rng = np.random.default_rng(R)
        X[:, : C // 2] += rng.standard_normal((R, C // 2)).astype(np.float32)
        with ebic.Matrix(X, exclude_missing=exclude, fill_value=1.0) as m:
            got = m.ranks()
        want = oracle.dense_ranks(X, exclude_missing=exclude, fill_value=1.0)
        assert np.array_equal(got, want), (R, C, exclude)


def _near_equal_rows(seed, R, C):
    """Rows whose values crowd into a few groups of float32 bit patterns one unit apart (so many
    share all but their lowest key bits), with exact ties, signed zeros, infinities and NaN."""
    rng = np.random.default_rng(seed)
    X = np.empty((R, C), dtype=np.float32)
    for r in range(R):
        groups = int(rng.integers(1, 5))
        bases = rng.integers(0x00800000, 0x7F000000, size=groups).astype(np.uint64)
        bases[rng.random(groups) < 0.4] |= 0x80000000  # negative values
        pick = rng.integers(0, groups, size=C)
        spread = int(rng.choice([1, 2, 4, 64, 200]))
        bits = (bases[pick] + rng.integers(0, spread, size=C).astype(np.uint64)) & 0xFFFFFFFF
        X[r] = bits.astype(np.uint32).view(np.float32)
        special = rng.random(C)
        X[r, special < 0.03] = np.float32(0.0)
        X[r, (special >= 0.03) & (special < 0.06)] = np.float32(-0.0)
        X[r, (special >= 0.06) & (special < 0.08)] = np.float32(np.inf)
        X[r, (special >= 0.08) & (special < 0.10)] = np.float32(np.nan)
        if r % 7 == 0:
            X[r, :] = X[r, 0]  # a row of one value
    return X


@pytest.mark.parametrize("C", [2, 5, 31, 32, 33, 48, 64])
def test_rank_transform_near_equal_values(ebic, C):
    """Rows of up to 64 columns are sorted on words that keep the top 26 (or 27) key bits beside
    the column, and rows whose sort could not order two values are ranked again exactly: runs of
    equal values, two values one key unit apart in either order, and longer runs of near-equal
    values all give the oracle's dense ranks, and the evaluation on them gives the oracle's
    counts."""
    X = _near_equal_rows(C, 1500, C)
    for exclude in (True, False):
        with ebic.Matrix(X, exclude_missing=exclude, fill_value=0.0) as m:
            got = m.ranks()
            want = oracle.dense_ranks(X, exclude_missing=exclude, fill_value=0.0)
            assert np.array_equal(got, want)
            cols, offs = synth.make_population(C + 1, 200, C, 1, min(C, 8))
            for neg in (False, True):
                c, b = ebic.eval_population(m, cols, offs, negative=neg, direct=True)
                ec, eb = oracle.eval_population(X, cols, offs, exclude_missing=exclude,
                                                fill_value=0.0, negative=neg)
                assert np.array_equal(c, ec) and np.array_equal(b, eb)


@pytest.mark.parametrize("pad", [7, 4])
@pytest.mark.parametrize("C", [3, 32, 48, 50, 64, 100, 300])
def test_rank_transform_reads_strided_device_rows(ebic, C, pad):
    # a device matrix whose rows are further apart than its columns (ld > cols) is ranked in place
    # (pad 4 keeps rows of a multiple of four columns on 16-byte boundaries: the vector loads)
    import torch
    from pins import tiny_matrix
    R = 1100
    Xw = tiny_matrix(C + 11, R, C + pad, nan_frac=0.05)
    Xw[:, : C // 2] += np.random.default_rng(C).standard_normal((R, C // 2)).astype(np.float32)
    dXw = torch.from_numpy(Xw).cuda()
    h = ebic.ebic_load_matrix(dXw, R, C, C + pad, ebic.EBIC_EXCLUDE_MISSING, 0.0)
    try:
        got = np.zeros((R, C), dtype=np.uint16)
        ebic.ebic_matrix_ranks(h, got)
    finally:
        ebic.ebic_free_matrix(h)
    want = oracle.dense_ranks(np.ascontiguousarray(Xw[:, :C]), exclude_missing=True, fill_value=0.0)
    assert np.array_equal(got, want)


def test_rank_transform_every_nan_pattern(ebic):
    """Every float32 NaN bit pattern (both signs, quiet and signalling payloads) is a missing value
    with exclusion on and takes the fill value's code with exclusion off, beside real values."""
    pos = np.arange(0x7F800001, 0x80000000, dtype=np.uint64)
    nans = np.concatenate([pos, pos | 0x80000000]).astype(np.uint32)
    per_row = 48
    R = (nans.size + per_row - 1) // per_row
    rng = np.random.default_rng(3)
    X = rng.standard_normal((R, 64)).astype(np.float32)
    flat = np.full(R * per_row, 0x7FC00000, np.uint32)
    flat[:nans.size] = nans
    X[:, :per_row] = flat.reshape(R, per_row).view(np.float32)
    with ebic.Matrix(X, exclude_missing=True) as m:
        got = m.ranks()
    assert (got[:, :per_row] == 0xFFFF).all()
    sample = rng.choice(R, 3000, replace=False)
    want = oracle.dense_ranks(np.ascontiguousarray(X[sample]), exclude_missing=True)
    assert np.array_equal(got[sample], want)
    with ebic.Matrix(X, exclude_missing=False, fill_value=0.25) as m:
        got = m.ranks()
    assert (got[:, :per_row] == got[:, :1]).all()
    want = oracle.dense_ranks(np.ascontiguousarray(X[sample]), exclude_missing=False,
                              fill_value=0.25)
    assert np.array_equal(got[sample], want)


@pytest.mark.parametrize("C", [17, 32, 64])
def test_rank_transform_subnormals_and_signed_zeros(ebic, C):
    """Subnormals of both signs, the smallest normals, and both zeros keep their order and ties."""
    rng = np.random.default_rng(C)
    bits = np.concatenate([
        rng.integers(1, 0x00800000, size=8).astype(np.uint32),             # positive subnormals
        rng.integers(1, 0x00800000, size=8).astype(np.uint32) | 0x80000000,  # negative subnormals
        np.array([0x00800000, 0x80800000, 0x00000000, 0x80000000, 0x00000001, 0x80000001],
                 np.uint32)])
    X = bits[rng.integers(0, bits.size, size=(5000, C))].view(np.float32)
    for exclude in (True, False):
        with ebic.Matrix(X, exclude_missing=exclude, fill_value=-0.0) as m:
            got = m.ranks()
        want = oracle.dense_ranks(X, exclude_missing=exclude, fill_value=-0.0)
        assert np.array_equal(got, want)


def test_rank_transform_many_slabs_per_cta(ebic):
    """A matrix of several slabs per CTA of the ranking launch (330,001 rows of 64 beta values,
    one row in twenty near-equal), on device memory: each CTA's list of rows to rank exactly is
    kept apart and every row gets the oracle's ranks."""
    import torch
    R, C = 330001, 64
    ds = synth.make_dataset(5, R, C, kind="beta", planted=[(4000, 8, False)], nan_frac=0.01)
    X = ds.X.copy()
    rows = np.random.default_rng(6).choice(R, R // 20, replace=False)
    X[rows] = _near_equal_rows(7, rows.size, C)
    with ebic.Matrix(torch.from_numpy(X).cuda(), exclude_missing=True) as m:
        got = m.ranks()
    want = oracle.dense_ranks(X, exclude_missing=True)
    assert np.array_equal(got, want)


def test_empty_population_is_a_noop(ebic):
    X = np.zeros((10, 3), np.float32)
    with ebic.Matrix(X) as m:
        c, b = ebic.eval_population(m, np.zeros(0, np.uint16), np.zeros(1, np.uint32))
        assert c.shape == (0,)


def test_invalid_candidates_rejected_on_host_and_device(ebic):
    import torch
    X = np.random.default_rng(0).standard_normal((100, 6)).astype(np.float32)
    bad = [synth.population_from_lists([[0, 0]]), synth.population_from_lists([[6]]),
           (np.zeros(0, np.uint16), np.array([0, 0], np.uint32)),
           (np.arange(3, dtype=np.uint16), np.array([1, 3], np.uint32))]
    with ebic.Matrix(X) as m:
        for cols, offs in bad:
            with pytest.raises(ebic.EbicError) as ei:
                ebic.eval_population(m, cols, offs)
            assert ei.value.code == ebic.EBIC_ERR_INVALID_ARG
            # device-resident lists: the device check defers the error to ebic_matrix_status
            n = len(offs) - 1
            cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
            dcols = dev_tensor(cols) if len(cols) else torch.zeros(1, dtype=torch.int16,
                                                                   device="cuda")
            ebic.eval_population(m, dcols, dev_tensor(offs), counts=cnt, want_bitmaps=False)
            assert m.status() == ebic.EBIC_ERR_INVALID_ARG
            assert m.status() == ebic.EBIC_OK  # cleared
            # ... and a host output makes the same call report it directly
            with pytest.raises(ebic.EbicError):
                ebic.eval_population(m, dcols, dev_tensor(offs), want_bitmaps=False)
            assert m.status() == ebic.EBIC_ERR_INVALID_ARG
        # the context is still usable
        cols, offs = synth.make_population(1, 20, 6, 1, 6)
        got, _ = ebic.eval_population(m, cols, offs)
        assert np.array_equal(got, oracle.eval_population(X, cols, offs)[0])


def _archive(cols, offs, counts, bm, idx):
    acand = [list(cols[offs[i]:offs[i + 1]]) for i in idx]
    acols, aoffs = synth.population_from_lists(acand)
    return acols, aoffs, bm[idx].copy()


@pytest.mark.parametrize("cfg", ["config1", "config2"])
def test_fitness_matches_oracle(ebic, cfg):
    ds, cols, offs = getattr(synth, cfg)()
    X = ds.X
    R = X.shape[0]
    cnt, bm = oracle.eval_population(X, cols, offs, negative=ds.negative)
    rng = np.random.default_rng(5)
    with ebic.Matrix(X) as m:
        for K in (0, 1, 7, 40):
            idx = rng.choice(len(cnt), size=K, replace=False)
            acols, aoffs, abm = _archive(cols, offs, cnt, bm, idx)
            f, ov = ebic.fitness(m, cols, offs, cnt, bm, acols, aoffs, abm)
            ef, eov = oracle.fitness(R, cols, offs, cnt, bm, acols, aoffs, abm)
            assert np.array_equal(f, ef)
            assert np.array_equal(ov.reshape(eov.shape), eov)
        # random archive bitmaps, device-resident everything
        import torch
        K = 20
        acand = [list(rng.choice(X.shape[1], rng.integers(1, 9), replace=False))
                 for _ in range(K)]
        acols, aoffs = synth.population_from_lists(acand)
        abm = synth.random_bitmaps(11, K, R, 0.3)
        n = len(cnt)
        fd = torch.zeros(n, dtype=torch.int64, device="cuda")
        od = torch.zeros((n, K), dtype=torch.int32, device="cuda")
        ebic.fitness(m, dev_tensor(cols), dev_tensor(offs), dev_tensor(cnt), dev_tensor(bm),
                     dev_tensor(acols), dev_tensor(aoffs), dev_tensor(abm), fitness_out=fd,
                     overlaps=od)
        assert m.status() == ebic.EBIC_OK
        ef, eov = oracle.fitness(R, cols, offs, cnt, bm, acols, aoffs, abm)
        assert np.array_equal(host(fd, np.uint64), ef)
        assert np.array_equal(host(od, np.uint32), eov)


def test_config3_full_size_sampled(ebic):
    """436,444 rows: all candidates on the GPU in the bench's configuration; 48 sampled
    candidates recomputed by the oracle one by one; all counts checked against properties that
    hold at any size (count == popcount of the bitmap, padding bits zero)."""
    import torch
    ds, cols, offs = synth.config3()
    X = ds.X
    R = X.shape[0]
    n = len(offs) - 1
    with ebic.Matrix(torch.from_numpy(X).cuda()) as m:
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        bm = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
        ebic.eval_population(m, dev_tensor(cols), dev_tensor(offs), counts=cnt, bitmaps=bm)
        assert m.status() == ebic.EBIC_OK
        got_c = host(cnt, np.uint32)
        got_b = host(bm, np.uint32)
    lut = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint32)
    pop = np.concatenate([lut[got_b[i:i + 64].view(np.uint8)].sum(axis=1, dtype=np.uint64)
                          for i in range(0, n, 64)])
    assert np.array_equal(pop, got_c)
    tail = R % 32
    if tail:
        assert np.all(got_b[:, -1] >> tail == 0)
    idx = np.random.default_rng(3).choice(n, size=48, replace=False)
    sc, so = synth.population_from_lists([list(cols[offs[i]:offs[i + 1]]) for i in idx])
    ec, eb = oracle.eval_population(X, sc, so)
    assert np.array_equal(got_c[idx], ec)
    assert np.array_equal(got_b[idx], eb)


def test_bounded_wait_expires_cleanly_and_context_survives(ebic):
    """Failure detection on the GPU without a fault: a wait that nothing satisfies expires after
    its limit, the kernel reports it, and the next evaluation runs normally."""
    rc = ebic.ebic_selftest_wait_timeout(1_000_000)
    assert rc == ebic.EBIC_ERR_DEVICE_TIMEOUT
    assert "expired" in ebic.ebic_last_error()
    ds, cols, offs = synth.config1()
    check_eval(ebic, ds.X, cols, offs)
