"""ebic_eval_fitness (one generation's scoring in one call) against the oracle, bit for bit:
counts, bitmaps, fitness and overlaps, on the fused pair-table pass (evaluation and archive
overlaps in one kernel),
on its fallbacks (EBIC_EVAL_DIRECT, no pair table, archives over 64 members) and with
device-resident inputs."""
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
    import torch
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32,
            np.dtype(np.uint64): np.int64}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def make_archive(rng, seed, cols, offs, bm, C, R, K):
    """K members: about half taken from the population (their bitmaps are candidates' bitmaps,
    so overlaps are large and some members share the candidates' columns), the rest random
    column sets with random bitmaps."""
    n = len(offs) - 1
    k_pop = min(K // 2, n)
    idx = rng.choice(n, size=k_pop, replace=False)
    lists = [list(cols[offs[i]:offs[i + 1]]) for i in idx]
    lists += [list(rng.choice(C, int(rng.integers(1, min(C, 8) + 1)), replace=False))
              for _ in range(K - k_pop)]
    acols, aoffs = synth.population_from_lists(lists)
    abm = np.concatenate([bm[idx], synth.random_bitmaps(seed, K - k_pop, R, 0.2)]) \
        if K else np.zeros((0, (R + 31) // 32), dtype=np.uint32)
    return acols, aoffs, np.ascontiguousarray(abm, dtype=np.uint32)


def random_matrix(rng, R, C):
    X = rng.standard_normal((R, C)).astype(np.float32)
    X[rng.random((R, C)) < 0.03] = np.nan
    X[rng.random((R, C)) < 0.03] = 0.5  # ties
    return X


@pytest.mark.parametrize("R,C", [(1, 3), (33, 5), (4095, 12), (4097, 40), (9000, 64),
                                 (1500, 200)])
@pytest.mark.parametrize("negative", [False, True])
def test_matches_oracle_all_routes(ebic, R, C, negative):
    rng = np.random.default_rng(R * 31 + C + negative)
    X = random_matrix(rng, R, C)
    cols, offs = synth.make_population(R + C, 150, C, 1, min(C, 12))
    ec, eb = oracle.eval_population(X, cols, offs, negative=negative)
    with ebic.Matrix(X) as m:
        m.build_pairs()
        for K in (0, 1, 20, 64, 65):
            acols, aoffs, abm = make_archive(rng, K + R, cols, offs, eb, C, R, K)
            ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
            for direct in (False, True):
                c, b, f, ov = ebic.eval_fitness(m, cols, offs, acols, aoffs, abm,
                                                negative=negative, direct=direct,
                                                want_bitmaps=True, want_overlaps=True)
                assert np.array_equal(c, ec) and np.array_equal(b, eb)
                assert np.array_equal(f, ef)
                if K:
                    assert np.array_equal(ov, eov)
            # the bench's form: no bitmaps, no overlaps (members sharing no column skipped)
            c, b, f, ov = ebic.eval_fitness(m, cols, offs, acols, aoffs, abm, negative=negative)
            assert b is None and ov is None
            assert np.array_equal(c, ec) and np.array_equal(f, ef)


def test_without_pair_table_is_the_two_calls(ebic):
    rng = np.random.default_rng(4)
    R, C = 3000, 30
    X = random_matrix(rng, R, C)
    cols, offs = synth.make_population(8, 200, C, 1, 10)
    ec, eb = oracle.eval_population(X, cols, offs)
    acols, aoffs, abm = make_archive(rng, 9, cols, offs, eb, C, R, 16)
    ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
    with ebic.Matrix(X) as m:
        c, _, f, _ = ebic.eval_fitness(m, cols, offs, acols, aoffs, abm)
    assert np.array_equal(c, ec) and np.array_equal(f, ef)


def test_long_candidates_sparse_and_dense_ranges(ebic):
    """Planted trend rows make long candidates (up to 64 columns) match a few rows in some
    4,096-row ranges (the compacted path) while short ones match most rows (the dense path)."""
    rng = np.random.default_rng(12)
    R, C = 20000, 64
    X = rng.random((R, C)).astype(np.float32)
    order = rng.permutation(C)
    rows = rng.choice(R, size=300, replace=False)
    X[np.ix_(rows, order)] = np.sort(rng.random((300, C)), axis=1).astype(np.float32)
    lists = [list(order[:L]) for L in (2, 5, 16, 40, 64)]
    lists += [list(order[::-1][:L]) for L in (3, 64)]
    c2, o2 = synth.make_population(5, 120, C, 1, 64)
    lists += [list(c2[o2[i]:o2[i + 1]]) for i in range(len(o2) - 1)]
    cols, offs = synth.population_from_lists(lists)
    for negative in (False, True):
        ec, eb = oracle.eval_population(X, cols, offs, negative=negative)
        acols, aoffs, abm = make_archive(rng, 3, cols, offs, eb, C, R, 24)
        ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
        with ebic.Matrix(X) as m:
            m.build_pairs()
            c, b, f, ov = ebic.eval_fitness(m, cols, offs, acols, aoffs, abm, negative=negative,
                                            want_bitmaps=True, want_overlaps=True)
            assert np.array_equal(c, ec) and np.array_equal(b, eb)
            assert np.array_equal(f, ef) and np.array_equal(ov, eov)


def test_device_resident_inputs_and_outputs(ebic):
    import torch
    rng = np.random.default_rng(21)
    R, C = 7000, 48
    X = random_matrix(rng, R, C)
    cols, offs = synth.make_population(6, 300, C, 2, 16)
    ec, eb = oracle.eval_population(X, cols, offs)
    acols, aoffs, abm = make_archive(rng, 5, cols, offs, eb, C, R, 20)
    ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
    n, K = len(offs) - 1, len(aoffs) - 1
    with ebic.Matrix(torch.from_numpy(X).cuda()) as m:
        m.build_pairs()
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        bm = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
        fit = torch.zeros(n, dtype=torch.int64, device="cuda")
        ov = torch.zeros((n, K), dtype=torch.int32, device="cuda")
        rc = ebic.ebic_eval_fitness(m.handle, dev_tensor(cols), dev_tensor(offs), n, 0,
                                    dev_tensor(acols), dev_tensor(aoffs), dev_tensor(abm), K,
                                    cnt, bm, fit, ov)
        assert rc == ebic.EBIC_OK
        assert m.status() == ebic.EBIC_OK
        assert np.array_equal(host(cnt, np.uint32), ec)
        assert np.array_equal(host(bm, np.uint32), eb)
        assert np.array_equal(host(fit, np.uint64), ef)
        assert np.array_equal(host(ov, np.uint32), eov)
        # the same call twice in a row on the same buffers gives the same results
        rc = ebic.ebic_eval_fitness(m.handle, dev_tensor(cols), dev_tensor(offs), n, 0,
                                    dev_tensor(acols), dev_tensor(aoffs), dev_tensor(abm), K,
                                    cnt, None, fit, None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        assert np.array_equal(host(cnt, np.uint32), ec)
        assert np.array_equal(host(fit, np.uint64), ef)


def test_invalid_lists_rejected(ebic):
    import torch
    rng = np.random.default_rng(2)
    R, C = 500, 10
    X = random_matrix(rng, R, C)
    good_c, good_o = synth.population_from_lists([[0, 1], [2, 3, 4]])
    bad_c, bad_o = synth.population_from_lists([[0, 1], [2, 2]])     # repeated column
    abm = synth.random_bitmaps(1, 2, R)
    with ebic.Matrix(X) as m:
        m.build_pairs()
        with pytest.raises(ebic.EbicError) as ei:
            ebic.eval_fitness(m, bad_c, bad_o, good_c, good_o, abm)
        assert ei.value.code == ebic.EBIC_ERR_INVALID_ARG
        with pytest.raises(ebic.EbicError) as ei:
            ebic.eval_fitness(m, good_c, good_o, bad_c, bad_o, abm)
        assert ei.value.code == ebic.EBIC_ERR_INVALID_ARG
        # device-resident lists: checked by the preparation kernel, reported as status
        n = 2
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        fit = torch.zeros(n, dtype=torch.int64, device="cuda")
        far_c, far_o = synth.population_from_lists([[0, 1], [3, C + 7]])  # column out of range
        gap_c = good_c.copy()
        gap_o = np.array([0, 2, 1], dtype=np.uint32)                        # offsets go backwards
        for cc, oo, ac, ao in ((bad_c, bad_o, good_c, good_o), (good_c, good_o, bad_c, bad_o),
                               (good_c, good_o, far_c, far_o), (good_c, good_o, gap_c, gap_o)):
            rc = ebic.ebic_eval_fitness(m.handle, dev_tensor(cc), dev_tensor(oo), n, 0,
                                        dev_tensor(ac), dev_tensor(ao), dev_tensor(abm), 2,
                                        cnt, None, fit, None)
            assert rc == ebic.EBIC_OK
            assert m.status() == ebic.EBIC_ERR_INVALID_ARG
        # the matrix stays usable
        ec, eb = oracle.eval_population(X, good_c, good_o)
        ef, _ = oracle.fitness(R, good_c, good_o, ec, eb, good_c, good_o, abm)
        c, _, f, _ = ebic.eval_fitness(m, good_c, good_o, good_c, good_o, abm)
        assert np.array_equal(c, ec) and np.array_equal(f, ef)


def test_fused_route_back_to_back_calls(ebic):
    """The fused route makes three kernel launches per call (preparation, pair pass, finalize);
    40 calls queued back to back on one stream (stream-ordered scratch memory reused from call
    to call, none of it zeroed by the host) on alternating populations and archives all give
    the oracle's results."""
    import torch
    rng = np.random.default_rng(33)
    R, C = 12000, 40
    X = random_matrix(rng, R, C)
    pops = []
    for k in range(2):
        cols, offs = synth.make_population(50 + k, 400 + 37 * k, C, 2, 14)
        ec, eb = oracle.eval_population(X, cols, offs)
        acols, aoffs, abm = make_archive(rng, 60 + k, cols, offs, eb, C, R, 12 + 8 * k)
        ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
        pops.append((cols, offs, acols, aoffs, abm, ec, ef))
    with ebic.Matrix(torch.from_numpy(X).cuda()) as m:
        m.build_pairs()
        dev = [tuple(dev_tensor(a) for a in p[:5]) for p in pops]
        outs = []
        for k in range(2):
            n = len(pops[k][1]) - 1
            outs.append((torch.zeros(n, dtype=torch.int32, device="cuda"),
                         torch.zeros(n, dtype=torch.int64, device="cuda")))
        before = ebic.ebic_launch_count()
        rc = ebic.ebic_eval_fitness(m.handle, *dev[0][:2], len(pops[0][1]) - 1, 0, *dev[0][2:],
                                    len(pops[0][3]) - 1, outs[0][0], None, outs[0][1], None)
        assert rc == ebic.EBIC_OK
        assert ebic.ebic_launch_count() - before == 3
        for it in range(40):
            k = it % 2
            cnt, fit = outs[k]
            cnt.zero_()
            fit.zero_()
            rc = ebic.ebic_eval_fitness(m.handle, *dev[k][:2], len(pops[k][1]) - 1, 0,
                                        *dev[k][2:], len(pops[k][3]) - 1, cnt, None, fit, None)
            assert rc == ebic.EBIC_OK
            if it >= 38:
                assert m.status() == ebic.EBIC_OK
                assert np.array_equal(host(cnt, np.uint32), pops[k][5])
                assert np.array_equal(host(fit, np.uint64), pops[k][6])


def test_config3_full_size_sampled(ebic):
    """436,444 rows in the bench's launch configuration (device inputs, no bitmaps, no
    overlaps, 20-member archive): 40 sampled candidates' counts and fitness recomputed by the
    oracle (a candidate's fitness depends only on it and the archive)."""
    import torch
    ds, cols, offs = synth.config3()
    X = ds.X
    R = X.shape[0]
    n = len(offs) - 1
    rng = np.random.default_rng(8)
    aidx = rng.choice(n, size=20, replace=False)
    acols, aoffs = synth.population_from_lists([list(cols[offs[i]:offs[i + 1]]) for i in aidx])
    _, abm = oracle.eval_population(X, acols, aoffs)
    with ebic.Matrix(torch.from_numpy(X).cuda(), exclude_missing=True) as m:
        m.build_pairs()
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        fit = torch.zeros(n, dtype=torch.int64, device="cuda")
        rc = ebic.ebic_eval_fitness(m.handle, dev_tensor(cols), dev_tensor(offs), n, 0,
                                    dev_tensor(acols), dev_tensor(aoffs), dev_tensor(abm), 20,
                                    cnt, None, fit, None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        got_c, got_f = host(cnt, np.uint32), host(fit, np.uint64)
    idx = rng.choice(n, size=40, replace=False)
    sc, so = synth.population_from_lists([list(cols[offs[i]:offs[i + 1]]) for i in idx])
    ec, eb = oracle.eval_population(X, sc, so)
    ef, _ = oracle.fitness(R, sc, so, ec, eb, acols, aoffs, abm)
    assert np.array_equal(got_c[idx], ec)
    assert np.array_equal(got_f[idx], ef)


def test_pinned_host_buffers_read_and_written_in_place(ebic):
    """Pinned host lists, archive and outputs (the kernels read and write them over the host
    link, no copies): the oracle's counts and fitness; an invalid pinned list is rejected with
    no deferred status left behind; device outputs with pinned inputs work too."""
    import torch
    rng = np.random.default_rng(41)
    R, C = 9000, 48
    X = random_matrix(rng, R, C)
    cols, offs = synth.make_population(42, 333, C, 2, 16)
    ec, eb = oracle.eval_population(X, cols, offs)
    acols, aoffs, abm = make_archive(rng, 43, cols, offs, eb, C, R, 11)
    ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
    n, K = len(offs) - 1, len(aoffs) - 1

    def pinned(a):
        view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
        return torch.from_numpy(np.ascontiguousarray(a).view(view)).pin_memory()

    with ebic.Matrix(torch.from_numpy(X).cuda()) as m:
        m.build_pairs()
        hc, ho, hac, hao, hab = pinned(cols), pinned(offs), pinned(acols), pinned(aoffs), pinned(abm)
        cnt = torch.full((n,), -1, dtype=torch.int32).pin_memory()
        fit = torch.full((n,), -1, dtype=torch.int64).pin_memory()
        for _ in range(3):
            rc = ebic.ebic_eval_fitness(m.handle, hc, ho, n, 0, hac, hao, hab, K, cnt, None, fit,
                                        None)
            assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
            assert np.array_equal(cnt.numpy().view(np.uint32), ec)
            assert np.array_equal(fit.numpy().view(np.uint64), ef)
        # device outputs, pinned inputs (asynchronous call)
        dcnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        dfit = torch.zeros(n, dtype=torch.int64, device="cuda")
        rc = ebic.ebic_eval_fitness(m.handle, hc, ho, n, 0, hac, hao, hab, K, dcnt, None, dfit,
                                    None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        assert np.array_equal(host(dcnt, np.uint32), ec)
        assert np.array_equal(host(dfit, np.uint64), ef)
        # a repeated column in a pinned list
        bad = cols.copy()
        bad[offs[5] + 1] = bad[offs[5]]
        rc = ebic.ebic_eval_fitness(m.handle, pinned(bad), ho, n, 0, hac, hao, hab, K, cnt, None,
                                    fit, None)
        assert rc == ebic.EBIC_ERR_INVALID_ARG
        assert m.status() == ebic.EBIC_OK
        # the same with the archive on the device: still the host check's verdict, no deferred
        # status; then the device archive with the good pinned list
        dac, dao, dab = dev_tensor(acols), dev_tensor(aoffs), dev_tensor(abm)
        rc = ebic.ebic_eval_fitness(m.handle, pinned(bad), ho, n, 0, dac, dao, dab, K, cnt, None,
                                    fit, None)
        assert rc == ebic.EBIC_ERR_INVALID_ARG
        assert m.status() == ebic.EBIC_OK
        rc = ebic.ebic_eval_fitness(m.handle, hc, ho, n, 0, dac, dao, dab, K, cnt, None, fit, None)
        assert rc == ebic.EBIC_OK
        assert np.array_equal(fit.numpy().view(np.uint64), ef)
        rc = ebic.ebic_eval_fitness(m.handle, hc, ho, n, 0, hac, hao, hab, K, cnt, None, fit, None)
        assert rc == ebic.EBIC_OK
        assert np.array_equal(fit.numpy().view(np.uint64), ef)


def test_c_and_ctypes_marshalling_give_the_same_scores(ebic):
    # the per-generation call through the C marshalling module and through ctypes, on pinned host
    # and device buffers: identical counts and fitness
    import torch
    if ebic._fast is None:
        pytest.skip("the C marshalling module is not built here")
    ds = synth.make_dataset(41, 6000, 30, kind="beta", planted=[(900, 6, False)], nan_frac=0.01)
    cols, offs = synth.make_population(42, 300, 30, 2, 12)
    acols, aoffs = synth.make_population(43, 5, 30, 3, 8)
    with ebic.Matrix(ds.X, exclude_missing=True) as m:
        m.build_pairs()
        _, abm = ebic.eval_population(m, acols, aoffs)
        got = []
        for use_c in (True, False):
            saved = ebic._fast
            if not use_c:
                ebic._fast = None
            try:
                hc = torch.from_numpy(cols.view(np.int16)).pin_memory()
                ho = torch.from_numpy(offs.view(np.int32)).pin_memory()
                cnt = torch.zeros(len(offs) - 1, dtype=torch.int32).pin_memory()
                fit = torch.zeros(len(offs) - 1, dtype=torch.int64).pin_memory()
                rc = ebic.ebic_eval_fitness(m.handle, hc, ho, len(offs) - 1, 0, acols, aoffs, abm,
                                            len(aoffs) - 1, cnt, None, fit, None,
                                            torch.cuda.current_stream())
                assert rc == 0, ebic.ebic_last_error()
                got.append((cnt.numpy().copy(), fit.numpy().copy()))
            finally:
                ebic._fast = saved
        assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])

