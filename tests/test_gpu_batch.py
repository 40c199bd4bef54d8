"""Batched evaluation (one persistent launch, direct and CUDA-graph replay) gives byte-identical
results to scoring each request alone, for mixed rank layouts, tile heights, negative options,
uneven candidate lengths (2-64) and uneven matrix sizes; a bad request fails alone."""
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


def _dev(a):
    import torch
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


# (rows, cols, tile) -> 8-bit ranks with 1/2/4-slab tiles and 16-bit ranks with VEC 4/2/1
SHAPES = [(3001, 40, 4), (20011, 64, 2), (777, 100, 1), (9000, 150, 1), (4100, 300, 1),
          (2600, 500, 1), (65, 20, 0), (12000, 127, 0)]


def _matrices(ebic):
    mats = []
    for i, (R, C, tile) in enumerate(SHAPES):
        ds = synth.make_dataset(100 + i, R, C, kind="normal" if i % 2 else "beta",
                                planted=synth.planted_specs_for(100 + i, R, C), nan_frac=0.01)
        m = ebic.Matrix(ds.X)
        if tile:
            m.set_tile(tile)
        mats.append((ds, m))
    return mats


def _requests(ebic, mats, n_pop, seed):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for p in range(n_pop):
        ds, m = mats[p % len(mats)]
        C = ds.X.shape[1]
        n = int(rng.integers(1, 400))
        cols, offs = synth.make_population(seed * 1000 + p, n, C, 2, min(64, C))
        flags = ebic.EBIC_NEGATIVE_TRENDS if p % 3 == 1 else 0
        want_bm = p % 5 != 4
        cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        bm = torch.full((n, m.words), -1, dtype=torch.int32, device="cuda") if want_bm else None
        reqs.append(dict(ds=ds, m=m, cols=cols, offs=offs, dcols=_dev(cols), doffs=_dev(offs),
                         n=n, flags=flags, counts=cnt, bitmaps=bm))
    return reqs


def _alone(ebic, r):
    return ebic.eval_population(r["m"], r["cols"], r["offs"],
                                negative=bool(r["flags"]), want_bitmaps=r["bitmaps"] is not None)


def _items(reqs):
    return [(r["m"].handle, r["dcols"], r["doffs"], r["n"], r["flags"], r["counts"],
             r["bitmaps"]) for r in reqs]


def _check_against_alone(ebic, reqs):
    for r in reqs:
        c, b = _alone(ebic, r)
        assert np.array_equal(r["counts"].cpu().numpy().view(np.uint32), c)
        if r["bitmaps"] is not None:
            assert np.array_equal(r["bitmaps"].cpu().numpy().view(np.uint32), b)


def test_batch_equals_alone(ebic):
    import torch
    mats = _matrices(ebic)
    reqs = _requests(ebic, mats, 24, seed=1)
    arr = ebic.make_requests(_items(reqs))
    assert ebic.ebic_eval_batch(arr, len(reqs)) == ebic.EBIC_OK, ebic.ebic_last_error()
    torch.cuda.synchronize()
    for _, m in mats:
        assert m.status() == ebic.EBIC_OK
    _check_against_alone(ebic, reqs)
    # and the oracle, on a few requests
    for r in reqs[:6]:
        c, b = oracle.eval_population(r["ds"].X, r["cols"], r["offs"],
                                      negative=bool(r["flags"]))
        assert np.array_equal(r["counts"].cpu().numpy().view(np.uint32), c)


def test_graph_replay_with_changing_compositions(ebic):
    import torch
    mats = _matrices(ebic)
    b = ebic.ebic_batch_create(64)
    try:
        for seed, n_pop in ((2, 30), (3, 7), (4, 64), (5, 1)):
            reqs = _requests(ebic, mats, n_pop, seed=seed)
            arr = ebic.make_requests(_items(reqs))
            assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK, ebic.ebic_last_error()
            rc, st = ebic.ebic_batch_status(b, len(reqs))
            assert rc == ebic.EBIC_OK and not any(st)
            _check_against_alone(ebic, reqs)
        # replaying the same composition twice gives the same bytes
        reqs = _requests(ebic, mats, 12, seed=6)
        arr = ebic.make_requests(_items(reqs))
        ebic.ebic_batch_run(b, arr, len(reqs))
        first = [r["counts"].clone() for r in reqs]
        ebic.ebic_batch_run(b, arr, len(reqs))
        torch.cuda.synchronize()
        assert all(torch.equal(a, r["counts"]) for a, r in zip(first, reqs))
    finally:
        ebic.ebic_batch_free(b)


def test_bad_request_fails_alone(ebic):
    mats = _matrices(ebic)
    reqs = _requests(ebic, mats, 6, seed=7)
    bad = reqs[2]
    C = bad["ds"].X.shape[1]
    cols = bad["cols"].copy()
    cols[0] = C  # out of range
    bad["dcols"] = _dev(cols)
    b = ebic.ebic_batch_create(8)
    try:
        arr = ebic.make_requests(_items(reqs))
        assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK
        rc, st = ebic.ebic_batch_status(b, len(reqs))
        assert rc == ebic.EBIC_ERR_INVALID_ARG
        assert st[2] != 0 and all(s == 0 for i, s in enumerate(st) if i != 2)
        assert bad["m"].status() == ebic.EBIC_ERR_INVALID_ARG
        assert int(bad["counts"].abs().sum()) == 0
        _check_against_alone(ebic, [r for i, r in enumerate(reqs) if i != 2])
    finally:
        ebic.ebic_batch_free(b)
        for _, m in mats:
            m.status()


def _with_pairs(ebic, mats, which):
    for i, (_, m) in enumerate(mats):
        if which(i):
            m.build_pairs()


def _check_against_direct(ebic, reqs):
    """The rank-code evaluator, whatever the matrix holds."""
    for r in reqs:
        c, b = ebic.eval_population(r["m"], r["cols"], r["offs"], negative=bool(r["flags"]),
                                    want_bitmaps=r["bitmaps"] is not None, direct=True)
        assert np.array_equal(r["counts"].cpu().numpy().view(np.uint32), c)
        if r["bitmaps"] is not None:
            assert np.array_equal(r["bitmaps"].cpu().numpy().view(np.uint32), b)


def test_batch_with_pair_tables(ebic):
    """Requests on matrices with a pair table run on the batched pair pass, the others on the
    rank-code pass, in one batch; both give the rank-code evaluator's bytes and the oracle's."""
    import torch
    mats = _matrices(ebic)
    _with_pairs(ebic, mats, lambda i: i % 2 == 0)
    reqs = _requests(ebic, mats, 32, seed=11)
    arr = ebic.make_requests(_items(reqs))
    assert ebic.ebic_eval_batch(arr, len(reqs)) == ebic.EBIC_OK, ebic.ebic_last_error()
    torch.cuda.synchronize()
    for _, m in mats:
        assert m.status() == ebic.EBIC_OK
    _check_against_direct(ebic, reqs)
    for r in reqs[:8]:
        c, _ = oracle.eval_population(r["ds"].X, r["cols"], r["offs"], negative=bool(r["flags"]))
        assert np.array_equal(r["counts"].cpu().numpy().view(np.uint32), c)
    # the captured graph, with compositions of pair and rank-code requests
    b = ebic.ebic_batch_create(64)
    try:
        for seed, n_pop in ((12, 40), (13, 3), (14, 64)):
            reqs = _requests(ebic, mats, n_pop, seed=seed)
            arr = ebic.make_requests(_items(reqs))
            assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK, ebic.ebic_last_error()
            rc, st = ebic.ebic_batch_status(b, len(reqs))
            assert rc == ebic.EBIC_OK and not any(st)
            _check_against_direct(ebic, reqs)
        # a bad request on a matrix with a table fails alone
        reqs = _requests(ebic, mats, 6, seed=15)
        bad = reqs[0]  # mats[0] has a table
        cols = bad["cols"].copy()
        cols[0] = bad["ds"].X.shape[1]
        bad["dcols"] = _dev(cols)
        arr = ebic.make_requests(_items(reqs))
        assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK
        rc, st = ebic.ebic_batch_status(b, len(reqs))
        assert rc == ebic.EBIC_ERR_INVALID_ARG
        assert st[0] != 0 and all(s == 0 for i, s in enumerate(st) if i != 0)
        assert bad["m"].status() == ebic.EBIC_ERR_INVALID_ARG
        assert int(bad["counts"].abs().sum()) == 0
        _check_against_direct(ebic, reqs[1:])
    finally:
        ebic.ebic_batch_free(b)


def _with_archives(ebic, reqs, seed, sizes=(0, 1, 7, 20, 64, 33)):
    """Give every request an archive (sizes cycled; about half the members are candidates of the
    request, so they overlap it and share its columns, the rest random column sets with random
    bitmaps), a fitness output, and the oracle's expected fitness."""
    import torch
    rng = np.random.default_rng(seed)
    for k, r in enumerate(reqs):
        X = r["ds"].X
        R, C = X.shape
        K = sizes[k % len(sizes)]
        n = r["n"]
        cols, offs = r["cols"], r["offs"]
        ec, eb = oracle.eval_population(X, cols, offs, negative=bool(r["flags"]))
        k_pop = min(K // 2, n)
        idx = rng.choice(n, size=k_pop, replace=False)
        lists = [list(cols[offs[i]:offs[i + 1]]) for i in idx]
        lists += [list(rng.choice(C, int(rng.integers(1, min(C, 8) + 1)), replace=False))
                  for _ in range(K - k_pop)]
        acols, aoffs = synth.population_from_lists(lists) if K else (
            np.zeros(0, dtype=np.uint16), np.zeros(1, dtype=np.uint32))
        abm = np.ascontiguousarray(np.concatenate(
            [eb[idx], synth.random_bitmaps(seed + k, K - k_pop, R, 0.3)]) if K else
            np.zeros((0, (R + 31) // 32), dtype=np.uint32), dtype=np.uint32)
        ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
        r.update(acols=acols, aoffs=aoffs, abm=abm, K=K, exp_counts=ec, exp_fit=ef,
                 dacols=_dev(acols) if K else None, daoffs=_dev(aoffs) if K else None,
                 dabm=_dev(abm) if K else None,
                 fit=torch.full((n,), -1, dtype=torch.int64, device="cuda"))


def _fit_items(reqs):
    return [(r["m"].handle, r["dcols"], r["doffs"], r["n"], r["flags"], r["counts"],
             r["bitmaps"], r["dacols"], r["daoffs"], r["dabm"], r["K"], r["fit"]) for r in reqs]


def _check_fitness(reqs):
    for r in reqs:
        assert np.array_equal(r["counts"].cpu().numpy().view(np.uint32), r["exp_counts"])
        assert np.array_equal(r["fit"].cpu().numpy().view(np.uint64), r["exp_fit"])


def test_batch_fitness_equals_oracle(ebic):
    """Requests with an archive get ebic_eval_fitness's fitness from the batched pass (overlaps
    fused there, 0 to 64 members, odd and even archive sizes, with and without bitmaps, both
    trend options), directly and through the captured graph, equal to the oracle's; a request
    without an archive in the same batch is unaffected; fitness on a matrix without a pair
    table is refused; a request with a bad archive list fails alone."""
    import torch
    mats = _matrices(ebic)
    _with_pairs(ebic, mats, lambda i: True)
    reqs = _requests(ebic, mats, 24, seed=31)
    _with_archives(ebic, reqs, seed=32)
    plain = _requests(ebic, mats, 3, seed=33)   # no fitness, same batch
    items = _fit_items(reqs) + _items(plain)
    arr = ebic.make_requests(items)
    assert ebic.ebic_eval_batch(arr, len(items)) == ebic.EBIC_OK, ebic.ebic_last_error()
    torch.cuda.synchronize()
    for _, m in mats:
        assert m.status() == ebic.EBIC_OK
    _check_fitness(reqs)
    _check_against_direct(ebic, [r for r in reqs if r["bitmaps"] is not None] + plain)
    b = ebic.ebic_batch_create(64)
    try:
        for seed in (34, 35):   # the graph, twice, on new compositions (scratch regrown)
            reqs = _requests(ebic, mats, 40 if seed == 34 else 64, seed=seed)
            _with_archives(ebic, reqs, seed=seed + 100, sizes=(20, 3, 64, 0, 2))
            arr = ebic.make_requests(_fit_items(reqs))
            assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK, ebic.ebic_last_error()
            rc, st = ebic.ebic_batch_status(b, len(reqs))
            assert rc == ebic.EBIC_OK and not any(st)
            _check_fitness(reqs)
        # a repeated column in one request's archive: that request fails alone
        reqs = _requests(ebic, mats, 6, seed=36)
        _with_archives(ebic, reqs, seed=136, sizes=(5,))
        bad = reqs[0]
        ac = bad["acols"].copy()
        ac[1] = ac[0]
        bad["dacols"] = _dev(ac)
        arr = ebic.make_requests(_fit_items(reqs))
        assert ebic.ebic_batch_run(b, arr, len(reqs)) == ebic.EBIC_OK
        rc, st = ebic.ebic_batch_status(b, len(reqs))
        assert rc == ebic.EBIC_ERR_INVALID_ARG
        assert st[0] != 0 and all(s == 0 for i, s in enumerate(st) if i != 0)
        assert bad["m"].status() == ebic.EBIC_ERR_INVALID_ARG
        _check_fitness(reqs[1:])
    finally:
        ebic.ebic_batch_free(b)
    # fitness needs the pair table
    ds = synth.make_dataset(7, 500, 12, kind="normal")
    with ebic.Matrix(ds.X) as m:
        cols, offs = synth.make_population(8, 10, 12, 2, 5)
        n = len(offs) - 1
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        fit = torch.zeros(n, dtype=torch.int64, device="cuda")
        arr = ebic.make_requests([(m.handle, _dev(cols), _dev(offs), n, 0, cnt, None, None, None,
                                   None, 0, fit)])
        assert ebic.ebic_eval_batch(arr, 1) == ebic.EBIC_ERR_UNSUPPORTED
