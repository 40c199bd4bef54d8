"""The route the product takes, at the workloads' real sizes, against the oracle bit for bit.

Every run that builds a pair table -- ebic_run, the batch, the server, the bench -- scores on the
pair-table pass, with the archive overlaps fused in (ebic_eval_fitness). This file checks that
route against the oracle (counts, bitmaps, fitness and overlaps; arXiv 1807.09932, Methods,
"Handling missing values" for the rule, "Support for Big Data" for the sizes) on:
  * the expression-shaped workload in full: 20,000 x 200, 1% NaN with exclusion on, negative
    trends on, 1,600 candidates of 2-20 columns, every candidate;
  * the methylation-shaped workload in full with negative trends: 436,444 x 64, every one of the
    1,600 candidates, on the fused route in the bench's launch form and on the pair route;
  * the largest matrix of the batched workload (144,826 x 221) with its largest population
    (3,095 candidates of 2-64 columns) through the captured batch graph, with an archive;
  * the two largest served runs (376,987 x 184 and 326,405 x 128) through the server's GPU
    backend, fitness inside the batch.
"""
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
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32,
            np.dtype(np.uint64): np.int64}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def _host(t, dtype):
    return t.cpu().numpy().view(dtype)


def _archive(ds, cols, offs, counts, k_pop=10, k_planted=10):
    """A converged run's archive: the planted biclusters' column orders (as many as there are,
    up to k_planted) and the k_pop candidates with the most matched rows."""
    lists = [list(p.cols) for p in ds.planted[:k_planted]]
    top = np.argsort(-counts.astype(np.int64), kind="stable")[:k_pop]
    lists += [list(cols[offs[i]:offs[i + 1]]) for i in top]
    return synth.population_from_lists(lists)


def test_config2_full_pair_and_fused_routes(ebic):
    import torch
    ds, cols, offs = synth.config2()
    X = ds.X
    R = X.shape[0]
    n = len(offs) - 1
    ec, eb = oracle.eval_population(X, cols, offs, negative=True)
    acols, aoffs = _archive(ds, cols, offs, ec)
    _, abm = oracle.eval_population(X, acols, aoffs, negative=True)
    K = len(aoffs) - 1
    ef, eov = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm)
    with ebic.Matrix(torch.from_numpy(X).cuda(), exclude_missing=True) as m:
        m.build_pairs()
        # everything out: counts, bitmaps, fitness and the full overlap matrix
        c, b, f, ov = ebic.eval_fitness(m, cols, offs, acols, aoffs, abm, negative=True,
                                        want_bitmaps=True, want_overlaps=True)
        assert np.array_equal(c, ec) and np.array_equal(b, eb)
        assert np.array_equal(f, ef) and np.array_equal(ov, eov)
        # the bench's form: device buffers, counts and fitness only
        cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        fit = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        rc = ebic.ebic_eval_fitness(m.handle, _dev(cols), _dev(offs), n,
                                    ebic.EBIC_NEGATIVE_TRENDS, _dev(acols), _dev(aoffs),
                                    _dev(abm), K, cnt, None, fit, None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        assert np.array_equal(_host(cnt, np.uint32), ec)
        assert np.array_equal(_host(fit, np.uint64), ef)
        # the pair route of ebic_eval_population, both trend options
        for neg in (False, True):
            pc, pb = ebic.eval_population(m, cols, offs, negative=neg)
            xc, xb = (ec, eb) if neg else oracle.eval_population(X, cols, offs, negative=False)
            assert np.array_equal(pc, xc) and np.array_equal(pb, xb)


def test_config3_full_with_negative_trends(ebic):
    import torch
    ds, cols, offs = synth.config3()
    X = ds.X
    R = X.shape[0]
    n = len(offs) - 1
    ec, eb = oracle.eval_population(X, cols, offs, negative=True)
    acols, aoffs = _archive(ds, cols, offs, ec)
    _, abm = oracle.eval_population(X, acols, aoffs, negative=True)
    K = len(aoffs) - 1
    ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm, want_overlaps=False)
    with ebic.Matrix(torch.from_numpy(X).cuda(), exclude_missing=True) as m:
        m.build_pairs()
        dcols, doffs = _dev(cols), _dev(offs)
        cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        fit = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        rc = ebic.ebic_eval_fitness(m.handle, dcols, doffs, n, ebic.EBIC_NEGATIVE_TRENDS,
                                    _dev(acols), _dev(aoffs), _dev(abm), K, cnt, None, fit, None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        assert np.array_equal(_host(cnt, np.uint32), ec)
        assert np.array_equal(_host(fit, np.uint64), ef)
        # pair route, counts and bitmaps of every candidate
        bm = torch.full((n, m.words), -1, dtype=torch.int32, device="cuda")
        cnt.fill_(-1)
        ebic.eval_population(m, dcols, doffs, negative=True, counts=cnt, bitmaps=bm)
        assert m.status() == ebic.EBIC_OK
        assert np.array_equal(_host(cnt, np.uint32), ec)
        assert np.array_equal(_host(bm, np.uint32), eb)


def test_config4_largest_matrix_through_the_batch_graph(ebic):
    import torch
    specs, pops = synth.config4_specs()
    d = max(range(len(specs)), key=lambda i: specs[i]["rows"])
    ds = synth.dataset_from_spec(specs[d])
    X = ds.X
    R, C = X.shape
    mine = [p for p in pops if p["dataset"] == d]
    big = max(mine, key=lambda p: p["n_cand"])
    small = min(mine, key=lambda p: p["n_cand"])
    cols, offs = synth.make_population(big["seed"], big["n_cand"], C, big["lmin"], big["lmax"])
    assert int(np.diff(offs).max()) > 32   # long candidates are in it
    scols, soffs = synth.make_population(small["seed"], small["n_cand"], C, small["lmin"],
                                         small["lmax"])
    n, ns = len(offs) - 1, len(soffs) - 1
    ec, eb = oracle.eval_population(X, cols, offs)
    acols, aoffs = _archive(ds, cols, offs, ec, k_pop=15, k_planted=5)
    _, abm = oracle.eval_population(X, acols, aoffs)
    K = len(aoffs) - 1
    ef, _ = oracle.fitness(R, cols, offs, ec, eb, acols, aoffs, abm, want_overlaps=False)
    sc, sb = oracle.eval_population(X, scols, soffs, negative=True)
    with ebic.Matrix(X) as m:
        m.build_pairs()
        cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        fit = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        scnt = torch.full((ns,), -1, dtype=torch.int32, device="cuda")
        sbm = torch.full((ns, m.words), -1, dtype=torch.int32, device="cuda")
        items = [(m.handle, _dev(cols), _dev(offs), n, 0, cnt, None, _dev(acols), _dev(aoffs),
                  _dev(abm), K, fit),
                 (m.handle, _dev(scols), _dev(soffs), ns, ebic.EBIC_NEGATIVE_TRENDS, scnt, sbm)]
        arr = ebic.make_requests(items)
        b = ebic.ebic_batch_create(8)
        try:
            for _ in range(2):   # capture, then replay
                assert ebic.ebic_batch_run(b, arr, len(items)) == ebic.EBIC_OK, \
                    ebic.ebic_last_error()
                rc, st = ebic.ebic_batch_status(b, len(items))
                assert rc == ebic.EBIC_OK and not any(st)
                assert np.array_equal(_host(cnt, np.uint32), ec)
                assert np.array_equal(_host(fit, np.uint64), ef)
                assert np.array_equal(_host(scnt, np.uint32), sc)
                assert np.array_equal(_host(sbm, np.uint32), sb)
                for t in (cnt, fit, scnt, sbm):
                    t.fill_(-1)
        finally:
            ebic.ebic_batch_free(b)


def test_config5_large_served_runs_equal_oracle(ebic):
    """The two largest served runs (376,987 x 184 and 326,405 x 128), two requests each arriving
    at once: batches hold one request of each run, so the batch graph's pair pass computes the
    fitness against each run's resident archive."""
    from paper_1807_09932_gb300 import serve
    runs = sorted(synth.config5_specs(), key=lambda r: -r["rows"])[:2]
    assert min(r["rows"] for r in runs) >= 200000
    be = serve.GpuBackend(max_batch=8, max_inflight=2, pair_budget=4 << 30)
    try:
        srv = serve.Server(be, hbm_budget=24 << 30, max_batch=8, max_inflight=2)
        data, arr = {}, []
        for i, spec in enumerate(runs):
            ds = synth.dataset_from_spec(spec)
            X = ds.X
            C = X.shape[1]
            pool_c, pool_o = synth.make_population(spec["seed"] + 1, 1600, C, 2, 16)
            pc, _ = oracle.eval_population(X, pool_c, pool_o)
            acols, aoffs = _archive(ds, pool_c, pool_o, pc)
            _, abm = oracle.eval_population(X, acols, aoffs)
            data[i] = (X, acols, aoffs, abm)
            srv.add_run(serve.RunSpec(run_id=i, X=X, max_cand=1600, max_len=16,
                                      archive_cols=acols, archive_offsets=aoffs))
            for k in range(2):
                c, o = synth.make_population(spec["seed"] + 10 + k, 1600, C, 2, 16)
                arr.append(serve.Request(run_id=i, cols=c, offsets=o, t_arrival=0.0,
                                         flags=ebic.EBIC_NEGATIVE_TRENDS if k == 1 else 0))
        st = serve.drive(srv, arr, {i: data[i][0].shape[0] for i in data})
        assert st["requests"] == 4
        assert all(be.runs[i]["pairs"] for i in data)
        for r in srv.done:
            X, acols, aoffs, abm = data[r.run_id]
            ec, eb = oracle.eval_population(X, r.cols, r.offsets, negative=bool(r.flags))
            ef, _ = oracle.fitness(X.shape[0], r.cols, r.offsets, ec, eb, acols, aoffs, abm,
                                   want_overlaps=False)
            assert np.array_equal(r.counts, ec)
            assert np.array_equal(r.fitness, ef)
    finally:
        be.close()
