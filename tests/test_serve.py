"""Serving loop: admission by device-memory footprint, continuous batching, one request in
flight per run, latency accounting (host-only with a fake backend and clock); on the GPU every
served result equals the same request scored alone."""
import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import serve, synth

from fake_backend import FakeBackend, FakeClock


def _spec(i, rows=300, cols=12, max_cand=50):
    ds = synth.make_dataset(500 + i, rows, cols, planted=[(60, 5, False)], nan_frac=0.01)
    ac, ao = synth.population_from_lists([[0, 1], [2, 3, 4]])
    return serve.RunSpec(run_id=i, X=ds.X, max_cand=max_cand, max_len=cols,
                         archive_cols=ac, archive_offsets=ao)


def _req(run_id, t, seed, n=20, cols=12):
    c, o = synth.make_population(seed, n, cols, 2, 6)
    return serve.Request(run_id=run_id, cols=c, offsets=o, t_arrival=t)


def _drive_fake(srv, clock, be, arrivals, rows_of):
    def spin(next_arrival):
        nxt = be.next_event(srv.inflight)
        cands = [t for t in (nxt, next_arrival) if t is not None]
        if cands:
            clock.t = max(clock.t, min(cands))
    return serve.drive(srv, arrivals, rows_of, spin=spin)


def test_percentile_matches_numpy():
    v = list(np.random.default_rng(0).random(101))
    for q in (0, 50, 90, 99, 100):
        assert abs(serve.percentile(v, q) - np.percentile(v, q)) < 1e-12


def test_admission_by_footprint():
    clock = FakeClock()
    be = FakeBackend(clock)
    specs = [_spec(i) for i in range(3)]
    need = be.footprint(specs[0])
    srv = serve.Server(be, hbm_budget=2 * need + 10)
    assert srv.add_run(specs[0]) and srv.add_run(specs[1])
    assert not srv.add_run(specs[2])          # waits for memory
    assert not srv.is_open(2) and srv.used == 2 * need
    srv.finish_run(0)                         # frees a run's memory -> the waiting run opens
    assert srv.is_open(2) and srv.used == 2 * need
    with pytest.raises(ValueError):
        serve.Server(be, hbm_budget=need - 1).add_run(specs[0])


def test_continuous_batching_and_latency_accounting():
    clock = FakeClock()
    be = FakeBackend(clock, fixed=1.0, per_eval=0.0)   # every batch takes 1 fake second
    srv = serve.Server(be, hbm_budget=1 << 40, max_batch=3, max_inflight=1)
    for i in range(5):
        srv.add_run(_spec(i))
    # five requests at t=0, one more at t=0.5 (arrives while the first batch runs)
    arr = [_req(i, 0.0, 10 + i) for i in range(5)] + [_req(0, 0.5, 99)]
    rows = {i: 300 for i in range(5)}
    st = _drive_fake(srv, clock, be, arr, rows)
    assert st["requests"] == 6
    # batch 1: runs 0,1,2 (max_batch 3); batch 2: runs 3,4 and run 0's second request, which
    # arrived during batch 1 and could only go once run 0's first request had finished
    assert be.launched == [[0, 1, 2], [3, 4, 5]]
    lat = sorted(round(r.latency, 9) for r in srv.done)
    assert lat == [1.0, 1.0, 1.0, 1.5, 2.0, 2.0]
    assert st["p50_ms"] == pytest.approx(1250.0)


def test_one_request_in_flight_per_run_and_results_exact():
    clock = FakeClock()
    be = FakeBackend(clock, fixed=0.1, per_eval=1e-8)
    srv = serve.Server(be, hbm_budget=1 << 40, max_batch=8, max_inflight=2)
    specs = [_spec(i) for i in range(3)]
    for s in specs:
        srv.add_run(s)
    arr = [_req(i % 3, 0.01 * i, 40 + i) for i in range(12)]
    st = _drive_fake(srv, clock, be, arr, {i: 300 for i in range(3)})
    assert st["requests"] == 12
    for batch in be.launched:  # never two requests of one run in a batch
        runs = [arr[rid].run_id for rid in batch]
        assert len(runs) == len(set(runs))
    for r in srv.done:
        X = specs[r.run_id].X
        c, _ = oracle.eval_population(X, r.cols, r.offsets)
        assert np.array_equal(r.counts, c)
        assert r.t_done >= r.t_launch >= r.t_arrival


def test_failed_launch_frees_its_runs():
    """A batch whose launch raises never ran: the error reaches the caller, its runs are not left
    marked busy, and the same requests go through on the next pump."""
    clock = FakeClock()
    be = FakeBackend(clock, fixed=0.1, per_eval=0.0)
    srv = serve.Server(be, hbm_budget=1 << 40, max_batch=4, max_inflight=1)
    for i in range(2):
        srv.add_run(_spec(i))
    real, calls = be.launch, []

    def flaky(reqs):
        calls.append(len(reqs))
        if len(calls) == 1:
            raise RuntimeError("launch failed")
        return real(reqs)

    be.launch = flaky
    reqs = [_req(0, 0.0, 70), _req(1, 0.0, 71)]
    for r in reqs:
        srv.submit(r)
    with pytest.raises(RuntimeError):
        srv.pump()
    assert not srv.busy_runs and not srv.inflight and not srv.queue
    for r in reqs:  # the failed batch's requests are the caller's to send again
        srv.submit(r)
    srv.pump()
    assert len(srv.inflight) == 1 and srv.busy_runs == {0, 1}
    clock.t = 1.0
    done = srv.pump()
    assert sorted(r.run_id for r in done) == [0, 1] and not srv.busy_runs


@pytest.mark.gpu
@pytest.mark.parametrize("pair_budget,spacing", [(0, 0.0005), (1 << 30, 0.0005), (1 << 30, 0.0)])
def test_served_results_equal_alone(pair_budget, spacing):
    """Served counts and fitness equal the per-population calls' and the oracle's counts, with
    runs on the rank-code pass (fitness per request) and on pair tables (fitness inside the
    batch, or the fused call for a batch of one); spacing 0: every request arrives at once, so
    batches hold many requests."""
    import torch
    from paper_1807_09932_gb300 import ebic
    be = serve.GpuBackend(max_batch=16, max_inflight=2, pair_budget=pair_budget)
    try:
        srv = serve.Server(be, hbm_budget=8 << 30, max_batch=16, max_inflight=2)
        specs = []
        for i in range(6):
            R, C = (3000 + 977 * i, [30, 64, 127, 150, 300, 40][i])
            ds = synth.make_dataset(700 + i, R, C, planted=synth.planted_specs_for(700 + i, R, C),
                                    nan_frac=0.01)
            pool_c, pool_o = synth.make_population(800 + i, 200, C, 2, 8)
            cnt, _ = oracle.eval_population(ds.X, pool_c, pool_o)
            top = np.argsort(-cnt.astype(np.int64), kind="stable")[:5]
            ac, ao = synth.population_from_lists(
                [list(pool_c[pool_o[j]:pool_o[j + 1]]) for j in top])
            specs.append(serve.RunSpec(run_id=i, X=ds.X, max_cand=400, max_len=min(C, 64),
                                       archive_cols=ac, archive_offsets=ao))
            srv.add_run(specs[-1])
        arr = []
        for k in range(30):
            i = k % 6
            C = specs[i].X.shape[1]
            c, o = synth.make_population(900 + k, int(50 + 10 * k), C, 2, min(C, 64))
            arr.append(serve.Request(run_id=i, cols=c, offsets=o, t_arrival=spacing * k,
                                     flags=ebic.EBIC_NEGATIVE_TRENDS if k % 4 == 3 else 0))
        st = serve.drive(srv, arr, {s.run_id: s.X.shape[0] for s in specs})
        assert st["requests"] == 30
        for r in srv.done:
            s = specs[r.run_id]
            m = be.runs[r.run_id]["m"]
            c, b = ebic.eval_population(m, r.cols, r.offsets, negative=bool(r.flags))
            _, abm = ebic.eval_population(m, s.archive_cols, s.archive_offsets)
            f, _ = ebic.fitness(m, r.cols, r.offsets, c, b, s.archive_cols, s.archive_offsets,
                                abm)
            assert np.array_equal(r.counts, c)
            assert np.array_equal(r.fitness, f)
            ec, eb = oracle.eval_population(s.X, r.cols, r.offsets, negative=bool(r.flags))
            assert np.array_equal(r.counts, ec)
        # the plain arm (pinned lists and outputs read and written in place) agrees
        stream = torch.cuda.Stream()
        for r in srv.done[:12]:
            p = serve.Request(run_id=r.run_id, cols=r.cols, offsets=r.offsets, t_arrival=0.0,
                              flags=r.flags)
            be.plain(p, stream)
            assert np.array_equal(p.counts, r.counts)
            assert np.array_equal(p.fitness, r.fitness)
    finally:
        be.close()


def test_batch_staging_layout_packs_every_list_on_aligned_offsets():
    """The GPU backend's host staging (no device needed): each request's columns and offsets sit
    on 256-byte boundaries without overlap, unpack to the request's own lists, and the outputs'
    counts and fitness slots are aligned, disjoint and sized for the request."""
    reqs = [_req(i % 3, 0.0, 40 + i, n=[1, 7, 33, 200][i % 4], cols=50) for i in range(9)]
    ins, outs, in_bytes, out_bytes = serve.GpuBackend._layout(reqs)
    a = serve.GpuBackend._ALIGN
    spans = []
    for r, (oc, oo), (cnt, fit) in zip(reqs, ins, outs):
        assert oc % a == 0 and oo % a == 0 and cnt % a == 0 and fit % a == 0
        spans.append(("in", oc, oc + 2 * int(r.offsets[-1])))
        spans.append(("in", oo, oo + 4 * (r.n_cand + 1)))
        spans.append(("out", cnt, cnt + 4 * r.n_cand))
        spans.append(("out", fit, fit + 8 * r.n_cand))
    for side, size in (("in", in_bytes), ("out", out_bytes)):
        s = sorted((lo, hi) for k, lo, hi in spans if k == side)
        assert all(h0 <= l1 for (_, h0), (l1, _) in zip(s, s[1:]))  # disjoint
        assert s[-1][1] <= size
    buf = np.zeros(in_bytes, dtype=np.uint8)
    serve.GpuBackend._pack(buf, reqs, ins)
    for r, (oc, oo) in zip(reqs, ins):
        tot = int(r.offsets[-1])
        assert np.array_equal(buf[oc:oc + 2 * tot].view(np.uint16), r.cols)
        assert np.array_equal(buf[oo:oo + 4 * (r.n_cand + 1)].view(np.uint32), r.offsets)


@pytest.mark.gpu
def test_served_lone_request_error_frees_the_slot():
    """A lone request whose list the library rejects (a column outside the matrix) raises from the
    pump; the slot it took is free again and the next request is served correctly."""
    from paper_1807_09932_gb300 import ebic
    be = serve.GpuBackend(max_batch=4, max_inflight=1, pair_budget=1 << 30)
    try:
        srv = serve.Server(be, hbm_budget=8 << 30, max_batch=4, max_inflight=1)
        ds = synth.make_dataset(720, 5000, 40, planted=synth.planted_specs_for(720, 5000, 40),
                                nan_frac=0.01)
        ac, ao = synth.population_from_lists([[0, 1, 2], [3, 4]])
        srv.add_run(serve.RunSpec(run_id=0, X=ds.X, max_cand=300, max_len=16,
                                  archive_cols=ac, archive_offsets=ao))
        c, o = synth.make_population(721, 100, 40, 2, 8)
        bad_c = c.copy()
        bad_c[5] = 40  # no such column
        srv.submit(serve.Request(run_id=0, cols=bad_c, offsets=o, t_arrival=0.0))
        with pytest.raises(ebic.EbicError):
            srv.pump()
        assert not srv.busy_runs and not any(s["busy"] for s in be.slots)
        good = serve.Request(run_id=0, cols=c, offsets=o, t_arrival=0.0)
        srv.submit(good)
        while not srv.done:
            srv.pump()
        ec, eb = oracle.eval_population(ds.X, c, o)
        _, abm = oracle.eval_population(ds.X, ac, ao)
        ef, _ = oracle.fitness(ds.X.shape[0], c, o, ec, eb, ac, ao, abm, want_overlaps=False)
        assert np.array_equal(good.counts, ec)
        assert np.array_equal(good.fitness, ef)
    finally:
        be.close()
