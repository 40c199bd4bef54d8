"""Autotuner: selection, cache round trip and keys (CPU, injected timing); on the GPU the tuned
tile shapes keep results identical and the chosen pair is the fastest measured."""
import numpy as np
import pytest

from paper_1807_09932_gb300 import autotune, synth


def test_select_picks_fastest_and_breaks_ties_by_shape():
    times = {(1, 0): 3.0, (1, 256): 2.0, (2, 0): 2.0, (2, 256): 5.0}
    bt, bc, ms, table = autotune.select(lambda t, c: times[(t, c)], (1, 2), (0, 256))
    assert (bt, bc, ms) == (1, 256, 2.0)
    assert table == times


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def measure(t, c):
        calls.append((t, c))
        return 10.0 - t + (c == 1024)

    key = autotune.shape_key(8, 64, 436444, 1600, 9.0, False)
    c1 = autotune.Cache(path)
    r1 = autotune.tune(key, measure, (1, 2), (0, 1024), cache=c1)
    assert r1[:2] == (2, 0) and r1[3] is False and len(calls) == 4
    c2 = autotune.Cache(path)            # a new process reads the same file
    r2 = autotune.tune(key, measure, (1, 2), (0, 1024), cache=c2)
    assert r2[:2] == (2, 0) and r2[3] is True and len(calls) == 4
    r3 = autotune.tune(key, measure, (1, 2), (0, 1024), cache=c2, force=True)
    assert r3[3] is False and len(calls) == 8


def test_shape_keys_separate_classes():
    k = autotune.shape_key
    assert k(8, 64, 436444, 1600, 9, False) != k(16, 200, 20000, 1600, 11, True)
    assert k(8, 64, 436444, 1600, 9, False) == k(8, 64, 436000, 1600, 9.2, False)
    assert k(8, 64, 436444, 1600, 9, False) != k(8, 64, 436444, 1600, 9, True)


@pytest.mark.gpu
def test_tuned_shapes_keep_results_and_pick_the_fastest(tmp_path):
    import torch
    from paper_1807_09932_gb300 import ebic
    import oracle
    ds, cols, offs = synth.config3(rows=50000)
    n = len(offs) - 1
    dc = torch.from_numpy(cols.view(np.int16)).cuda()
    do = torch.from_numpy(offs.view(np.int32)).cuda()
    with ebic.Matrix(ds.X) as m:
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        bm = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
        cache = autotune.Cache(str(tmp_path / "t.json"))
        tile, chunk, ms, hit = autotune.tune_matrix(m, dc, do, n, float(np.diff(offs).mean()),
                                                    cnt, bm, cache=cache, iters=2)
        assert not hit and tile in (1, 2, 4) and ms > 0
        table = cache.get(next(iter(cache.entries)))["table"]
        assert ms == min(table.values())
        got_c, got_b = ebic.eval_population(m, cols, offs)
        exp_c, exp_b = oracle.eval_population(ds.X, cols, offs)
        assert np.array_equal(got_c, exp_c) and np.array_equal(got_b, exp_b)
        assert autotune.tune_matrix(m, dc, do, n, float(np.diff(offs).mean()), cnt, bm,
                                    cache=cache)[3] is True
