"""The generation loops against the generation-loop oracle (oracle/ga.py, definition D12).

Both loops -- the host loop (ebic_run, and ebic_run_custom with the oracle's scores) and the
device loop (ebic_run with EBIC_RUN_ON_DEVICE) -- must reach the oracle's archive: the same
members in the same order, with the same row counts, qualities and (from ebic_run) bitmaps.
The paper says only that the search is evolutionary over a population (Methods, "Support for
Big Data"); the operators are D12.

On the CPU: ebic_run_custom (the host loop, scored by the CPU oracle through callbacks) over
parameter sets that exercise each rule -- tabu hits and repeats on few columns, no elites,
tournaments of one, certain crossover and mutation, thresholds 0 and 1, negative trends.
On the GPU: ebic_run with both loops, on rank codes and on the pair table.
"""
import numpy as np
import pytest

from oracle import ga
from paper_1807_09932_gb300 import synth

CASES = {
    "planted": dict(seed_data=8, R=1500, C=12, kw=dict(population=160, generations=6,
                                                       archive_size=8, elite=8, max_init_len=4,
                                                       max_len=8)),
    "few columns": dict(seed_data=19, R=900, C=5, kw=dict(population=120, generations=7,
                                                          archive_size=4, elite=4,
                                                          max_init_len=4, max_len=5)),
    "no elites, tournament of one": dict(seed_data=3, R=700, C=9,
                                         kw=dict(population=90, generations=6, archive_size=6,
                                                 elite=0, tournament=1, max_init_len=3,
                                                 max_len=6, seed=11)),
    "always cross and mutate, threshold 0": dict(seed_data=4, R=1200, C=16,
                                                 kw=dict(population=100, generations=5,
                                                         archive_size=10, p_crossover=1.0,
                                                         p_mutation=1.0, overlap_threshold=0.0,
                                                         max_len=10, seed=12)),
    "threshold 1, one retry": dict(seed_data=5, R=800, C=7,
                                   kw=dict(population=150, generations=6, archive_size=12,
                                           overlap_threshold=1.0, tabu_retries=1, max_len=7,
                                           seed=13)),
    "negative trends": dict(seed_data=6, R=1000, C=20, negative=True,
                            kw=dict(population=140, generations=6, archive_size=16,
                                    max_len=12, seed=14)),
    "length-one candidates": dict(seed_data=7, R=600, C=6,
                                  kw=dict(population=60, generations=6, archive_size=5,
                                          min_len=1, max_init_len=3, max_len=6, seed=15)),
}


def _data(case):
    ds = synth.make_dataset(case["seed_data"], case["R"], case["C"], kind="normal",
                            planted=[(case["R"] // 5, min(case["C"] - 1, 6), False),
                                     (case["R"] // 6, min(case["C"] - 1, 4), True)],
                            nan_frac=0.01)
    return ds.X


def _oracle_archive(X, case):
    p = ga.Params(negative=case.get("negative", False), **case["kw"])
    arch, _ = ga.run(X, p)
    return arch


def _same(res, arch, bitmaps=True):
    assert res["members"] == [m.cols for m in arch]
    assert [int(x) for x in res["counts"]] == [m.count for m in arch]
    assert [int(x) for x in res["quality"]] == [m.q for m in arch]
    if bitmaps:
        assert np.array_equal(res["bitmaps"], np.array([m.bitmap for m in arch], np.uint32)
                              .reshape(len(arch), res["bitmaps"].shape[1]))


def _params(ebic, case, flags=0):
    kw = dict(case["kw"])
    if case.get("negative"):
        flags |= ebic.EBIC_NEGATIVE_TRENDS
    return ebic.ebic_params_default(flags=flags, **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_loop_equals_oracle_on_cpu(name):
    from ga_oracle import OracleScorer
    from paper_1807_09932_gb300 import ebic
    case = CASES[name]
    X = _data(case)
    sc = OracleScorer(X, negative=case.get("negative", False))
    res = ebic.ebic_run_custom(X.shape[0], X.shape[1], _params(ebic, case), sc.evaluator)
    assert sc.error is None
    _same(res, _oracle_archive(X, case), bitmaps=False)


@pytest.mark.gpu
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("name", sorted(CASES))
def test_gpu_loops_equal_oracle(name, pairs):
    from paper_1807_09932_gb300 import ebic
    case = CASES[name]
    X = _data(case)
    arch = _oracle_archive(X, case)
    with ebic.Matrix(X) as m:
        if pairs:
            m.build_pairs()
        host = ebic.ebic_run(m.handle, _params(ebic, case))
        dev = ebic.ebic_run(m.handle, _params(ebic, case, ebic.EBIC_RUN_ON_DEVICE))
    _same(host, arch)
    _same(dev, arch)
