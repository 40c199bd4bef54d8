"""Pair-table evaluation (an exact alternative encoding of the same rule) against the oracle and
against the rank-code evaluator, bit for bit."""
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


@pytest.mark.parametrize("R,C", [(1, 3), (33, 5), (1000, 40), (4097, 64), (777, 127), (2000, 128),
                                 (1500, 200), (600, 300)])
def test_pairs_match_oracle_and_direct(ebic, R, C):
    rng = np.random.default_rng(R + 7 * C)
    X = rng.standard_normal((R, C)).astype(np.float32)
    X[rng.random((R, C)) < 0.05] = np.nan
    X[rng.random((R, C)) < 0.05] = 0.25          # ties
    cols, offs = synth.make_population(R * C, 120, C, 1, min(C, 64))
    with ebic.Matrix(X) as m:
        size = m.build_pairs()
        assert size == C * C * ((m.words + 511) // 512 * 512) * 4 + 512  # and the all-ones row
        for neg in (False, True):
            c, b = ebic.eval_population(m, cols, offs, negative=neg)
            ec, eb = oracle.eval_population(X, cols, offs, negative=neg)
            assert np.array_equal(c, ec) and np.array_equal(b, eb)
            dc, db = ebic.eval_population(m, cols, offs, negative=neg, direct=True)
            assert np.array_equal(c, dc) and np.array_equal(b, db)
            c2, _ = ebic.eval_population(m, cols, offs, negative=neg, want_bitmaps=False)
            assert np.array_equal(c2, ec)


def test_pairs_exclusion_off_and_fill(ebic):
    from pins import tiny_matrix, all_candidates
    X = tiny_matrix(9, 500, 5, nan_frac=0.2)
    cols, offs = synth.population_from_lists(all_candidates(5, 4))
    for fill in (0.0, 2.0):
        with ebic.Matrix(X, exclude_missing=False, fill_value=fill) as m:
            m.build_pairs()
            for neg in (False, True):
                c, b = ebic.eval_population(m, cols, offs, negative=neg)
                ec, eb = oracle.eval_population(X, cols, offs, exclude_missing=False,
                                                fill_value=fill, negative=neg)
                assert np.array_equal(c, ec) and np.array_equal(b, eb)


def test_pair_table_limit_and_drop(ebic):
    X = np.random.default_rng(3).standard_normal((5000, 64)).astype(np.float32)
    cols, offs = synth.make_population(4, 50, 64, 2, 10)
    with ebic.Matrix(X) as m:
        need = 64 * 64 * ((m.words + 511) // 512 * 512) * 4 + 512  # and the all-ones row
        with pytest.raises(ebic.EbicError) as ei:
            m.build_pairs(max_bytes=need - 1)
        assert ei.value.code == ebic.EBIC_ERR_UNSUPPORTED
        assert m.build_pairs(max_bytes=need) == need
        a, _ = ebic.eval_population(m, cols, offs)
        m.drop_pairs()
        b, _ = ebic.eval_population(m, cols, offs)
        assert np.array_equal(a, b)


def test_pairs_config3_full_size_sampled(ebic):
    import torch
    ds, cols, offs = synth.config3()
    n = len(offs) - 1
    with ebic.Matrix(torch.from_numpy(ds.X).cuda()) as m:
        m.build_pairs()
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        bm = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
        dc = torch.from_numpy(cols.view(np.int16)).cuda()
        do = torch.from_numpy(offs.view(np.int32)).cuda()
        ebic.eval_population(m, dc, do, counts=cnt, bitmaps=bm)
        assert m.status() == ebic.EBIC_OK
        got_c = cnt.cpu().numpy().view(np.uint32)
        got_b = bm.cpu().numpy().view(np.uint32)
    idx = np.random.default_rng(11).choice(n, size=40, replace=False)
    sc, so = synth.population_from_lists([list(cols[offs[i]:offs[i + 1]]) for i in idx])
    ec, eb = oracle.eval_population(ds.X, sc, so)
    assert np.array_equal(got_c[idx], ec) and np.array_equal(got_b[idx], eb)
