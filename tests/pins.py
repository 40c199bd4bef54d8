"""Checks that pin the oracle to facts independent of itself.

Each check raises AssertionError on a mismatch. They are written against the ``oracle`` module's
public functions, so the mutation tests can run them against a deliberately broken build of the
oracle and confirm that each planted mistake is caught.

Sources of truth used here (never the oracle's own formula retyped):
  * Python's ``sorted`` (a library sort) for "the values follow the column order";
  * Python sets of row indices for overlaps;
  * ``scipy.stats.rankdata(method="dense")`` for dense ranks;
  * the closed form P(row follows an order of L i.i.d. continuous values) = 1/L!
    (2/L! with the negative-trend option, L >= 2);
  * algebraic invariants of the "greater or equal" rule and planted-bicluster recovery.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

import oracle
from paper_1807_09932_gb300 import synth

# value pool with ties, signed zeros, infinities and subnormals (IEEE edge cases)
EDGE_POOL = np.array([-np.inf, -2.0, -1.0, -1e-45, -0.0, 0.0, 1e-45, 1.4e-45, 1.0, 1.0, 2.0,
                      3.0, np.inf], dtype=np.float32)


def tiny_matrix(seed, R, C, nan_frac=0.1, pool=EDGE_POOL):
    rng = np.random.default_rng(seed)
    X = rng.choice(pool, size=(R, C)).astype(np.float32)
    X[rng.random((R, C)) < nan_frac] = np.nan
    return X


def all_candidates(C, max_len):
    out = []
    for L in range(1, max_len + 1):
        out.extend(itertools.permutations(range(C), L))
    return out


def brute_force(X, cands, exclude_missing, fill_value, negative):
    """Counts and bitmaps by sorting each row's gathered values with Python's sorted()."""
    R = X.shape[0]
    W = (R + 31) // 32
    counts = np.zeros(len(cands), dtype=np.uint32)
    bitmaps = np.zeros((len(cands), W), dtype=np.uint32)
    for p, cand in enumerate(cands):
        for r in range(R):
            vals = [float(X[r, c]) for c in cand]
            if any(math.isnan(v) for v in vals):
                if exclude_missing:
                    continue
                vals = [fill_value if math.isnan(v) else v for v in vals]
            ok = vals == sorted(vals) or (negative and vals == sorted(vals, reverse=True))
            if ok:
                counts[p] += 1
                bitmaps[p, r // 32] |= np.uint32(1 << (r % 32))
    return counts, bitmaps


def check_bruteforce(seed, R=45, C=5, max_len=4, nan_frac=0.1):
    X = tiny_matrix(seed, R, C, nan_frac)
    cands = all_candidates(C, max_len)
    cols, offs = synth.population_from_lists(cands)
    for excl in (True, False):
        for neg in (False, True):
            for fill in (0.0, 999.0):
                exp_c, exp_b = brute_force(X, cands, excl, fill, neg)
                got_c, got_b = oracle.eval_population(X, cols, offs, exclude_missing=excl,
                                                      fill_value=fill, negative=neg)
                assert np.array_equal(got_c, exp_c), (seed, excl, neg, fill)
                assert np.array_equal(got_b, exp_b), (seed, excl, neg, fill)


def check_closed_form(seed, R=60000, C=8, negative=False):
    """Mean match rate 1/L! (2/L! with negative trends) on an i.i.d. continuous background."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, C)).astype(np.float32)
    cands = []
    for L in (1, 2, 3, 4, 5):
        for _ in range(4):
            cands.append(list(rng.choice(C, size=L, replace=False)))
    cols, offs = synth.population_from_lists(cands)
    counts, _ = oracle.eval_population(X, cols, offs, negative=negative, want_bitmaps=False)
    for cand, n in zip(cands, counts):
        L = len(cand)
        p = 1.0 / math.factorial(L)
        if negative and L >= 2:
            p *= 2.0
        p = min(p, 1.0)
        sigma = math.sqrt(R * p * (1 - p))
        assert abs(int(n) - R * p) <= 5 * sigma + 1e-9, (cand, int(n), R * p, sigma)


def check_invariants(seed, R=500, C=12):
    """L=1 counts non-missing rows; appending/prepending a column never adds rows; a reversed
    candidate matches the same rows under the negative option; strictly increasing maps of the
    values leave results unchanged; negating the matrix swaps increasing and decreasing."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, C)).astype(np.float32)
    X[rng.random((R, C)) < 0.05] = np.nan
    # planted increasing rows so long candidates still match something
    order = rng.permutation(C)
    rows = rng.choice(R, size=R // 4, replace=False)
    X[np.ix_(rows, order)] = np.sort(X[np.ix_(rows, order)], axis=1)

    # L = 1
    cands = [[j] for j in range(C)]
    cols, offs = synth.population_from_lists(cands)
    cnt, _ = oracle.eval_population(X, cols, offs)
    assert np.array_equal(cnt, (~np.isnan(X)).sum(axis=0).astype(np.uint32))
    cnt_off, _ = oracle.eval_population(X, cols, offs, exclude_missing=False)
    assert np.all(cnt_off == R)

    # append / prepend monotonicity, nested along the planted order and along random orders
    for base in [list(order)] + [list(rng.permutation(C)) for _ in range(3)]:
        prefixes = [base[:k] for k in range(1, C + 1)]
        suffixes = [base[k:] for k in range(C)]
        for chain in (prefixes, suffixes[::-1]):
            cols, offs = synth.population_from_lists(chain)
            for neg in (False, True):
                c, b = oracle.eval_population(X, cols, offs, negative=neg)
                for i in range(len(chain) - 1):
                    assert c[i + 1] <= c[i]
                    assert np.all((b[i + 1] & ~b[i]) == 0), "longer candidate gained a row"
    # the planted order must keep its planted rows (minus NaN rows) at full length
    cols, offs = synth.population_from_lists([list(order)])
    _, b = oracle.eval_population(X, cols, offs)
    for r in rows:
        if not np.isnan(X[r]).any():
            assert b[0, r // 32] >> (r % 32) & 1

    # reversal under the negative-trend option
    cands = [list(rng.choice(C, size=rng.integers(1, 7), replace=False)) for _ in range(40)]
    rev = [c[::-1] for c in cands]
    cols, offs = synth.population_from_lists(cands)
    rcols, roffs = synth.population_from_lists(rev)
    c1, b1 = oracle.eval_population(X, cols, offs, negative=True)
    c2, b2 = oracle.eval_population(X, rcols, roffs, negative=True)
    assert np.array_equal(c1, c2) and np.array_equal(b1, b2)
    # increasing along reverse(c) is decreasing along c, so the union of the two increasing
    # results is the negative-option result
    a1, ab1 = oracle.eval_population(X, cols, offs)
    a2, ab2 = oracle.eval_population(X, rcols, roffs)
    assert np.array_equal(ab1 | ab2, b1)

    # strictly increasing maps leave every result unchanged: an exact power-of-two scaling, and
    # each row's values replaced by their dense ranks (scipy), NaN kept
    from scipy.stats import rankdata
    ranked = np.full_like(X, np.nan)
    for r in range(R):
        m = ~np.isnan(X[r])
        ranked[r, m] = rankdata(X[r, m].astype(np.float64), method="dense")
    for Y in ((X * np.float32(4)).astype(np.float32), ranked.astype(np.float32)):
        for neg in (False, True):
            d1 = oracle.eval_population(X, cols, offs, negative=neg)
            d2 = oracle.eval_population(Y, cols, offs, negative=neg)
            assert np.array_equal(d1[1], d2[1])

    # negation: increasing on -X == decreasing on X == increasing on reversed candidates of X
    n1 = oracle.eval_population(-X, cols, offs)[1]
    assert np.array_equal(n1, ab2)


def check_planted_recovery(seed):
    ds = synth.make_dataset(seed, 3000, 40, kind="beta",
                            planted=[(300, 8, False), (200, 6, True), (150, 12, False)],
                            nan_frac=0.01, exclude_missing=True)
    X = ds.X
    cands = [list(p.cols) for p in ds.planted]
    cols, offs = synth.population_from_lists(cands)
    for neg in (False, True):
        cnt, bm = oracle.eval_population(X, cols, offs, negative=neg)
        for i, p in enumerate(ds.planted):
            got = set(np.nonzero(np.unpackbits(bm[i].view(np.uint8), bitorder="little"))[0])
            want = {int(r) for r in p.rows if not np.isnan(X[r, p.cols]).any()}
            if p.negative and not neg:
                # a decreasing bicluster is not recovered in the increasing direction ...
                assert len(want & got) <= len(want) // 10 + 2
            else:
                assert want <= got, (i, neg, len(want - got))
            assert cnt[i] == len(got)
    # ... but is recovered by its reversed order without the option
    for i, p in enumerate(ds.planted):
        if p.negative:
            rc, ro = synth.population_from_lists([list(p.cols[::-1])])
            _, bm = oracle.eval_population(X, rc, ro)
            got = set(np.nonzero(np.unpackbits(bm[0].view(np.uint8), bitorder="little"))[0])
            want = {int(r) for r in p.rows if not np.isnan(X[r, p.cols]).any()}
            assert want <= got


def bits_to_rows(words):
    return set(np.nonzero(np.unpackbits(np.asarray(words, dtype="<u4").view(np.uint8),
                                        bitorder="little"))[0].tolist())


def check_fitness(seed, R=700, C=30, P=60, K=7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, C)).astype(np.float32)
    cols, offs = synth.make_population(seed + 1, P, C, 1, 6)
    counts, bm = oracle.eval_population(X, cols, offs)
    cands = [list(cols[offs[i]:offs[i + 1]]) for i in range(P)]

    # K = 0: F = n * 2^(L-1)
    ecols, eoffs = np.zeros(0, np.uint16), np.zeros(1, np.uint32)
    ebm = np.zeros((0, bm.shape[1]), np.uint32)
    f0, _ = oracle.fitness(R, cols, offs, counts, bm, ecols, eoffs, ebm)
    assert [int(v) for v in f0] == [int(n) * 2 ** (len(c) - 1) for n, c in zip(counts, cands)]

    # archive containing each candidate itself: p = 0
    fs, ov = oracle.fitness(R, cols, offs, counts, bm, cols, offs, bm)
    assert np.all(fs == 0)
    assert np.array_equal(np.diag(ov), counts)

    # random archive (random bitmaps and column sets): brute force with Python sets
    acands = [list(rng.choice(C, size=rng.integers(1, 6), replace=False)) for _ in range(K)]
    acols, aoffs = synth.population_from_lists(acands)
    abm = synth.random_bitmaps(seed + 2, K, R, density=0.4)
    fit, ov = oracle.fitness(R, cols, offs, counts, bm, acols, aoffs, abm)
    arows = [bits_to_rows(abm[a]) for a in range(K)]

    def q(n, L):
        return n * 2 ** (min(L, 33) - 1)

    for i, cand in enumerate(cands):
        rows_i = bits_to_rows(bm[i])
        assert len(rows_i) == counts[i]
        pen = 0
        for a in range(K):
            o = len(rows_i & arows[a])
            assert ov[i, a] == o
            # a penalises only when it shares a column and is at least as good as the candidate
            if set(cand) & set(acands[a]) and q(len(arows[a]), len(acands[a])) >= q(
                    len(rows_i), len(cand)):
                pen = max(pen, o)
        assert int(fit[i]) == q(int(counts[i]) - pen, len(cand))

    # a better candidate (superset of an archived bicluster's columns, fewer rows but a higher
    # quality) is not penalised by it; the archived one is penalised by the better one
    sub = [list(range(4))]
    sup = [list(range(6))]
    Xs = np.tile(np.arange(6, dtype=np.float32), (R, 1))      # every row increasing
    Xs[: R // 3, 5] = -1.0                                    # a third fail the 6-column chain
    sc, so = synth.population_from_lists(sub)
    pc, po = synth.population_from_lists(sup)
    nsub, bsub = oracle.eval_population(Xs, sc, so)
    nsup, bsup = oracle.eval_population(Xs, pc, po)
    assert q(int(nsup[0]), 6) > q(int(nsub[0]), 4)
    fsup, _ = oracle.fitness(R, pc, po, nsup, bsup, sc, so, bsub)
    assert int(fsup[0]) == q(int(nsup[0]), 6)
    fsub, osub = oracle.fitness(R, sc, so, nsub, bsub, pc, po, bsup)
    assert int(fsub[0]) == q(int(nsub[0]) - int(osub[0, 0]), 4)

    # disjoint columns: no penalty whatever the row overlap
    dc, do = synth.population_from_lists([[0, 1, 2]])
    dcnt, dbm = oracle.eval_population(X, dc, do)
    ac, ao = synth.population_from_lists([[3, 4]])
    full = np.full((1, dbm.shape[1]), 0xFFFFFFFF, np.uint32)
    fd, od = oracle.fitness(R, dc, do, dcnt, dbm, ac, ao, full)
    assert int(fd[0]) == int(dcnt[0]) * 4 and od[0, 0] == dcnt[0]

    # long candidates: the weight is 2^(min(L,33)-1)
    lc, lo = synth.population_from_lists([list(range(30))])
    one = np.array([1], np.uint32)
    fl, _ = oracle.fitness(R, lc, lo, one, np.zeros((1, bm.shape[1]), np.uint32),
                           ecols, eoffs, ebm)
    assert int(fl[0]) == 2 ** 29


def check_dense_ranks(seed, R=300, C=17):
    from scipy.stats import rankdata
    X = tiny_matrix(seed, R, C, nan_frac=0.15)
    got = oracle.dense_ranks(X, exclude_missing=True)
    for r in range(R):
        m = ~np.isnan(X[r])
        want = np.full(C, 0xFFFF, np.int64)
        if m.any():
            want[m] = rankdata(X[r, m].astype(np.float64), method="dense") - 1
        assert np.array_equal(got[r].astype(np.int64), want), r
    got_off = oracle.dense_ranks(X, exclude_missing=False, fill_value=999.0)
    Y = np.where(np.isnan(X), np.float32(999.0), X)
    for r in range(R):
        want = rankdata(Y[r].astype(np.float64), method="dense") - 1
        assert np.array_equal(got_off[r].astype(np.int64), want)
