"""Pins for the generation-loop oracle (oracle/ga.py), on the CPU.

The paper defines no operators (it says only that the search is evolutionary, Methods, "Support
for Big Data"); D12 is this project's definition. Each pin below fixes a part of the oracle by
something other than the oracle itself:
  * the generator: the published splitmix64 known-answer vector, and uniformity of below(n);
  * the random candidate: a partial Fisher-Yates shuffle, so every ordered selection is equally
    likely (chi-square over all of them);
  * crossover, the four mutations and the tournament: hand-worked cases with scripted draws;
  * the duplicate rule and the tabu rule: a repeat of an elite, a repeat of an earlier child and
    a tabu hit, hand-worked;
  * admission: a strictly worse member replaced, a member at least as good blocking an offer,
    an overlap at the limit, no shared column, an earlier admitted offer blocking a later one;
  * a whole run: invariants of the archive and recovery of a planted bicluster.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import ga

HERE = os.path.dirname(os.path.abspath(__file__))


class Scripted:
    """A generator that returns scripted below() draws and unit() values, in order."""

    def __init__(self, draws=(), units=()):
        self.draws = list(draws)
        self.units = list(units)
        self.asked = []

    def below(self, n):
        v = self.draws.pop(0)
        assert 0 <= v < n, (v, n)
        self.asked.append(n)
        return v

    def unit(self):
        return self.units.pop(0)


P = ga.Params(min_len=2, max_init_len=4, max_len=6, tabu_retries=2)


def test_splitmix64_known_answer():
    g = json.load(open(os.path.join(HERE, "golden", "splitmix64_seed1234567.json")))
    rng = ga.SplitMix64(g["seed"])
    assert [rng.next() for _ in range(5)] == [int(x) for x in g["outputs"]]


def test_below_is_uniform_and_unit_in_range():
    rng = ga.SplitMix64(42)
    n, draws = 7, 70000
    hist = np.bincount([rng.below(n) for _ in range(draws)], minlength=n)
    chi2 = float(((hist - draws / n) ** 2 / (draws / n)).sum())
    assert chi2 < 22.5            # 6 degrees of freedom, p = 0.001
    u = [rng.unit() for _ in range(10000)]
    assert min(u) >= 0.0 and max(u) < 1.0 and abs(np.mean(u) - 0.5) < 0.01


def test_random_candidate_is_a_uniform_ordered_selection():
    p = ga.Params(min_len=2, max_init_len=2)
    rng = ga.SplitMix64(7)
    C, draws = 4, 24000
    seen = {}
    for _ in range(draws):
        c = tuple(ga.random_candidate(rng, C, p))
        assert len(c) == 2 and len(set(c)) == 2 and all(0 <= x < C for x in c)
        seen[c] = seen.get(c, 0) + 1
    assert set(seen) == set(itertools.permutations(range(C), 2))   # all 12, nothing else
    exp = draws / 12
    chi2 = sum((v - exp) ** 2 / exp for v in seen.values())
    assert chi2 < 31.3            # 11 degrees of freedom, p = 0.001
    # lengths uniform in [min_len, max_init_len]
    p = ga.Params(min_len=1, max_init_len=3)
    lens = np.bincount([len(ga.random_candidate(rng, 10, p)) for _ in range(9000)], minlength=4)
    assert lens[0] == 0 and all(abs(lens[L] - 3000) < 200 for L in (1, 2, 3))


def test_random_candidate_by_hand():
    # L = 2 + 1 = 3; swaps (0,2), (1,1+2=3), (2,2+0=2) on [0,1,2,3,4] -> [2,3,0,1,4]
    rng = Scripted([1, 2, 2, 0])
    assert ga.random_candidate(rng, 5, P) == [2, 3, 0]
    assert rng.asked == [3, 5, 4, 3]


def test_unused_column_by_hand():
    rng = Scripted([1, 3, 0])
    assert ga.unused_column(rng, [1, 3], 5) == 0     # 1 and 3 are held: the third draw
    # every column but one held: the draws miss until the last resort, the smallest unused
    class Always:
        def below(self, n):
            return 0
    assert ga.unused_column(Always(), [0, 1, 2, 4], 5) == 3


def test_crossover_by_hand():
    a, b = [3, 1, 4, 5], [9, 2, 6, 5, 3]
    # cut = 1 + 1: prefix [3, 1], then b's columns not held, in b's order, up to max_len 6
    assert ga.crossover(Scripted([1]), a, b, 10, P) == [3, 1, 9, 2, 6, 5]
    assert ga.crossover(Scripted([1]), a, b, 10, ga.Params(max_len=4)) == [3, 1, 9, 2]
    # everything of b already held, child shorter than min_len: unused columns appended
    p = ga.Params(min_len=3, max_len=6)
    rng = Scripted([0, 7, 4, 8])
    assert ga.crossover(rng, [4, 2], [4], 10, p) == [4, 7, 8]   # 4 held: redrawn


def test_mutations_by_hand():
    C = 8
    # swap: first = 0, i = 1, j = 1 -> 2 (j >= i moves past i)
    c = [5, 6, 7]
    ga.mutate(Scripted([0, 1, 1]), c, C, P)
    assert c == [5, 7, 6]
    # substitute: first = 1, position 2, then the unused column 3
    c = [5, 6, 7]
    ga.mutate(Scripted([1, 2, 3]), c, C, P)
    assert c == [5, 6, 3]
    # insert: first = 2, the unused column (drawn 6 = held, then 1), then before position 0
    c = [5, 6, 7]
    ga.mutate(Scripted([2, 6, 1, 0]), c, C, P)
    assert c == [1, 5, 6, 7]
    # delete: first = 3, position 0
    c = [5, 6, 7]
    ga.mutate(Scripted([3, 0]), c, C, P)
    assert c == [6, 7]
    # delete not allowed at min_len: the next operator in order (swap) is taken
    c = [5, 6]
    ga.mutate(Scripted([3, 0, 0]), c, C, P)
    assert c == [6, 5]
    # at max_len with every column held: swap is the only operator left
    c = list(range(6))
    ga.mutate(Scripted([1, 0, 0]), c, 6, ga.Params(min_len=6, max_len=6))
    assert c == [1, 0, 2, 3, 4, 5]


def test_tournament_by_hand():
    pop = [[0, 1], [2, 3], [4, 5], [6, 7]]
    fit = np.array([5, 9, 9, 1], np.uint64)
    cnt = np.array([5, 9, 10, 1], np.uint32)
    p = ga.Params(tournament=3)
    # draws 0, 1, 2: 1 beats 0 on fitness, 2 beats 1 on count
    assert ga.tournament(Scripted([0, 1, 2]), pop, fit, cnt, p) == 2
    # equal keys: the lexicographically smaller sequence, then the lower index
    fit2 = np.array([4, 4, 4, 4], np.uint64)
    cnt2 = np.array([3, 3, 3, 3], np.uint32)
    assert ga.tournament(Scripted([3, 1, 2]), pop, fit2, cnt2, p) == 1
    pop3 = [[1, 2], [1, 2]]
    assert ga.tournament(Scripted([1, 0]), pop3, fit2[:2], cnt2[:2], ga.Params(tournament=2)) == 0


def test_elites_by_hand():
    pop = [[0, 1], [2, 3], [4, 5], [6, 7, 8], [1, 0]]
    fit = np.array([10, 20, 5, 10, 10], np.uint64)
    cnt = np.array([9, 3, 9, 9, 9], np.uint32)
    # fitness first (1), then among fitness 10 the count ties, so length (3), then the smaller
    # sequence ([0, 1] before [1, 0])
    assert ga.elites(pop, fit, cnt, ga.Params(elite=4)) == [1, 3, 0, 4]
    assert ga.elites(pop, fit, cnt, ga.Params(elite=9)) == [1, 3, 0, 4, 2]


def test_tabu_hit_is_mutated_then_replaced():
    pop = [[0, 1], [2, 3]]
    fit = np.array([2, 1], np.uint64)
    cnt = np.array([2, 1], np.uint32)
    p = ga.Params(min_len=2, max_init_len=2, max_len=2, tournament=1, p_crossover=0.0,
                  p_mutation=0.0, tabu_retries=1)
    # parent 0 is tabu; one swap (the only retry) gives [1, 0], also tabu; then a random
    # candidate: L = 2, swaps (0, 2) and (1, 1) on [0, 1, 2, 3] give [2, 1]
    rng = Scripted(draws=[0,          # tournament: parent 0
                          0, 0, 0,    # mutate: swap i = 0, j = 0 -> 1
                          0, 2, 0],   # random candidate: L = 2, swap (0, 2), swap (1, 1)
                   units=[0.9, 0.9])
    tabu = {(0, 1), (1, 0)}
    child = ga.breed_child(rng, pop, fit, cnt, tabu, 4, p)
    assert child == [2, 1]
    # not tabu: bred as drawn, no further draws
    rng = Scripted(draws=[1], units=[0.9, 0.9])
    assert ga.breed_child(rng, pop, fit, cnt, {(0, 1)}, 4, p) == [2, 3]
    assert rng.draws == []


def test_duplicates_in_slot_order_by_hand():
    p = ga.Params(min_len=2, max_init_len=2, max_len=3, tabu_retries=2)
    tabu = {(2, 1)}
    first = [[1, 2]]                      # an elite
    children = [[1, 2], [3, 4], [3, 4], [5, 6]]
    rngs = [Scripted([0, 0, 0,            # repeats the elite: swap -> [2, 1], tabu
                      0, 0, 0,            # swap -> [1, 2], held; the two retries are spent
                      0, 5, 6]),          # random: L = 2, swaps (0, 5), (1, 7) -> [5, 7]
            Scripted([]),                 # [3, 4]: no repeat, placed as bred
            Scripted([3, 0, 0]),          # repeats the child before: delete is not allowed at
                                          # min_len, so the next operator, swap -> [4, 3]
            Scripted([])]
    out = ga.place_children(first, children, rngs, tabu, 10, p)
    assert out == [[1, 2], [5, 7], [3, 4], [4, 3], [5, 6]]
    assert len({tuple(c) for c in out}) == len(out)


def _member(cols, count, q, W=1):
    return ga.Member(cols=list(cols), count=count, q=q, bitmap=np.zeros(W, np.uint32))


def test_admission_by_hand():
    thr = 0.5
    # a strictly worse member overlapping the offer by more than the limit is replaced
    arch = [_member([0, 1], 10, 10)]
    off = [_member([1, 2], 10, 20)]
    out = ga.admit(arch, off, lambda t, a: 6, lambda t, u: 0, thr, 4)
    assert [m.cols for m in out] == [[1, 2]]
    # a member at least as good blocks it (equal quality counts as at least as good)
    arch = [_member([0, 1], 10, 20)]
    out = ga.admit(arch, off, lambda t, a: 6, lambda t, u: 0, thr, 4)
    assert [m.cols for m in out] == [[0, 1]]
    # an overlap exactly at the limit (0.5 x 10 = 5) is not more than it: both kept, by quality
    out = ga.admit(arch, [_member([1, 2], 10, 30)], lambda t, a: 5, lambda t, u: 0, thr, 4)
    assert [m.cols for m in out] == [[1, 2], [0, 1]]
    # no shared column: no penalty whatever the overlap
    out = ga.admit(arch, [_member([2, 3], 10, 5)], lambda t, a: 10, lambda t, u: 0, thr, 4)
    assert [m.cols for m in out] == [[0, 1], [2, 3]]
    # an offer admitted earlier in the generation blocks a later one sharing a column
    offs = [_member([4, 5], 8, 40), _member([5, 6], 8, 30), _member([7, 8], 8, 30)]
    out = ga.admit([], offs, lambda t, a: 0, lambda t, u: 8, thr, 4)
    assert [m.cols for m in out] == [[4, 5], [7, 8]]
    # a member already replaced in this generation no longer blocks
    arch = [_member([0, 1], 10, 10), _member([1, 9], 10, 15)]
    offs = [_member([1, 2], 10, 20), _member([9, 3], 10, 12)]
    ov = {(0, 0): 6, (0, 1): 6, (1, 0): 0, (1, 1): 9}
    out = ga.admit(arch, offs, lambda t, a: ov[(t, a)], lambda t, u: 0, thr, 4)
    assert [m.cols for m in out] == [[1, 2], [9, 3]]
    # the archive keeps the best K, ordered by (q, count, length, columns)
    offs = [_member([1], 3, 3), _member([2], 3, 3), _member([0], 4, 3), _member([3, 4], 3, 3)]
    out = ga.admit([], offs, lambda t, a: 0, lambda t, u: 0, thr, 3)
    assert [m.cols for m in out] == [[0], [3, 4], [1]]


def test_offers_by_hand():
    pop = [[0, 1], [2, 3], [0, 1], [4, 5], [6, 7]]
    counts = np.array([4, 0, 4, 8, 2], np.uint32)
    arch = [_member([4, 5], 8, 16)]
    # [2, 3] has no rows, [0, 1] once (lower index), [4, 5] is archived
    assert ga.offers(pop, counts, arch, 1) == [0, 4]
    assert ga.offers(pop, counts, arch, 0) == []


def _planted_matrix(seed, R, C, rows, order):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, C)).astype(np.float32)
    X[np.ix_(rows, order)] = np.sort(X[np.ix_(rows, order)], axis=1)
    return X


def test_whole_run_invariants_and_planted_recovery():
    R, C = 600, 12
    order = [7, 2, 9, 4, 11]
    rows = np.arange(0, 600, 3)
    X = _planted_matrix(3, R, C, rows, order)
    p = ga.Params(population=120, generations=12, archive_size=6, elite=6, max_init_len=4,
                  max_len=8, seed=99)
    arch, _ = ga.run(X, p)
    assert 1 <= len(arch) <= p.archive_size
    W = (R + 31) // 32
    seqs = [tuple(m.cols) for m in arch]
    assert len(set(seqs)) == len(seqs)
    keys = [(-m.q, -m.count, -len(m.cols), m.cols) for m in arch]
    assert keys == sorted(keys)
    cols, offs = ga.csr([m.cols for m in arch])
    c, b = oracle.eval_population(X, cols, offs)
    assert np.array_equal(c, [m.count for m in arch])
    assert np.array_equal(b, np.array([m.bitmap for m in arch]).reshape(len(arch), W))
    assert all(m.q == m.count << (min(len(m.cols), 33) - 1) for m in arch)
    # members sharing a column overlap by at most the threshold of the larger one's rows
    for i, j in itertools.combinations(range(len(arch)), 2):
        if set(arch[i].cols) & set(arch[j].cols):
            o = int(np.unpackbits((b[i] & b[j]).view(np.uint8)).sum())
            assert o <= 0.5 * max(arch[i].count, arch[j].count)
    # the best member is a subsequence of the planted order matched by (nearly) all its rows
    best = arch[0].cols
    it = iter(order)
    assert len(best) >= 4 and all(x in it for x in best)
    # deterministic
    arch2, _ = ga.run(X, p)
    assert [(m.cols, m.count) for m in arch2] == [(m.cols, m.count) for m in arch]


def test_sequences_run_out_on_few_columns():
    # 3 columns, lengths 2..3: 12 sequences in all, population 10 -- repeats and tabu hits are
    # unavoidable; the loop still runs and every placed child is a valid candidate
    X = np.random.default_rng(5).standard_normal((200, 3)).astype(np.float32)
    p = ga.Params(population=10, generations=5, archive_size=4, elite=2, max_init_len=3,
                  max_len=3, seed=5)
    arch, _ = ga.run(X, p)
    assert all(2 <= len(m.cols) <= 3 and len(set(m.cols)) == len(m.cols) for m in arch)
