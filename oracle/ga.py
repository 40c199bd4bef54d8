"""EBIC generation-loop oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the genetic algorithm that drives the search. The paper says only
that EBIC searches with evolutionary computation over a population of candidate biclusters
(arXiv 1807.09932, Methods, "Support for Big Data") and that the search is driven by counting
rows (Methods, "Handling missing values"). The operators are this project's definition D12 (the
generator D12.1, the operators D12.2, the initial population D12.3, a generation D12.4), written
out here step by step in the order that definition gives them. Scoring uses this package's plain
CPU evaluation and fitness (D1-D9); nothing here imports the CUDA library.

Only ``tests/`` may import this module. Pure Python loops: small populations only.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import eval_population, fitness

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
UNUSED_DRAWS = 1 << 16
REDRAWS = 32


# ---- D12.1 the generator ---------------------------------------------------------------------

def mix(z):
    """splitmix64's output function (Steele, Lea and Flood, OOPSLA 2014)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    def __init__(self, state):
        self.s = state & MASK64

    def next(self):
        self.s = (self.s + GAMMA) & MASK64
        return mix(self.s)

    def below(self, n):
        return self.next() % n

    def unit(self):
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def copy(self):
        return SplitMix64(self.s)


def child_generator(seed, gen, slot):
    """The generator of child slot `slot` of generation `gen`."""
    return SplitMix64(mix((mix((seed + GAMMA * (gen + 1)) & MASK64) + slot) & MASK64))


# ---- parameters ------------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    population: int = 1600
    generations: int = 100
    archive_size: int = 20
    elite: int = 16
    tournament: int = 4
    min_len: int = 2
    max_init_len: int = 6
    max_len: int = 64
    p_crossover: float = 0.5
    p_mutation: float = 0.7
    overlap_threshold: float = 0.5
    tabu_retries: int = 8
    seed: int = 1807099320
    negative: bool = False

    def f32(self, name):
        """A probability or threshold as the float32 value the parameters hold, widened."""
        return float(np.float32(getattr(self, name)))


# ---- D12.2 the operators -----------------------------------------------------------------------

def random_candidate(rng, C, p):
    L = p.min_len + rng.below(p.max_init_len - p.min_len + 1)
    cols = list(range(C))
    for i in range(L):
        j = i + rng.below(C - i)
        cols[i], cols[j] = cols[j], cols[i]
    return cols[:L]


def unused_column(rng, c, C):
    for _ in range(UNUSED_DRAWS):
        x = rng.below(C)
        if x not in c:
            return x
    return min(x for x in range(C) if x not in c)


def crossover(rng, a, b, C, p):
    cut = 1 + rng.below(len(a))
    child = list(a[:cut])
    for x in b:
        if len(child) >= p.max_len:
            break
        if x not in child:
            child.append(x)
    while len(child) < p.min_len:
        child.append(unused_column(rng, child, C))
    return child


def mutate(rng, c, C, p):
    """Mutates the list c in place."""
    first = rng.below(4)
    for k in range(4):
        op = (first + k) % 4
        if op == 0 and len(c) >= 2:                       # swap two positions
            i = rng.below(len(c))
            j = rng.below(len(c) - 1)
            if j >= i:
                j += 1
            c[i], c[j] = c[j], c[i]
            return
        if op == 1 and len(c) < C:                        # substitute by an unused column
            i = rng.below(len(c))
            c[i] = unused_column(rng, c, C)
            return
        if op == 2 and len(c) < p.max_len and len(c) < C:  # insert an unused column
            x = unused_column(rng, c, C)
            i = rng.below(len(c) + 1)
            c.insert(i, x)
            return
        if op == 3 and len(c) > p.min_len:                # delete a column
            del c[rng.below(len(c))]
            return


# ---- D12.3 the initial population ------------------------------------------------------------

def initial_population(C, p):
    rng = SplitMix64(p.seed)
    seen, pop = set(), []
    for _ in range(p.population):
        c = random_candidate(rng, C, p)
        t = 0
        while t < REDRAWS and tuple(c) in seen:
            c = random_candidate(rng, C, p)
            t += 1
        seen.add(tuple(c))
        pop.append(c)
    return pop


# ---- D12.4 a generation ----------------------------------------------------------------------

def quality(n, L):
    return int(n) << (min(L, 33) - 1)


def comes_before(i, j, pop, fit, counts):
    """Step 3's order: i before j."""
    if fit[i] != fit[j]:
        return fit[i] > fit[j]
    if counts[i] != counts[j]:
        return counts[i] > counts[j]
    if len(pop[i]) != len(pop[j]):
        return len(pop[i]) > len(pop[j])
    if pop[i] != pop[j]:
        return pop[i] < pop[j]
    return i < j


def order_key(i, pop, fit, counts):
    return (-int(fit[i]), -int(counts[i]), -len(pop[i]), pop[i], i)


def elites(pop, fit, counts, p):
    order = sorted(range(len(pop)), key=lambda i: order_key(i, pop, fit, counts))
    return order[:min(p.elite, len(pop))]


def offers(pop, counts, archive, K):
    """Step 4: the indices of up to 2K offered candidates, in offer order."""
    held = {tuple(m.cols) for m in archive}
    cand = [i for i in range(len(pop)) if counts[i] > 0]
    cand.sort(key=lambda i: (-quality(counts[i], len(pop[i])), -int(counts[i]), -len(pop[i]),
                             pop[i], i))
    out, taken = [], set()
    for i in cand:
        if len(out) >= 2 * K:
            break
        s = tuple(pop[i])
        if s in held or s in taken:
            continue
        taken.add(s)
        out.append(i)
    return out


@dataclasses.dataclass
class Member:
    cols: list
    count: int
    q: int
    bitmap: np.ndarray


def shares_column(a, b):
    return bool(set(a) & set(b))


def admit(archive, offered, overlap_with_member, overlap_between_offers, threshold, K):
    """Step 5. `offered`: Members in offer order; overlap_with_member(t, a) = o(offer t, member
    a); overlap_between_offers(t, u) = popcount(M_t & M_u). Returns the new archive."""
    alive = [True] * len(archive)
    admitted = []
    for t, c in enumerate(offered):
        limit = threshold * float(c.count)
        ok, evict = True, []
        for a, m in enumerate(archive):
            if not ok:
                break
            if not alive[a] or not shares_column(c.cols, m.cols):
                continue
            if float(overlap_with_member(t, a)) <= limit:
                continue
            if c.q > m.q:
                evict.append(a)
            else:
                ok = False
        for u in admitted:
            if not ok:
                break
            if shares_column(c.cols, offered[u].cols) and \
                    float(overlap_between_offers(t, u)) > limit:
                ok = False
        if not ok:
            continue
        for a in evict:
            alive[a] = False
        admitted.append(t)
    merged = [m for a, m in enumerate(archive) if alive[a]] + [offered[t] for t in admitted]
    merged.sort(key=lambda m: (-m.q, -m.count, -len(m.cols), m.cols))   # stable
    return merged[:K]


def tournament(rng, pop, fit, counts, p):
    best = rng.below(len(pop))
    for _ in range(p.tournament - 1):
        c = rng.below(len(pop))
        if comes_before(c, best, pop, fit, counts):
            best = c
    return best


def breed_child(rng, pop, fit, counts, tabu, C, p):
    """Step 6, one child from its own generator (left where the breeding ends)."""
    a = tournament(rng, pop, fit, counts, p)
    child = list(pop[a])
    if rng.unit() < p.f32("p_crossover"):
        b = tournament(rng, pop, fit, counts, p)
        child = crossover(rng, pop[a], pop[b], C, p)
    if rng.unit() < p.f32("p_mutation"):
        mutate(rng, child, C, p)
    t = 0
    while t < p.tabu_retries and tuple(child) in tabu:
        mutate(rng, child, C, p)
        t += 1
    t = 0
    while t < REDRAWS and tuple(child) in tabu:
        child = random_candidate(rng, C, p)
        t += 1
    return child


def place_children(first, children, generators, tabu, C, p):
    """Step 6, the pass in slot order: `first` are the elites' sequences, `children[k]` the
    child bred for the next slot and `generators[k]` its generator where breeding left it."""
    nxt = [list(c) for c in first]
    held = {tuple(c) for c in nxt}
    for child, rng in zip(children, generators):
        child = list(child)
        if tuple(child) in held:
            def taken():
                return tuple(child) in tabu or tuple(child) in held
            t = 0
            while t < p.tabu_retries and taken():
                mutate(rng, child, C, p)
                t += 1
            t = 0
            while t < REDRAWS and taken():
                child = random_candidate(rng, C, p)
                t += 1
        nxt.append(child)
        held.add(tuple(child))
    return nxt


def csr(lists):
    offs = np.zeros(len(lists) + 1, np.uint32)
    offs[1:] = np.cumsum([len(c) for c in lists])
    cols = np.array([x for c in lists for x in c], np.uint16)
    return cols, offs


def run(X, p, exclude_missing=True, fill_value=0.0):
    """The whole generation loop on the float32 matrix X. Returns the archive (Members, best
    first) and the number of generations run."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    R, C = X.shape
    W = (R + 31) // 32
    K = p.archive_size
    pop = initial_population(C, p)
    archive = []
    tabu = set()
    for g in range(p.generations):
        # 1. scores against the archive
        cols, offs = csr(pop)
        counts, bms = eval_population(X, cols, offs, exclude_missing=exclude_missing,
                                      fill_value=fill_value, negative=p.negative)
        acols, aoffs = csr([m.cols for m in archive]) if archive else (
            np.zeros(0, np.uint16), np.zeros(1, np.uint32))
        abm = np.array([m.bitmap for m in archive], np.uint32).reshape(len(archive), W)
        fit, ov = fitness(R, cols, offs, counts, bms, acols, aoffs, abm)
        # 2. tabu set
        for c in pop:
            tabu.add(tuple(c))
        # 3. elites; 4. offers; 5. admission
        el = elites(pop, fit, counts, p)
        idx = offers(pop, counts, archive, K)
        offered = [Member(list(pop[i]), int(counts[i]), quality(counts[i], len(pop[i])),
                          bms[i].copy()) for i in idx]
        if idx:
            ocols, ooffs = csr([pop[i] for i in idx])
            obm = np.ascontiguousarray(bms[idx])
            _, pair = fitness(R, ocols, ooffs, counts[idx], obm, ocols, ooffs, obm)
        else:
            pair = np.zeros((0, 0), np.uint32)
        archive = admit(archive, offered, lambda t, a: ov[idx[t], a], lambda t, u: pair[t, u],
                        p.f32("overlap_threshold"), K)
        if g + 1 == p.generations:
            break
        # 6. the next population
        first = [pop[e] for e in el]
        children, gens = [], []
        for slot in range(len(first), p.population):
            rng = child_generator(p.seed, g, slot)
            children.append(breed_child(rng, pop, fit, counts, tabu, C, p))
            gens.append(rng)
        pop = place_children(first, children, gens, tabu, C, p)
    return archive, p.generations
