// Host genetic algorithm of EBIC: ebic_run (scoring on the GPU) and ebic_run_custom (scoring by
// caller callbacks).
//
// The paper states that EBIC searches with evolutionary computation over a population (up to
// 65,535 candidates; 1,600 or fewer usually converge; Methods, "Support for Big Data") and that
// the search is driven by counting rows (Methods, "Handling missing values"). It does not define
// the operators. The generation loop below is the project's definition:
//   * random initial candidates (length uniform in [min_len, max_init_len], distinct columns);
//   * every generation: score (counts, penalised fitness and overlaps against the archive),
//     update the archive, then breed the next population: the `elite` best survive unchanged;
//     the others are tournament winners, crossed over (order-preserving: a prefix of parent A,
//     then parent B's columns not yet present, in B's order) and mutated (swap, substitute,
//     insert or delete one column);
//   * tabu list: a child whose exact column sequence was already evaluated, or already sits in the
//     new population, is mutated again (up to tabu_retries times), then replaced by a random one;
//   * archive: the best `archive_size` distinct candidates by quality n << (min(L,33)-1)
//     (ties: more rows, longer, lexicographically smaller columns). Each generation up to 2K
//     candidates are offered, best quality first: one is admitted unless a member sharing a
//     column overlaps it by more than overlap_threshold x its row count without being strictly
//     worse; strictly worse members it overlaps that much are replaced by it.
// Random draws come from splitmix64 counter generators: the initial population from one seeded
// with `seed`, and child slot j of generation g from its own, seeded from (seed, g, j). A child is
// bred against the tabu list alone, so the children of a generation are bred in parallel (host
// threads); a pass in slot order then gives a child that repeats an earlier one of the same new
// population further mutations, or a random replacement, from its own generator. Every decision
// depends only on draws and exact integer scores, so a run is reproducible bit for bit, whatever
// the number of threads, and independent of which evaluator produced the (identical) scores.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ebic.h"
#include "ebic_internal.h"

using namespace ebic;

namespace {

struct Rng {  // splitmix64 (Steele, Lea, Flood 2014), as a counter-based generator
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint32_t below(uint32_t n) { return (uint32_t)(next() % n); }
  double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// The generator of child slot `slot` of generation `gen`: its state is the splitmix64 output
// function applied twice, over (seed, gen) and then the slot.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
Rng child_stream(uint64_t seed, uint32_t gen, uint32_t slot) {
  return Rng{mix64(mix64(seed + 0x9E3779B97F4A7C15ull * ((uint64_t)gen + 1)) + slot)};
}

// A candidate: up to kMaxLen columns held inline, so copying, crossing and mutating the
// population allocates nothing. The members the GA uses behave as std::vector's do.
struct Cand {
  uint32_t n = 0;
  uint16_t c[kMaxLen];
  Cand() = default;
  template <class It>
  Cand(It b, It e) {
    for (; b != e; ++b) c[n++] = (uint16_t)*b;
  }
  Cand(const Cand& o) : n(o.n) { std::memcpy(c, o.c, (size_t)n * 2); }
  Cand& operator=(const Cand& o) {
    n = o.n;
    std::memcpy(c, o.c, (size_t)n * 2);
    return *this;
  }
  size_t size() const { return n; }
  uint16_t* begin() { return c; }
  uint16_t* end() { return c + n; }
  const uint16_t* begin() const { return c; }
  const uint16_t* end() const { return c + n; }
  uint16_t& operator[](size_t i) { return c[i]; }
  uint16_t operator[](size_t i) const { return c[i]; }
  void push_back(uint16_t x) { c[n++] = x; }
  uint16_t* insert(uint16_t* pos, uint16_t x) {
    std::memmove(pos + 1, pos, (size_t)(end() - pos) * 2);
    *pos = x;
    ++n;
    return pos;
  }
  uint16_t* erase(uint16_t* pos) {
    std::memmove(pos, pos + 1, (size_t)(end() - pos - 1) * 2);
    --n;
    return pos;
  }
  bool operator==(const Cand& o) const {
    return n == o.n && std::memcmp(c, o.c, (size_t)n * 2) == 0;
  }
  bool operator!=(const Cand& o) const { return !(*this == o); }
  bool operator<(const Cand& o) const {
    return std::lexicographical_compare(begin(), end(), o.begin(), o.end());
  }
};

struct CandHash {
  size_t operator()(const Cand& c) const {
    uint64_t h = 1469598103934665603ull;  // FNV-1a
    for (uint16_t x : c) { h ^= x; h *= 1099511628211ull; }
    return (size_t)(h ^ c.size());
  }
};

// An exact set of column sequences without an allocation per entry: the sequences sit in one
// arena, found by open addressing (linear probing) on their FNV-1a hash; clear() keeps the
// capacity for the next generation.
class CandSet {
 public:
  void clear() {
    std::fill(slots_.begin(), slots_.end(), 0u);
    arena_.clear();
    ent_.clear();
  }
  size_t count(const Cand& c) const { return find(c, CandHash()(c)) ? 1 : 0; }
  bool insert(const Cand& c) { return insert(c, CandHash()(c)); }
  // the same with the sequence's hash (CandHash) already computed
  size_t count(const Cand& c, uint64_t h) const { return find(c, h) ? 1 : 0; }
  bool insert(const Cand& c, uint64_t h) {
    if (find(c, h)) return false;
    if ((ent_.size() + 1) * 2 > slots_.size()) grow();
    ent_.push_back(Ent{(uint32_t)arena_.size(), (uint32_t)c.size(), h});
    arena_.insert(arena_.end(), c.begin(), c.end());
    place((uint32_t)ent_.size(), h);
    return true;
  }

 private:
  struct Ent {
    uint32_t off, len;
    uint64_t h;
  };
  static size_t slot_of(uint64_t h) {  // spread the hash's bits before masking
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    return (size_t)h;
  }
  bool find(const Cand& c, uint64_t h) const {
    if (slots_.empty()) return false;
    const size_t mask = slots_.size() - 1;
    for (size_t i = slot_of(h) & mask;; i = (i + 1) & mask) {
      const uint32_t s = slots_[i];
      if (s == 0) return false;
      const Ent& e = ent_[s - 1];
      if (e.h == h && e.len == c.size() &&
          std::equal(c.begin(), c.end(), arena_.begin() + e.off))
        return true;
    }
  }
  void place(uint32_t entry_plus_one, uint64_t h) {
    const size_t mask = slots_.size() - 1;
    size_t i = slot_of(h) & mask;
    while (slots_[i] != 0) i = (i + 1) & mask;
    slots_[i] = entry_plus_one;
  }
  void grow() {
    slots_.assign(slots_.empty() ? 4096 : slots_.size() * 2, 0u);
    for (size_t k = 0; k < ent_.size(); ++k) place((uint32_t)k + 1, ent_[k].h);
  }
  std::vector<uint16_t> arena_;
  std::vector<Ent> ent_;
  std::vector<uint32_t> slots_;  // entry index + 1, 0 = empty
};

// The sequences of the population being built, as indices into it (no copy): open addressing on
// the sequences' FNV-1a hashes, the hashes kept beside the population.
class SlotSet {
 public:
  void reset(size_t n_max) {
    size_t cap = 64;
    while (cap < 2 * n_max) cap <<= 1;
    slots_.assign(cap, 0u);
  }
  bool contains(const Cand& c, uint64_t h, const std::vector<Cand>& seqs,
                const std::vector<uint64_t>& hashes) const {
    const size_t mask = slots_.size() - 1;
    for (size_t i = spread(h) & mask;; i = (i + 1) & mask) {
      const uint32_t s = slots_[i];
      if (s == 0) return false;
      if (hashes[s - 1] == h && seqs[s - 1] == c) return true;
    }
  }
  void add(uint32_t index, uint64_t h) {  // the caller keeps the set at most half full
    const size_t mask = slots_.size() - 1;
    size_t i = spread(h) & mask;
    while (slots_[i] != 0) i = (i + 1) & mask;
    slots_[i] = index + 1;
  }

 private:
  static size_t spread(uint64_t h) {
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    return (size_t)h;
  }
  std::vector<uint32_t> slots_;  // index + 1, 0 = empty
};

uint64_t quality(uint32_t n, size_t L) { return (uint64_t)n << ((L < 33 ? L : 33) - 1); }

// Scoring of one generation, implemented by the GPU (ebic_run) or by callbacks.
struct Evaluator {
  virtual ~Evaluator() = default;
  virtual int evaluate(const std::vector<uint16_t>& cols, const std::vector<uint32_t>& offs,
                       uint32_t n, uint32_t* counts, uint64_t* fitness, uint32_t* overlaps) = 0;
  // Scoring in two halves, so that the caller can work between them: begin issues the scoring
  // (the lists must stay unchanged until end), end writes counts, fitness and overlaps. By
  // default begin does it all.
  virtual int evaluate_begin(const std::vector<uint16_t>& cols, const std::vector<uint32_t>& offs,
                             uint32_t n, uint32_t* counts, uint64_t* fitness, uint32_t* overlaps) {
    return evaluate(cols, offs, n, counts, fitness, overlaps);
  }
  virtual int evaluate_end() { return EBIC_OK; }
  virtual int pair_overlaps(const std::vector<uint32_t>& idx, uint32_t* out) = 0;
  // The same in two halves, so that the caller can work between them: begin issues the work for
  // `idx`, end (called once after each begin) writes the [t][t] overlaps to out. By default
  // begin does it all.
  virtual int pair_overlaps_begin(const std::vector<uint32_t>& idx) {
    pending_.assign(idx.size() * idx.size(), 0u);
    return idx.empty() ? EBIC_OK : pair_overlaps(idx, pending_.data());
  }
  virtual int pair_overlaps_end(uint32_t* out) {
    std::copy(pending_.begin(), pending_.end(), out);
    return EBIC_OK;
  }
  std::vector<uint32_t> pending_;
  virtual int set_archive(const std::vector<int32_t>& src) = 0;
  virtual bool has_bitmaps() const { return false; }
  virtual int archive_bitmaps(uint32_t* out, uint32_t k) { (void)out; (void)k; return EBIC_OK; }
};

struct Member {
  Cand cols;
  uint32_t count;
  uint64_t q;
  int32_t src;  // population index (>= 0) or -(old archive index + 1)
};

bool member_before(const Member& a, const Member& b) {
  if (a.q != b.q) return a.q > b.q;
  if (a.count != b.count) return a.count > b.count;
  if (a.cols.size() != b.cols.size()) return a.cols.size() > b.cols.size();
  return a.cols < b.cols;
}

bool shares_column(const Cand& a, const Cand& b) {
  for (uint16_t x : a)
    for (uint16_t y : b)
      if (x == y) return true;
  return false;
}

// The variation operators, drawing from `rng` (set per child). One Breeder per thread: the
// column list is scratch.
struct Breeder {
  const ebic_params& p;
  int32_t ncols;
  Rng rng;
  std::vector<uint16_t> all_cols;  // 0 .. ncols-1 between calls

  Breeder(const ebic_params& prm, int32_t nc) : p(prm), ncols(nc), rng{prm.seed} {
    all_cols.resize((size_t)nc);
    for (int32_t i = 0; i < nc; ++i) all_cols[(size_t)i] = (uint16_t)i;
  }

  Cand random_candidate() {
    const uint32_t L = p.min_len + rng.below(p.max_init_len - p.min_len + 1);
    uint32_t js[kMaxLen];
    for (uint32_t i = 0; i < L; ++i) {  // partial Fisher-Yates over the column list
      js[i] = i + rng.below((uint32_t)ncols - i);
      std::swap(all_cols[i], all_cols[js[i]]);
    }
    Cand c(all_cols.begin(), all_cols.begin() + L);
    for (uint32_t i = L; i-- > 0;) std::swap(all_cols[i], all_cols[js[i]]);  // back to 0..ncols-1
    return c;
  }

  uint16_t unused_column(const Cand& c) {  // callers ensure c.size() < ncols
    for (uint32_t t = 0; t < kUnusedDraws; ++t) {
      const uint16_t x = (uint16_t)rng.below((uint32_t)ncols);
      if (std::find(c.begin(), c.end(), x) == c.end()) return x;
    }
    for (int32_t x = 0; x < ncols; ++x)  // after kUnusedDraws misses: the smallest unused one
      if (std::find(c.begin(), c.end(), (uint16_t)x) == c.end()) return (uint16_t)x;
    return 0;
  }

  Cand crossover(const Cand& a, const Cand& b) {
    const uint32_t cut = 1 + rng.below((uint32_t)a.size());
    Cand child(a.begin(), a.begin() + cut);
    for (uint16_t x : b) {
      if (child.size() >= p.max_len) break;
      if (std::find(child.begin(), child.end(), x) == child.end()) child.push_back(x);
    }
    while (child.size() < p.min_len) child.push_back(unused_column(child));
    return child;
  }

  void mutate(Cand& c) {
    const uint32_t first = rng.below(4);
    for (uint32_t k = 0; k < 4; ++k) {
      switch ((first + k) % 4) {
        case 0:  // swap two positions
          if (c.size() >= 2) {
            const uint32_t i = rng.below((uint32_t)c.size());
            uint32_t j = rng.below((uint32_t)c.size() - 1);
            if (j >= i) ++j;
            std::swap(c[i], c[j]);
            return;
          }
          break;
        case 1:  // substitute a column by an unused one
          if ((int32_t)c.size() < ncols) {
            const uint32_t i = rng.below((uint32_t)c.size());
            c[i] = unused_column(c);
            return;
          }
          break;
        case 2:  // insert an unused column
          if (c.size() < p.max_len && (int32_t)c.size() < ncols) {
            const uint16_t x = unused_column(c);
            const uint32_t i = rng.below((uint32_t)c.size() + 1);
            c.insert(c.begin() + i, x);
            return;
          }
          break;
        default:  // delete a column
          if (c.size() > p.min_len) {
            c.erase(c.begin() + rng.below((uint32_t)c.size()));
            return;
          }
          break;
      }
    }
  }
};

// Host threads for the breeding of a generation: start(n, f) has the pool's threads call
// f(i, worker) for i in [0, n) and returns at once, so the caller can issue other work; finish()
// has the caller (worker 0) take the calls still left, and returns when all have returned.
class Workers {
 public:
  explicit Workers(unsigned n) : n_(n < 1 ? 1 : n) {
    for (unsigned w = 1; w < n_; ++w) threads_.emplace_back([this, w] { loop(w); });
  }
  ~Workers() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
      ++epoch_;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  unsigned size() const { return n_; }
  void start(uint32_t n, std::function<void(uint32_t, unsigned)> f) {
    job_ = std::move(f);
    n_items_ = n;
    next_.store(0, std::memory_order_relaxed);
    if (n_ == 1 || n < 2 * kChunk) {  // not worth waking the pool: finish() does it all
      pooled_ = false;
      return;
    }
    pooled_ = true;
    {
      std::lock_guard<std::mutex> g(m_);
      busy_ = n_ - 1;
      ++epoch_;
    }
    cv_.notify_all();
  }
  void finish() {
    work(0);
    if (pooled_) {
      std::unique_lock<std::mutex> lk(m_);
      done_cv_.wait(lk, [this] { return busy_ == 0; });
    }
    job_ = nullptr;
  }

 private:
  static constexpr uint32_t kChunk = 16;
  void work(unsigned w) {
    for (;;) {
      const uint32_t b = next_.fetch_add(kChunk, std::memory_order_relaxed);
      if (b >= n_items_) return;
      const uint32_t e = std::min(b + kChunk, n_items_);
      for (uint32_t i = b; i < e; ++i) job_(i, w);
    }
  }
  void loop(unsigned w) {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return epoch_ != seen; });
        seen = epoch_;
        if (stop_) return;
      }
      work(w);
      {
        std::lock_guard<std::mutex> g(m_);
        if (--busy_ == 0) done_cv_.notify_one();
      }
    }
  }
  unsigned n_;
  std::vector<std::thread> threads_;
  std::mutex m_;
  std::condition_variable cv_, done_cv_;
  std::function<void(uint32_t, unsigned)> job_;  // set before the threads are woken
  uint32_t n_items_ = 0;
  bool pooled_ = false;
  std::atomic<uint32_t> next_{0};
  unsigned busy_ = 0;
  uint64_t epoch_ = 0;
  bool stop_ = false;
};

// Host threads that breed a generation: EBIC_HOST_THREADS when set (1 .. 64), else the cores (at
// most 16) with at least 128 children each. The result does not depend on the count.
unsigned breeding_threads(uint32_t population) {
  if (const char* e = std::getenv("EBIC_HOST_THREADS")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 1 && v <= 64) return (unsigned)v;
  }
  const unsigned hw = std::thread::hardware_concurrency();
  unsigned n = hw == 0 ? 1 : (hw > 16 ? 16 : hw);
  const unsigned by_size = population / 128;  // at least 128 children per thread
  if (n > by_size) n = by_size;
  return n < 1 ? 1 : n;
}

std::string check_params(const ebic_params& p, int32_t ncols) {
  if (p.population < 1) return "population must be >= 1";
  if (p.archive_size < 1 || p.archive_size > 4096) return "archive_size must be in [1, 4096]";
  if (p.min_len < 1) return "min_len must be >= 1";
  if (p.max_init_len < p.min_len) return "max_init_len must be >= min_len";
  if (p.max_len < p.max_init_len) return "max_len must be >= max_init_len";
  if (p.max_len > (uint32_t)EBIC_MAX_CANDIDATE_LEN || (int64_t)p.max_len > ncols)
    return "max_len must be <= 64 and <= cols";
  if (p.elite > p.population) return "elite must be <= population";
  if (p.tournament < 1) return "tournament must be >= 1";
  if (!(p.p_crossover >= 0.f && p.p_crossover <= 1.f) ||
      !(p.p_mutation >= 0.f && p.p_mutation <= 1.f))
    return "probabilities must be in [0, 1]";
  if (!(p.overlap_threshold >= 0.f)) return "overlap_threshold must be >= 0";
  if (p.flags & ~(EBIC_NEGATIVE_TRENDS | EBIC_RUN_ON_DEVICE)) return "unknown flag";
  return "";
}

// The initial population: random candidates from the generator seeded with `seed`, a repeat
// drawn again (up to 32 times).
void initial_population(const ebic_params& p, int32_t ncols, std::vector<Cand>& pop,
                        std::vector<uint64_t>& pop_h) {
  Breeder ga(p, ncols);
  CandSet seen;
  pop.clear();
  pop_h.clear();
  for (uint32_t i = 0; i < p.population; ++i) {
    Cand c = ga.random_candidate();
    for (int t = 0; t < 32 && seen.count(c); ++t) c = ga.random_candidate();
    seen.insert(c);
    pop_h.push_back(CandHash()(c));
    pop.push_back(std::move(c));
  }
}

int run_ga(int64_t rows, int32_t ncols, const ebic_params& p, Evaluator& ev, ebic_result** out) {
  const uint32_t P = p.population, K = p.archive_size;
  Workers workers(breeding_threads(P));
  std::vector<Breeder> breeders;
  breeders.reserve(workers.size());
  for (unsigned w = 0; w < workers.size(); ++w) breeders.emplace_back(p, ncols);
  CandSet tabu, in_archive, picked;
  SlotSet in_next;  // the next population's sequences so far
  std::vector<Cand> pop;
  std::vector<uint64_t> pop_h;  // each candidate's CandHash, computed once
  pop.reserve(P);
  pop_h.reserve(P);
  initial_population(p, ncols, pop, pop_h);
  std::vector<Member> archive;
  std::vector<uint16_t> cols;
  std::vector<uint32_t> offs;
  std::vector<uint32_t> counts(P), overlaps((size_t)P * K), elites;
  std::vector<uint64_t> fitness(P), qual(P);
  struct SortKey {
    uint64_t fit, head4;
    uint32_t count, len, idx;
  };
  std::vector<SortKey> skeys(P), top_keys;  // skeys[i]: candidate i's order key
  std::vector<uint32_t> heap;
  heap.reserve(P);
  std::vector<Cand> kids;  // a generation's children before the pass in slot order
  std::vector<uint64_t> kids_h;
  std::vector<Rng> kids_rng;
  uint64_t evaluated = 0;
  uint32_t gen = 0;
  for (; gen < p.generations; ++gen) {
    cols.clear();
    offs.assign(1, 0u);
    for (const Cand& c : pop) {
      cols.insert(cols.end(), c.begin(), c.end());
      offs.push_back((uint32_t)cols.size());
    }
    int rc = ev.evaluate_begin(cols, offs, P, counts.data(), fitness.data(), overlaps.data());
    if (rc != EBIC_OK) return rc;
    for (uint32_t i = 0; i < P; ++i) tabu.insert(pop[i], pop_h[i]);  // while the GPU scores
    rc = ev.evaluate_end();
    if (rc != EBIC_OK) return rc;
    evaluated += P;
    const size_t K_eval = archive.size();  // overlaps is [P][K_eval]

    // The generation's order, best first: higher fitness, then more rows, longer, then the
    // lexicographically smaller sequence (equal-length sequences compare their first four columns
    // packed high to low, then the rest), then the lower index. It is a total order; tournaments
    // compare with it directly and only the `elite` best are sorted out.
    for (uint32_t i = 0; i < P; ++i) {
      uint64_t k = 0;
      for (size_t j = 0; j < 4; ++j) k = (k << 16) | (j < pop[i].size() ? pop[i][j] : 0u);
      skeys[i] = SortKey{fitness[i], k, counts[i], (uint32_t)pop[i].size(), i};
    }
    auto before = [&](const SortKey& a, const SortKey& b) {
      if (a.fit != b.fit) return a.fit > b.fit;
      if (a.count != b.count) return a.count > b.count;
      if (a.len != b.len) return a.len > b.len;
      if (a.head4 != b.head4) return a.head4 < b.head4;
      if (a.len > 4) {
        const Cand& ca = pop[a.idx];
        const Cand& cb = pop[b.idx];
        const auto ta = ca.begin() + 4, tb = cb.begin() + 4;
        if (!std::equal(ta, ca.end(), tb))
          return std::lexicographical_compare(ta, ca.end(), tb, cb.end());
      }
      return a.idx < b.idx;
    };
    {
      const uint32_t ne = std::min(p.elite, P);
      top_keys = skeys;
      std::partial_sort(top_keys.begin(), top_keys.begin() + ne, top_keys.end(), before);
      elites.resize(ne);
      for (uint32_t r = 0; r < ne; ++r) elites[r] = top_keys[r].idx;
    }

    // ---- archive update ----
    // Offer up to 2K non-archived candidates with rows, best raw quality first. A candidate is
    // admitted unless a member sharing a column overlaps it by more than the threshold without
    // being strictly worse; strictly worse members that overlap it that much are replaced.
    in_archive.clear();
    for (const Member& m : archive) in_archive.insert(m.cols);
    // the offers in member_before order (ties between equal sequences by population index):
    // candidates with rows popped from a heap until 2K distinct non-archived ones are taken, the
    // same as sorting all of them after dropping later duplicates
    std::vector<Member> offers;
    {
      for (uint32_t i = 0; i < P; ++i) qual[i] = quality(counts[i], pop[i].size());
      auto after = [&](uint32_t a, uint32_t b) {  // heap order: true when a comes after b
        if (qual[a] != qual[b]) return qual[a] < qual[b];
        if (counts[a] != counts[b]) return counts[a] < counts[b];
        if (pop[a].size() != pop[b].size()) return pop[a].size() < pop[b].size();
        if (pop[a] != pop[b]) return pop[b] < pop[a];
        return a > b;
      };
      heap.clear();
      for (uint32_t i = 0; i < P; ++i)
        if (counts[i] != 0) heap.push_back(i);
      std::make_heap(heap.begin(), heap.end(), after);
      picked.clear();
      while (!heap.empty() && offers.size() < 2 * (size_t)K) {
        std::pop_heap(heap.begin(), heap.end(), after);
        const uint32_t i = heap.back();
        heap.pop_back();
        if (in_archive.count(pop[i]) || picked.count(pop[i])) continue;
        picked.insert(pop[i]);
        offers.push_back(Member{pop[i], counts[i], qual[i], (int32_t)i});
      }
    }
    std::vector<uint32_t> top;
    for (const Member& m : offers) top.push_back((uint32_t)m.src);
    // their pairwise overlaps are computed while the next population is built (it depends on
    // neither the archive nor the overlaps, and the archive update draws no random numbers):
    // the host threads start breeding, then this thread issues the overlaps
    std::vector<Cand> next;
    std::vector<uint64_t> next_h;
    const bool breed = gen + 1 < p.generations;
    if (breed) {
      next.reserve(P);
      next_h.reserve(P);
      in_next.reset(P);
      for (uint32_t e : elites) {
        in_next.add((uint32_t)next.size(), pop_h[e]);
        next.push_back(pop[e]);
        next_h.push_back(pop_h[e]);
      }
      // the children of slots elite .. P-1, each from its own generator and against the tabu
      // list only (read-only here), in parallel
      const uint32_t n_child = P - (uint32_t)next.size();
      kids.resize(n_child);
      kids_h.resize(n_child);
      kids_rng.resize(n_child);
      const uint32_t slot0 = (uint32_t)next.size();
      workers.start(n_child, [&, slot0](uint32_t k, unsigned w) {
        Breeder& b = breeders[w];
        b.rng = child_stream(p.seed, gen, slot0 + k);
        auto tournament = [&]() {
          uint32_t best = b.rng.below(P);
          for (uint32_t t = 1; t < p.tournament; ++t) {
            const uint32_t c = b.rng.below(P);
            if (before(skeys[c], skeys[best])) best = c;
          }
          return best;
        };
        const uint32_t a = tournament();
        Cand child = pop[a];
        if (b.rng.unit() < p.p_crossover) child = b.crossover(pop[a], pop[tournament()]);
        if (b.rng.unit() < p.p_mutation) b.mutate(child);
        uint64_t h = CandHash()(child);
        for (uint32_t t = 0; t < p.tabu_retries && tabu.count(child, h); ++t) {
          b.mutate(child);
          h = CandHash()(child);
        }
        for (int t = 0; t < 32 && tabu.count(child, h); ++t) {
          child = b.random_candidate();
          h = CandHash()(child);
        }
        kids[k] = child;
        kids_h[k] = h;
        kids_rng[k] = b.rng;
      });
    }
    rc = ev.pair_overlaps_begin(top);
    if (breed) workers.finish();
    if (rc != EBIC_OK) return rc;
    if (breed) {
      const uint32_t n_child = (uint32_t)kids.size();
      // in slot order: a child that repeats one already in the new population is varied again
      // from its own generator, like a tabu child
      for (uint32_t k = 0; k < n_child; ++k) {
        Cand& child = kids[k];
        uint64_t h = kids_h[k];
        if (in_next.contains(child, h, next, next_h)) {
          Breeder& b = breeders[0];
          b.rng = kids_rng[k];
          auto taken = [&]() {
            return tabu.count(child, h) || in_next.contains(child, h, next, next_h);
          };
          for (uint32_t t = 0; t < p.tabu_retries && taken(); ++t) {
            b.mutate(child);
            h = CandHash()(child);
          }
          for (int t = 0; t < 32 && taken(); ++t) {
            child = b.random_candidate();
            h = CandHash()(child);
          }
        }
        in_next.add((uint32_t)next.size(), h);
        next_h.push_back(h);
        next.push_back(child);
      }
    }
    std::vector<uint32_t> pair((size_t)top.size() * top.size());
    rc = ev.pair_overlaps_end(pair.data());
    if (rc != EBIC_OK) return rc;
    std::vector<bool> alive(archive.size(), true);
    std::vector<size_t> admitted;  // positions in `offers`
    for (size_t t = 0; t < offers.size(); ++t) {
      const Member& c = offers[t];
      const uint32_t i = (uint32_t)c.src;
      const double limit = (double)p.overlap_threshold * (double)c.count;
      bool ok = true;
      std::vector<size_t> evict;
      for (size_t a = 0; a < K_eval && ok; ++a) {
        if (!alive[a] || !shares_column(c.cols, archive[a].cols)) continue;
        if ((double)overlaps[(size_t)i * K_eval + a] <= limit) continue;
        if (c.q > archive[a].q) evict.push_back(a); else ok = false;
      }
      for (size_t u : admitted) {  // admitted earlier: at least as good, never replaced here
        if (!ok) break;
        if (shares_column(c.cols, offers[u].cols) && (double)pair[t * top.size() + u] > limit)
          ok = false;
      }
      if (!ok) continue;
      for (size_t a : evict) alive[a] = false;
      admitted.push_back(t);
    }
    std::vector<Member> merged;
    for (size_t a = 0; a < archive.size(); ++a) {
      if (!alive[a]) continue;
      Member m = archive[a];
      m.src = -(int32_t)a - 1;
      merged.push_back(m);
    }
    for (size_t t : admitted) merged.push_back(offers[t]);
    std::stable_sort(merged.begin(), merged.end(), member_before);
    if (merged.size() > K) merged.resize(K);
    std::vector<int32_t> src;
    for (const Member& m : merged) src.push_back(m.src);
    rc = ev.set_archive(src);
    if (rc != EBIC_OK) return rc;
    archive = merged;

    if (gen + 1 == p.generations) { ++gen; break; }
    pop.swap(next);  // the next population, built above
    pop_h.swap(next_h);
  }

  // ---- result ----
  ebic_result* r = new ebic_result();
  std::memset(r, 0, sizeof(*r));
  r->n = (uint32_t)archive.size();
  r->words = (rows + 31) / 32;
  r->generations_run = gen;
  r->candidates_evaluated = evaluated;
  size_t tot = 0;
  for (const Member& m : archive) tot += m.cols.size();
  r->cols = new uint16_t[tot > 0 ? tot : 1];
  r->offsets = new uint32_t[r->n + 1];
  r->counts = new uint32_t[r->n > 0 ? r->n : 1];
  r->quality = new uint64_t[r->n > 0 ? r->n : 1];
  r->offsets[0] = 0;
  size_t o = 0;
  for (uint32_t i = 0; i < r->n; ++i) {
    std::copy(archive[i].cols.begin(), archive[i].cols.end(), r->cols + o);
    o += archive[i].cols.size();
    r->offsets[i + 1] = (uint32_t)o;
    r->counts[i] = archive[i].count;
    r->quality[i] = archive[i].q;
  }
  if (ev.has_bitmaps()) {
    r->bitmaps = new uint32_t[(size_t)r->n * (size_t)r->words + 1];
    int rc = ev.archive_bitmaps(r->bitmaps, r->n);
    if (rc != EBIC_OK) {
      ebic_free_result(r);
      return rc;
    }
  }
  *out = r;
  return EBIC_OK;
}

// ---- scoring by caller callbacks ---------------------------------------------------------------
struct CallbackEvaluator : Evaluator {
  const ebic_evaluator* cb;
  explicit CallbackEvaluator(const ebic_evaluator* c) : cb(c) {}
  int evaluate(const std::vector<uint16_t>& cols, const std::vector<uint32_t>& offs, uint32_t n,
               uint32_t* counts, uint64_t* fitness, uint32_t* overlaps) override {
    int rc = cb->evaluate(cb->user, cols.data(), offs.data(), n, counts, fitness, overlaps);
    return rc == 0 ? EBIC_OK : set_last_error(EBIC_ERR_INVALID_ARG, "evaluate callback failed");
  }
  int pair_overlaps(const std::vector<uint32_t>& idx, uint32_t* out) override {
    int rc = cb->pair_overlaps(cb->user, idx.data(), (uint32_t)idx.size(), out);
    return rc == 0 ? EBIC_OK : set_last_error(EBIC_ERR_INVALID_ARG, "pair_overlaps callback failed");
  }
  int set_archive(const std::vector<int32_t>& src) override {
    int rc = cb->set_archive(cb->user, src.data(), (uint32_t)src.size());
    return rc == 0 ? EBIC_OK : set_last_error(EBIC_ERR_INVALID_ARG, "set_archive callback failed");
  }
};

// ---- scoring on the GPU: device-resident bitmaps and archive ------------------------------------
#define GA_CUDA(expr)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      (void)cudaGetLastError();                                                          \
      return set_last_error(e_ == cudaErrorMemoryAllocation ? EBIC_ERR_OOM : EBIC_ERR_CUDA, \
                            (std::string(#expr) + ": " + cudaGetErrorString(e_)).c_str()); \
    }                                                                                    \
  } while (0)

struct GpuEvaluator : Evaluator {
  const ebic_matrix* m;
  cudaStream_t s;
  uint32_t flags, P, K, T, max_len;
  int64_t W;
  std::vector<void*> allocs;
  uint16_t *dcols = nullptr, *acols = nullptr, *pcols = nullptr;
  uint32_t *doffs = nullptr, *dcounts = nullptr, *dbm = nullptr, *dov = nullptr;
  uint32_t *aoffs = nullptr, *abm = nullptr, *abm_next = nullptr;
  uint32_t *poffs = nullptr, *pcounts = nullptr, *pbm = nullptr, *pov = nullptr;
  uint64_t *dfit = nullptr, *pfit = nullptr;
  int32_t* didx = nullptr;  // rows to gather (population index, or -(archive index + 1))
  // the offers' lists, staged in pinned memory and sent in one copy to a device block of the
  // same layout: gather indices [T], columns [T * max_len], offsets [T + 1], counts [T]
  char *hstage = nullptr, *dstage = nullptr;
  size_t st_cols = 0, st_offs = 0, st_cnt = 0, st_bytes = 0;
  uint32_t* hpov = nullptr;  // pinned [T][T]: the pair overlaps' copy-back
  uint32_t pending_t = 0;
  // pinned copy-backs of a generation's scores, and where evaluate_end puts them
  uint32_t *hcnt = nullptr, *hov = nullptr;
  uint64_t* hfit = nullptr;
  uint32_t *out_counts = nullptr, *out_overlaps = nullptr;
  uint64_t* out_fitness = nullptr;
  uint32_t out_n = 0, out_k = 0;
  std::vector<uint16_t> pop_cols, arch_cols;
  std::vector<uint32_t> pop_offs, arch_offs{0}, host_counts;
  uint32_t n_arch = 0;

  GpuEvaluator(const ebic_matrix* mm, cudaStream_t st, const ebic_params& p, int64_t words)
      : m(mm), s(st), flags(p.flags & EBIC_NEGATIVE_TRENDS), P(p.population), K(p.archive_size),
        T(2 * p.archive_size), max_len(p.max_len), W(words) {}
  ~GpuEvaluator() override {
    cudaStreamSynchronize(s);
    for (void* a : allocs) cudaFree(a);
    if (hpov) cudaFreeHost(hpov);
    if (hstage) cudaFreeHost(hstage);
    if (hcnt) cudaFreeHost(hcnt);
    if (hfit) cudaFreeHost(hfit);
    if (hov) cudaFreeHost(hov);
  }
  template <class X>
  cudaError_t alloc(X** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (n ? n : 1) * sizeof(X));
    if (e == cudaSuccess) allocs.push_back(v);
    *p = static_cast<X*>(v);
    return e;
  }
  int init() {
    GA_CUDA(alloc(&dcols, (size_t)P * max_len));
    GA_CUDA(alloc(&doffs, (size_t)P + 1));
    GA_CUDA(alloc(&dcounts, P));
    GA_CUDA(alloc(&dbm, (size_t)P * W));
    GA_CUDA(alloc(&dfit, P));
    GA_CUDA(alloc(&dov, (size_t)P * K));
    GA_CUDA(alloc(&acols, (size_t)K * max_len));
    GA_CUDA(alloc(&aoffs, (size_t)K + 1));
    GA_CUDA(alloc(&abm, (size_t)K * W));
    GA_CUDA(alloc(&abm_next, (size_t)K * W));
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    st_cols = up16((size_t)T * 4);
    st_offs = st_cols + up16((size_t)T * max_len * 2);
    st_cnt = st_offs + up16(((size_t)T + 1) * 4);
    st_bytes = st_cnt + up16((size_t)T * 4);
    GA_CUDA(alloc(&dstage, st_bytes));
    GA_CUDA(cudaMallocHost(&hstage, st_bytes));
    pcols = reinterpret_cast<uint16_t*>(dstage + st_cols);
    poffs = reinterpret_cast<uint32_t*>(dstage + st_offs);
    pcounts = reinterpret_cast<uint32_t*>(dstage + st_cnt);
    GA_CUDA(alloc(&pbm, (size_t)T * W));
    GA_CUDA(alloc(&pfit, T));
    GA_CUDA(alloc(&pov, (size_t)T * T));
    GA_CUDA(alloc(&didx, (size_t)std::max(T, K)));
    GA_CUDA(cudaMallocHost(&hpov, (size_t)std::max(T, 1u) * std::max(T, 1u) * 4));
    GA_CUDA(cudaMallocHost(&hcnt, (size_t)P * 4));
    GA_CUDA(cudaMallocHost(&hfit, (size_t)P * 8));
    GA_CUDA(cudaMallocHost(&hov, (size_t)P * std::max(K, 1u) * 4));
    return EBIC_OK;
  }
  int evaluate(const std::vector<uint16_t>& cols, const std::vector<uint32_t>& offs, uint32_t n,
               uint32_t* counts, uint64_t* fitness, uint32_t* overlaps) override {
    int rc = evaluate_begin(cols, offs, n, counts, fitness, overlaps);
    return rc != EBIC_OK ? rc : evaluate_end();
  }
  int evaluate_end() override {
    GA_CUDA(cudaStreamSynchronize(s));
    std::memcpy(out_counts, hcnt, (size_t)out_n * 4);
    std::memcpy(out_fitness, hfit, (size_t)out_n * 8);
    if (out_k) std::memcpy(out_overlaps, hov, (size_t)out_n * out_k * 4);
    host_counts.assign(out_counts, out_counts + out_n);
    return ebic_matrix_status(const_cast<ebic_matrix*>(m), s);
  }
  int evaluate_begin(const std::vector<uint16_t>& cols, const std::vector<uint32_t>& offs,
                     uint32_t n, uint32_t* counts, uint64_t* fitness,
                     uint32_t* overlaps) override {
    pop_cols = cols;
    pop_offs = offs;
    // pageable-source copies return once the source is staged
    GA_CUDA(cudaMemcpyAsync(dcols, cols.data(), cols.size() * 2, cudaMemcpyHostToDevice, s));
    GA_CUDA(cudaMemcpyAsync(doffs, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice, s));
    // one generation's scoring in one call: with a pair table on the matrix, the evaluation and
    // the archive overlaps run as one pass (the bitmaps are still written: the archive update
    // needs the offered candidates' rows)
    int rc = ebic_eval_fitness(m, dcols, doffs, n, flags, acols, aoffs, abm, n_arch, dcounts, dbm,
                               dfit, n_arch ? dov : nullptr, s);
    if (rc != EBIC_OK) return rc;
    GA_CUDA(cudaMemcpyAsync(hcnt, dcounts, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GA_CUDA(cudaMemcpyAsync(hfit, dfit, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    if (n_arch)
      GA_CUDA(cudaMemcpyAsync(hov, dov, (size_t)n * n_arch * 4, cudaMemcpyDeviceToHost, s));
    out_counts = counts;
    out_fitness = fitness;
    out_overlaps = overlaps;
    out_n = n;
    out_k = n_arch;
    return EBIC_OK;
  }
  int pair_overlaps(const std::vector<uint32_t>& idx, uint32_t* out) override {
    int rc = pair_overlaps_begin(idx);
    return rc != EBIC_OK ? rc : pair_overlaps_end(out);
  }
  int pair_overlaps_end(uint32_t* out) override {
    GA_CUDA(cudaStreamSynchronize(s));
    std::memcpy(out, hpov, (size_t)pending_t * pending_t * 4);
    return EBIC_OK;
  }
  int pair_overlaps_begin(const std::vector<uint32_t>& idx) override {
    const uint32_t t = (uint32_t)idx.size();
    pending_t = t;
    if (t == 0) return EBIC_OK;
    // the staging block is free: the previous generation's copy completed before its
    // pair_overlaps_end returned
    int32_t* hi = reinterpret_cast<int32_t*>(hstage);
    uint16_t* hc = reinterpret_cast<uint16_t*>(hstage + st_cols);
    uint32_t* ho = reinterpret_cast<uint32_t*>(hstage + st_offs);
    uint32_t* hn = reinterpret_cast<uint32_t*>(hstage + st_cnt);
    ho[0] = 0;
    for (uint32_t k = 0; k < t; ++k) {
      const uint32_t i = idx[k];
      hi[k] = (int32_t)i;
      const uint32_t b = pop_offs[i], e = pop_offs[i + 1];
      std::copy(pop_cols.begin() + b, pop_cols.begin() + e, hc + ho[k]);
      ho[k + 1] = ho[k] + (e - b);
      hn[k] = host_counts[i];
    }
    GA_CUDA(cudaMemcpyAsync(dstage, hstage, st_bytes, cudaMemcpyHostToDevice, s));
    GA_CUDA(launch_gather_rows(dbm, dbm, reinterpret_cast<const int32_t*>(dstage), t, W, pbm, s));
    int rc = ebic_fitness(m, pcols, poffs, t, pcounts, pbm, pcols, poffs, pbm, t, 0, pfit, pov, s);
    if (rc != EBIC_OK) return rc;
    GA_CUDA(cudaMemcpyAsync(hpov, pov, (size_t)t * t * 4, cudaMemcpyDeviceToHost, s));
    // the lists were built here, valid by construction; a device-side rejection would still
    // show in the sticky status word that the next evaluation reads
    return EBIC_OK;
  }
  int set_archive(const std::vector<int32_t>& src) override {
    std::vector<uint16_t> c;
    std::vector<uint32_t> o{0};
    for (size_t k = 0; k < src.size(); ++k) {
      if (src[k] >= 0) {
        const uint32_t i = (uint32_t)src[k];
        c.insert(c.end(), pop_cols.begin() + pop_offs[i], pop_cols.begin() + pop_offs[i + 1]);
      } else {
        const uint32_t a = (uint32_t)(-src[k] - 1);
        c.insert(c.end(), arch_cols.begin() + arch_offs[a], arch_cols.begin() + arch_offs[a + 1]);
      }
      o.push_back((uint32_t)c.size());
    }
    // the new archive's rows, gathered from the population's and the old archive's bitmaps
    if (!src.empty()) {
      GA_CUDA(cudaMemcpyAsync(didx, src.data(), src.size() * 4, cudaMemcpyHostToDevice, s));
      GA_CUDA(launch_gather_rows(dbm, abm, didx, (uint32_t)src.size(), W, abm_next, s));
    }
    std::swap(abm, abm_next);
    arch_cols = c;
    arch_offs = o;
    n_arch = (uint32_t)src.size();
    if (!c.empty())
      GA_CUDA(cudaMemcpyAsync(acols, c.data(), c.size() * 2, cudaMemcpyHostToDevice, s));
    GA_CUDA(cudaMemcpyAsync(aoffs, o.data(), o.size() * 4, cudaMemcpyHostToDevice, s));
    return EBIC_OK;  // stream-ordered before the next evaluation; sources already staged
  }
  bool has_bitmaps() const override { return true; }
  int archive_bitmaps(uint32_t* out, uint32_t k) override {
    if (k) GA_CUDA(cudaMemcpyAsync(out, abm, (size_t)k * W * 4, cudaMemcpyDeviceToHost, s));
    GA_CUDA(cudaStreamSynchronize(s));
    return EBIC_OK;
  }
};

}  // namespace

extern "C" {

int ebic_params_default(ebic_params* p) {
  if (!p) return set_last_error(EBIC_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->population = 1600;
  p->generations = 100;
  p->archive_size = 20;
  p->elite = 16;
  p->tournament = 4;
  p->min_len = 2;
  p->max_init_len = 6;
  p->max_len = 64;
  p->p_crossover = 0.5f;
  p->p_mutation = 0.7f;
  p->overlap_threshold = 0.5f;
  p->tabu_retries = 8;
  p->flags = 0;
  p->seed = 1807099320ull;
  return EBIC_OK;
}

int ebic_run_custom(int64_t rows, int32_t cols, const ebic_params* p, const ebic_evaluator* ev,
                    ebic_result** out) {
  if (!p || !ev || !out || !ev->evaluate || !ev->pair_overlaps || !ev->set_archive)
    return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (rows < 1 || cols < 1 || cols > EBIC_MAX_COLS)
    return set_last_error(EBIC_ERR_INVALID_ARG, "rows/cols out of range");
  std::string why = check_params(*p, cols);
  if (!why.empty()) return set_last_error(EBIC_ERR_INVALID_ARG, why.c_str());
  if (p->flags & EBIC_RUN_ON_DEVICE)
    return set_last_error(EBIC_ERR_UNSUPPORTED, "EBIC_RUN_ON_DEVICE is for ebic_run");
  try {
    CallbackEvaluator e(ev);
    return run_ga(rows, cols, *p, e, out);
  } catch (const std::bad_alloc&) {
    return set_last_error(EBIC_ERR_OOM, "host allocation failed");
  }
}

int ebic_run(const ebic_matrix* m, const ebic_params* p, void* stream, ebic_result** out) {
  if (!m || !p || !out) return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  MatrixView v;
  matrix_view(m, &v);
  if (v.total_rows != v.L.rows)
    return set_last_error(EBIC_ERR_UNSUPPORTED,
                          "ebic_run scores the whole matrix; this matrix is one row shard of it");
  std::string why = check_params(*p, v.L.cols);
  if (!why.empty()) return set_last_error(EBIC_ERR_INVALID_ARG, why.c_str());
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { (void)cudaGetLastError(); prev = -1; }
  if (prev != v.device) (void)cudaSetDevice(v.device);
  int rc;
  try {
    if (p->flags & EBIC_RUN_ON_DEVICE) {
      std::vector<Cand> pop;
      std::vector<uint64_t> pop_h;
      initial_population(*p, v.L.cols, pop, pop_h);
      std::vector<uint16_t> c((size_t)p->population * kMaxLen, 0);
      std::vector<uint32_t> n(p->population);
      for (uint32_t i = 0; i < p->population; ++i) {
        n[i] = (uint32_t)pop[i].size();
        std::copy(pop[i].begin(), pop[i].end(), c.begin() + (size_t)i * kMaxLen);
      }
      rc = run_ga_on_device(m, v.L.rows, v.L.cols, v.L.words, *p,
                            static_cast<cudaStream_t>(stream), c.data(), n.data(), pop_h.data(),
                            out);
    } else {
      GpuEvaluator e(m, static_cast<cudaStream_t>(stream), *p, v.L.words);
      rc = e.init();
      if (rc == EBIC_OK) rc = run_ga(v.L.rows, v.L.cols, *p, e, out);
    }
  } catch (const std::bad_alloc&) {
    rc = set_last_error(EBIC_ERR_OOM, "host allocation failed");
  }
  if (prev >= 0 && prev != v.device) (void)cudaSetDevice(prev);
  return rc;
}

int ebic_free_result(ebic_result* r) {
  if (!r) return EBIC_OK;
  delete[] r->cols;
  delete[] r->offsets;
  delete[] r->counts;
  delete[] r->quality;
  delete[] r->bitmaps;
  delete r;
  return EBIC_OK;
}

}  // extern "C"
