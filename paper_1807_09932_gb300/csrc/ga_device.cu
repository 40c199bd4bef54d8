// The EBIC generation loop on the device: ebic_run with EBIC_RUN_ON_DEVICE.
//
// The loop is the host loop of ga.cpp, decision for decision, with no host round trip per
// generation. Its definition (the operators, the per-child generators, the tabu list, the
// slot-order handling of duplicate children, the archive rule) is the one ga.cpp states; every
// decision depends only on draws and exact integer scores, so the device loop's archive equals
// the host loop's bit for bit (the GPU tests compare them). The mapping:
//   * scoring: ebic_eval_fitness on device lists, against the archive padded to K members with
//     empty ones (one column, no rows: a member without rows never penalises a candidate);
//   * the tabu list: an exact set of the evaluated sequences (open addressing on their FNV-1a
//     hash, the sequences kept in an arena), filled by a thread per candidate;
//   * the generation's order and the order of the archive offers: each candidate's rank counted
//     by a warp (the orders are total), then elites and offers read off the ranks;
//   * breeding: a thread per child, from the child's own generator, against the tabu list;
//   * duplicate children: a table of the new population's sequences holds each sequence's first
//     slot (atomicMin); one warp then walks the slots in order and re-varies the (rare) children
//     whose sequence an earlier slot holds, exactly as the host's slot-order pass does;
//   * the archive update: one warp, offers in order, a lane per archive member or admitted offer.
// Supported: archive_size <= 32 (offers <= 64), columns <= EBIC_MAX_COLS; other runs use the host
// loop (the call reports EBIC_ERR_UNSUPPORTED when the flag asks for the device loop).
#include <cstring>
#include <string>
#include <vector>

#include "ebic.h"
#include "ebic_internal.h"

namespace ebic {
namespace gadev {

constexpr uint32_t kMaxArch = 32;             // archive members in the device loop
constexpr uint32_t kMaxOffers = 2 * kMaxArch;
constexpr int kSetWords = (EBIC_MAX_COLS + 31) / 32;  // a column set as a bitmask

// ---- generators and candidates (the same arithmetic as the host loop) ------------------------
struct Rng {  // splitmix64 (Steele, Lea, Flood 2014)
  uint64_t s;
  __device__ uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  __device__ uint32_t below(uint32_t n) { return (uint32_t)(next() % n); }
  __device__ double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

__device__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ Rng child_stream(uint64_t seed, uint32_t gen, uint32_t slot) {
  return Rng{mix64(mix64(seed + 0x9E3779B97F4A7C15ull * ((uint64_t)gen + 1)) + slot)};
}

struct Cand {
  uint32_t n;
  uint16_t c[kMaxLen];
};

__device__ uint64_t cand_hash(const uint16_t* c, uint32_t n) {  // FNV-1a, then the length
  uint64_t h = 1469598103934665603ull;
  for (uint32_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h ^ (uint64_t)n;
}

__device__ bool contains_col(const Cand& c, uint16_t x) {
  for (uint32_t i = 0; i < c.n; ++i)
    if (c.c[i] == x) return true;
  return false;
}

__device__ bool seq_equal(const uint16_t* a, uint32_t na, const uint16_t* b, uint32_t nb) {
  if (na != nb) return false;
  for (uint32_t i = 0; i < na; ++i)
    if (a[i] != b[i]) return false;
  return true;
}

// Sequences in device memory sit at 128-byte strides (kMaxLen columns): they are read as 16-byte
// chunks, all of a sequence's chunks issued before any is used, instead of one column at a time.
constexpr int kChunks = kMaxLen / 8;
__device__ void load_chunks(const uint16_t* g, uint32_t n, uint4 (&v)[kChunks]) {
  const uint4* p = reinterpret_cast<const uint4*>(g);
#pragma unroll
  for (int k = 0; k < kChunks; ++k) v[k] = (uint32_t)(8 * k) < n ? p[k] : make_uint4(0, 0, 0, 0);
}
__device__ uint16_t chunk_col(const uint4 (&v)[kChunks], uint32_t i) {
  const uint4 w = v[i >> 3];
  const uint32_t j = i & 7, x = (j >> 1) == 0 ? w.x : (j >> 1) == 1 ? w.y : (j >> 1) == 2 ? w.z : w.w;
  return (uint16_t)((j & 1) ? (x >> 16) : (x & 0xFFFFu));
}
// the sequence at g (device memory, 16-byte aligned) equals c
__device__ bool equal_global(const uint16_t* g, uint32_t ng, const uint16_t* c, uint32_t n) {
  if (ng != n) return false;
  uint4 v[kChunks];
  load_chunks(g, n, v);
  for (uint32_t i = 0; i < n; ++i)
    if (chunk_col(v, i) != c[i]) return false;
  return true;
}

// a < b lexicographically (a proper prefix is smaller)
__device__ bool seq_less(const uint16_t* a, uint32_t na, const uint16_t* b, uint32_t nb) {
  const uint32_t n = na < nb ? na : nb;
  for (uint32_t i = 0; i < n; ++i)
    if (a[i] != b[i]) return a[i] < b[i];
  return na < nb;
}

struct Ops {  // the run's parameters the operators read
  uint32_t P, min_len, max_init_len, max_len, tournament, tabu_retries, elite;
  int32_t ncols;
  float p_crossover, p_mutation;
  uint64_t seed;
};

// A column not in c: uniform draws, as on the host; after kUnusedDraws misses (both loops have
// the same bound) the smallest unused column.
__device__ uint16_t unused_column(const Ops& o, Rng& r, const Cand& c) {
  for (uint32_t t = 0; t < kUnusedDraws; ++t) {
    const uint16_t x = (uint16_t)r.below((uint32_t)o.ncols);
    if (!contains_col(c, x)) return x;
  }
  for (int32_t x = 0; x < o.ncols; ++x)
    if (!contains_col(c, (uint16_t)x)) return (uint16_t)x;
  return 0;  // unreachable: callers ensure c.n < ncols
}

// L distinct columns by a partial Fisher-Yates shuffle of 0 .. ncols-1, the touched positions
// kept in a small map (the host shuffles a full list and restores it)
__device__ void random_candidate(const Ops& o, Rng& r, Cand& out) {
  const uint32_t L = o.min_len + r.below(o.max_init_len - o.min_len + 1);
  uint32_t pos[2 * kMaxLen], val[2 * kMaxLen];
  uint32_t nm = 0;
  auto get = [&](uint32_t p) {
    for (uint32_t k = 0; k < nm; ++k)
      if (pos[k] == p) return val[k];
    return p;
  };
  auto set = [&](uint32_t p, uint32_t v) {
    for (uint32_t k = 0; k < nm; ++k)
      if (pos[k] == p) {
        val[k] = v;
        return;
      }
    pos[nm] = p;
    val[nm] = v;
    ++nm;
  };
  for (uint32_t i = 0; i < L; ++i) {
    const uint32_t j = i + r.below((uint32_t)o.ncols - i);
    const uint32_t vi = get(i), vj = get(j);
    set(i, vj);
    set(j, vi);
  }
  out.n = L;
  for (uint32_t i = 0; i < L; ++i) out.c[i] = (uint16_t)get(i);
}

__device__ void crossover(const Ops& o, Rng& r, const Cand& a, const Cand& b, Cand& child) {
  const uint32_t cut = 1 + r.below(a.n);
  child.n = cut;
  for (uint32_t i = 0; i < cut; ++i) child.c[i] = a.c[i];
  for (uint32_t i = 0; i < b.n; ++i) {
    if (child.n >= o.max_len) break;
    if (!contains_col(child, b.c[i])) child.c[child.n++] = b.c[i];
  }
  while (child.n < o.min_len) {
    const uint16_t x = unused_column(o, r, child);
    child.c[child.n++] = x;
  }
}

__device__ void mutate(const Ops& o, Rng& r, Cand& c) {
  const uint32_t first = r.below(4);
  for (uint32_t k = 0; k < 4; ++k) {
    switch ((first + k) % 4) {
      case 0:  // swap two positions
        if (c.n >= 2) {
          const uint32_t i = r.below(c.n);
          uint32_t j = r.below(c.n - 1);
          if (j >= i) ++j;
          const uint16_t t = c.c[i];
          c.c[i] = c.c[j];
          c.c[j] = t;
          return;
        }
        break;
      case 1:  // substitute a column by an unused one
        if ((int32_t)c.n < o.ncols) {
          const uint32_t i = r.below(c.n);
          c.c[i] = unused_column(o, r, c);
          return;
        }
        break;
      case 2:  // insert an unused column
        if (c.n < o.max_len && (int32_t)c.n < o.ncols) {
          const uint16_t x = unused_column(o, r, c);
          const uint32_t i = r.below(c.n + 1);
          for (uint32_t m = c.n; m > i; --m) c.c[m] = c.c[m - 1];
          c.c[i] = x;
          ++c.n;
          return;
        }
        break;
      default:  // delete a column
        if (c.n > o.min_len) {
          const uint32_t i = r.below(c.n);
          for (uint32_t m = i; m + 1 < c.n; ++m) c.c[m] = c.c[m + 1];
          --c.n;
          return;
        }
        break;
    }
  }
}

// ---- populations: fixed-stride sequences ------------------------------------------------------
struct Pop {
  uint16_t* c;   // [n][kMaxLen]
  uint32_t* n;   // [n] lengths
  uint64_t* h;   // [n] CandHash
};

__device__ void load_cand(const Pop& p, uint32_t i, Cand& out) {
  out.n = p.n[i];
  uint4 v[kChunks];
  load_chunks(p.c + (size_t)i * kMaxLen, out.n, v);
  for (uint32_t k = 0; k < out.n; ++k) out.c[k] = chunk_col(v, k);
}
__device__ void store_cand(const Pop& p, uint32_t i, const Cand& c, uint64_t h) {
  p.n[i] = c.n;
  for (uint32_t k = 0; k < c.n; ++k) p.c[(size_t)i * kMaxLen + k] = c.c[k];
  p.h[i] = h;
}

// ---- an exact set of sequences (the tabu list) -------------------------------------------------
struct SeqSet {
  // slot: the hash's high 32 bits (a tag) << 32 | entry + 1; 0 = empty; mask + 1 slots, at most
  // half used. A probe that meets no equal tag costs one load.
  unsigned long long* slots;
  uint64_t mask;
  uint32_t* ent_n;
  uint16_t* arena;   // entry e's sequence at arena + e * kMaxLen
  uint32_t* n_ent;
};

__device__ uint64_t spread(uint64_t h) {
  h ^= h >> 33;
  h *= 0xFF51AFD7ED558CCDull;
  h ^= h >> 33;
  return h;
}

__device__ bool set_contains(const SeqSet& s, const uint16_t* c, uint32_t n, uint64_t h) {
  const uint32_t tag = (uint32_t)(h >> 32);
  uint64_t i = spread(h) & s.mask;
  for (uint64_t k = 0; k <= s.mask; ++k, i = (i + 1) & s.mask) {
    const unsigned long long v = *reinterpret_cast<volatile const unsigned long long*>(s.slots + i);
    if (v == 0) return false;
    const uint32_t e = (uint32_t)v;
    if ((uint32_t)(v >> 32) == tag &&
        equal_global(s.arena + (size_t)(e - 1) * kMaxLen, s.ent_n[e - 1], c, n))
      return true;
  }
  return false;
}

// Inserts a sequence that is not in the set; concurrent inserts of distinct sequences are safe.
__device__ void set_insert(const SeqSet& s, const uint16_t* c, uint32_t n, uint64_t h) {
  const uint32_t e = atomicAdd(s.n_ent, 1u);
  s.ent_n[e] = n;
  for (uint32_t k = 0; k < n; ++k) s.arena[(size_t)e * kMaxLen + k] = c[k];
  __threadfence();  // the entry is complete before a slot points to it
  const unsigned long long v = ((unsigned long long)(uint32_t)(h >> 32) << 32) | (e + 1u);
  uint64_t i = spread(h) & s.mask;
  for (uint64_t k = 0; k <= s.mask; ++k, i = (i + 1) & s.mask)
    if (atomicCAS(s.slots + i, 0ull, v) == 0ull) return;
}

// ---- kernels -----------------------------------------------------------------------------------
// the evaluated population joins the tabu list (its sequences are distinct)
__global__ void tabu_insert_kernel(SeqSet tabu, Pop pop, uint32_t P) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const uint32_t n = pop.n[i];
  const uint16_t* c = pop.c + (size_t)i * kMaxLen;
  if (!set_contains(tabu, c, n, pop.h[i])) set_insert(tabu, c, n, pop.h[i]);
}

struct OrderArgs {
  Pop pop;
  uint32_t P, elite;
  const uint64_t* fitness;
  const uint32_t* counts;
  uint32_t* rank;          // [P] position in the generation's order
  uint32_t* elites;        // [elite]
  uint32_t* offer_sorted;  // [P] candidates with rows in the offer order
  uint32_t* n_offerable;   // zeroed before the launch
};

__device__ uint64_t quality_of(uint32_t n, uint32_t L) {
  return (uint64_t)n << ((L < 33u ? L : 33u) - 1u);
}

// The generation's order: higher fitness, more rows, longer, lexicographically smaller, lower
// index. The offer order (candidates with rows): higher quality, more rows, longer,
// lexicographically smaller, lower index. A warp counts the candidates before its own.
__global__ void order_kernel(OrderArgs a) {
  const uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= a.P) return;
  const uint64_t fi = a.fitness[i];
  const uint32_t ci = a.counts[i], li = a.pop.n[i];
  const uint64_t qi = quality_of(ci, li);
  const uint16_t* si = a.pop.c + (size_t)i * kMaxLen;
  uint32_t nb = 0, no = 0;
  for (uint32_t j = lane; j < a.P; j += 32) {
    if (j == i) continue;
    const uint64_t fj = a.fitness[j];
    const uint32_t cj = a.counts[j], lj = a.pop.n[j];
    const uint16_t* sj = a.pop.c + (size_t)j * kMaxLen;
    bool b;  // j before i in the generation's order
    if (fj != fi) b = fj > fi;
    else if (cj != ci) b = cj > ci;
    else if (lj != li) b = lj > li;
    else if (!seq_equal(sj, lj, si, li)) b = seq_less(sj, lj, si, li);
    else b = j < i;
    nb += b;
    if (ci != 0 && cj != 0) {
      const uint64_t qj = quality_of(cj, lj);
      bool o;  // j before i in the offer order
      if (qj != qi) o = qj > qi;
      else if (cj != ci) o = cj > ci;
      else if (lj != li) o = lj > li;
      else if (!seq_equal(sj, lj, si, li)) o = seq_less(sj, lj, si, li);
      else o = j < i;
      no += o;
    }
  }
  nb = __reduce_add_sync(0xFFFFFFFFu, nb);
  no = __reduce_add_sync(0xFFFFFFFFu, no);
  if (lane == 0) {
    a.rank[i] = nb;
    if (nb < a.elite) a.elites[nb] = i;
    if (ci != 0) {
      a.offer_sorted[no] = i;
      atomicAdd(a.n_offerable, 1u);
    }
  }
}

struct Archive {  // members in order; `size` of them real, the rest (to K) empty
  uint16_t* c;     // [K][kMaxLen]
  uint32_t* n;     // [K]
  uint32_t* count; // [K]
  uint64_t* q;     // [K]
  uint32_t* size;  // [1]
  uint16_t* csr_cols;  // the padded list the scoring reads: [K * kMaxLen]
  uint32_t* csr_offs;  // [K + 1]
};

// Up to 2K offers: candidates with rows in the offer order, skipping archived sequences. One
// warp; lane a holds archive member a's hash.
__global__ void offers_kernel(Pop pop, const uint32_t* offer_sorted, const uint32_t* n_offerable,
                              Archive arch, uint32_t T, uint32_t* offers, uint32_t* n_offers) {
  __shared__ uint64_t ah[kMaxArch];
  __shared__ uint64_t oh[kMaxOffers];
  const int lane = threadIdx.x;
  const uint32_t ka = *arch.size;
  if (lane < (int)ka) ah[lane] = cand_hash(arch.c + (size_t)lane * kMaxLen, arch.n[lane]);
  __syncwarp();
  const uint32_t no = *n_offerable;
  uint32_t t = 0;
  // candidate r = base + lane is skipped when its sequence is archived, already offered, or held
  // by an earlier candidate of the same 32 (a population can repeat a sequence when its retries
  // ran out); the others are taken in order
  for (uint32_t base = 0; base < no && t < T; base += 32) {
    const uint32_t r = base + lane;
    bool take = false;
    uint32_t i = 0;
    uint64_t h = 0;
    const uint16_t* c = nullptr;
    uint32_t n = 0;
    if (r < no) {
      i = offer_sorted[r];
      h = pop.h[i];
      c = pop.c + (size_t)i * kMaxLen;
      n = pop.n[i];
      take = true;
      for (uint32_t a = 0; a < ka && take; ++a)
        if (ah[a] == h && seq_equal(arch.c + (size_t)a * kMaxLen, arch.n[a], c, n)) take = false;
      for (uint32_t k = 0; k < t && take; ++k)
        if (oh[k] == h && seq_equal(pop.c + (size_t)offers[k] * kMaxLen, pop.n[offers[k]], c, n))
          take = false;
    }
    for (int k = 0; k < 31; ++k) {  // an earlier candidate of the same 32 with this sequence
      const uint64_t hk = __shfl_sync(0xFFFFFFFFu, h, k);
      const uint32_t ik = __shfl_sync(0xFFFFFFFFu, i, k);
      if (k < lane && take && base + k < no && hk == h &&
          seq_equal(pop.c + (size_t)ik * kMaxLen, pop.n[ik], c, n))
        take = false;
    }
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, take);
    const uint32_t before = __popc(m & ((1u << lane) - 1u));
    if (take && t + before < T) {
      offers[t + before] = i;
      oh[t + before] = h;
    }
    __syncwarp();
    t += __popc(m);
    if (t > T) t = T;
  }
  __syncwarp();
  if (lane == 0) *n_offers = t;
}

// pair[t][u] = popcount(M_t & M_u) for offers u < t < n_offers, from the population's bitmaps:
// each CTA takes a contiguous range of words, stages the offers' words of a 128-word chunk in
// shared memory (rows padded to 129 words), and a thread per pair accumulates over its chunks;
// one atomic per pair and CTA.
constexpr int kOvChunk = 128;
__global__ void __launch_bounds__(256) offer_overlap_kernel(const uint32_t* __restrict__ bm,
                                                            int64_t W, const uint32_t* offers,
                                                            const uint32_t* n_offers, uint32_t T,
                                                            uint32_t* pair) {
  __shared__ uint32_t rowsw[kMaxOffers][kOvChunk + 1];
  __shared__ uint32_t idx[kMaxOffers];
  const uint32_t nt = *n_offers;
  if (nt < 2) return;
  for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) idx[t] = offers[t];
  const uint32_t n_pairs = nt * (nt - 1) / 2;
  const int64_t per = (W + gridDim.x - 1) / gridDim.x;
  const int64_t w0 = (int64_t)blockIdx.x * per, w1 = w0 + per < W ? w0 + per : W;
  constexpr int kPairsPerThread = (kMaxOffers * (kMaxOffers - 1) / 2 + 255) / 256;
  uint32_t acc[kPairsPerThread];
#pragma unroll
  for (int k = 0; k < kPairsPerThread; ++k) acc[k] = 0;
  for (int64_t c0 = w0; c0 < w1; c0 += kOvChunk) {
    const int cw = (int)(w1 - c0 < kOvChunk ? w1 - c0 : kOvChunk);
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nt * kOvChunk; k += blockDim.x) {
      const uint32_t t = k / kOvChunk, w = k % kOvChunk;
      rowsw[t][w] = (int)w < cw ? __ldg(bm + (size_t)idx[t] * W + c0 + w) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPairsPerThread; ++k) {
      const uint32_t pr = threadIdx.x + 256u * k;
      if (pr >= n_pairs) continue;
      // pr -> (t, u), u < t: t is the largest with t (t - 1) / 2 <= pr
      uint32_t t = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)pr)) * 0.5f);
      while (t * (t - 1) / 2 > pr) --t;
      while ((t + 1) * t / 2 <= pr) ++t;
      const uint32_t u = pr - t * (t - 1) / 2;
      uint32_t a = 0;
      for (int w = 0; w < cw; ++w) a += __popc(rowsw[t][w] & rowsw[u][w]);
      acc[k] += a;
    }
  }
#pragma unroll
  for (int k = 0; k < kPairsPerThread; ++k) {
    const uint32_t pr = threadIdx.x + 256u * k;
    if (pr >= n_pairs || acc[k] == 0) continue;
    uint32_t t = (uint32_t)((1.0f + sqrtf(1.0f + 8.0f * (float)pr)) * 0.5f);
    while (t * (t - 1) / 2 > pr) --t;
    while ((t + 1) * t / 2 <= pr) ++t;
    const uint32_t u = pr - t * (t - 1) / 2;
    atomicAdd(pair + (size_t)t * T + u, acc[k]);
  }
}

struct BreedArgs {
  Ops o;
  const uint32_t* gen;  // the generation number (device memory, so a captured graph replays)
  Pop pop, next;
  const uint32_t* rank;
  const uint32_t* elites;
  SeqSet tabu;
  Rng* kid_rng;  // [P - elite]
};

// The next population: slots 0 .. elite-1 the elites, then a thread per child, from the child's
// own generator, against the tabu list only.
__global__ void breed_kernel(BreedArgs a) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  const Ops& o = a.o;
  if (s >= o.P) return;
  Cand child;
  if (s < o.elite) {
    const uint32_t e = a.elites[s];
    load_cand(a.pop, e, child);
    store_cand(a.next, s, child, a.pop.h[e]);
    return;
  }
  Rng r = child_stream(o.seed, *a.gen, s);
  auto tournament = [&]() {
    uint32_t best = r.below(o.P);
    for (uint32_t t = 1; t < o.tournament; ++t) {
      const uint32_t c = r.below(o.P);
      if (a.rank[c] < a.rank[best]) best = c;
    }
    return best;
  };
  const uint32_t pa = tournament();
  load_cand(a.pop, pa, child);
  if (r.unit() < (double)o.p_crossover) {
    const uint32_t pb = tournament();
    Cand A, B;
    load_cand(a.pop, pa, A);
    load_cand(a.pop, pb, B);
    crossover(o, r, A, B, child);
  }
  if (r.unit() < (double)o.p_mutation) mutate(o, r, child);
  uint64_t h = cand_hash(child.c, child.n);
  for (uint32_t t = 0; t < o.tabu_retries && set_contains(a.tabu, child.c, child.n, h); ++t) {
    mutate(o, r, child);
    h = cand_hash(child.c, child.n);
  }
  for (int t = 0; t < 32 && set_contains(a.tabu, child.c, child.n, h); ++t) {
    random_candidate(o, r, child);
    h = cand_hash(child.c, child.n);
  }
  store_cand(a.next, s, child, h);
  a.kid_rng[s - o.elite] = r;
}

// The new population's table: each sequence's first slot (slot + 1; 0 = empty).
struct SlotTable {
  uint32_t* v;
  uint64_t mask;
};

__device__ uint64_t table_find(const SlotTable& t, const Pop& next, const uint16_t* c, uint32_t n,
                               uint64_t h, bool& found) {
  uint64_t i = spread(h) & t.mask;
  for (uint64_t k = 0; k <= t.mask; ++k, i = (i + 1) & t.mask) {
    const uint32_t v = t.v[i];
    if (v == 0) {
      found = false;
      return i;
    }
    const uint32_t s = v - 1;
    if (next.h[s] == h && equal_global(next.c + (size_t)s * kMaxLen, next.n[s], c, n)) {
      found = true;
      return i;
    }
  }
  found = false;
  return ~0ull;  // unreachable: the table is at most half full
}

__global__ void first_slot_kernel(SlotTable t, Pop next, uint32_t P) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  const uint64_t h = next.h[s];
  const uint32_t n = next.n[s];
  const uint16_t* c = next.c + (size_t)s * kMaxLen;
  uint64_t i = spread(h) & t.mask;
  for (uint64_t k = 0; k <= t.mask; ++k, i = (i + 1) & t.mask) {
    uint32_t v = atomicCAS(t.v + i, 0u, s + 1);
    if (v == 0) return;  // claimed an empty slot
    // an equal sequence only ever meets its equals here: keep the lowest slot
    const uint32_t o = v - 1;
    if (next.h[o] == h && equal_global(next.c + (size_t)o * kMaxLen, next.n[o], c, n)) {
      atomicMin(t.v + i, s + 1);
      return;
    }
  }
}

__global__ void dup_flag_kernel(SlotTable t, Pop next, uint32_t P, uint32_t elite, uint8_t* dup) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  if (s < elite) {  // elites are kept as they are, repeats included (as on the host)
    dup[s] = 0;
    return;
  }
  bool found;
  const uint64_t i = table_find(t, next, next.c + (size_t)s * kMaxLen, next.n[s], next.h[s], found);
  dup[s] = (found && t.v[i] != s + 1) ? 1 : 0;
}

// Duplicate children, in two phases with the host pass's result.
// Phase A (a thread per duplicate slot s): the slot's retry chain from its own generator, with a
// sequence taken when it is tabu or first held (in the breeding's result) by a slot before s.
// Every sequence the host pass would take is so taken, except one that an earlier duplicate slot
// took as its replacement. The result's first slot in the table is kept: if it is after s, taking
// the sequence makes that slot a duplicate.
struct Spec {
  Pop seq;         // the phase-A result per slot
  int32_t* disp;   // [P] the later slot it displaces, or -1
};

__device__ bool first_before(const SlotTable& t, const Pop& next, const uint16_t* c, uint32_t n,
                             uint64_t h, uint32_t s, int32_t* later) {
  bool f;
  const uint64_t i = table_find(t, next, c, n, h, f);
  if (later) *later = (f && t.v[i] - 1 > s) ? (int32_t)(t.v[i] - 1) : -1;
  return f && t.v[i] - 1 < s;
}

constexpr uint32_t kInSpec = 0x80000000u;  // accepted-list slot flag: sequence in the phase-A buffer

__device__ const uint16_t* accepted_seq(uint32_t slot_flag, const Pop& next, const Pop& spec,
                                        uint32_t& n) {
  const uint32_t s = slot_flag & ~kInSpec;
  const Pop& p = (slot_flag & kInSpec) ? spec : next;
  n = p.n[s];
  return p.c + (size_t)s * kMaxLen;
}

__device__ void retry_chain(const Ops& o, Rng& r, Cand& child, uint64_t& h, const SeqSet& tabu,
                            const SlotTable& t, const Pop& next, uint32_t s,
                            const uint64_t* acc_h, const uint32_t* acc_slot, uint32_t n_acc,
                            const Pop& spec) {
  auto taken = [&]() {
    if (set_contains(tabu, child.c, child.n, h)) return true;
    if (first_before(t, next, child.c, child.n, h, s, nullptr)) return true;
    for (uint32_t k = 0; k < n_acc; ++k)  // replacements taken by earlier slots (phase B)
      if (acc_h[k] == h) {
        uint32_t na;
        const uint16_t* ca = accepted_seq(acc_slot[k], next, spec, na);
        if (equal_global(ca, na, child.c, child.n)) return true;
      }
    return false;
  };
  for (uint32_t k = 0; k < o.tabu_retries && taken(); ++k) {
    mutate(o, r, child);
    h = cand_hash(child.c, child.n);
  }
  for (int k = 0; k < 32 && taken(); ++k) {
    random_candidate(o, r, child);
    h = cand_hash(child.c, child.n);
  }
}

__global__ void spec_kernel(Ops o, SlotTable t, Pop next, SeqSet tabu, const Rng* kid_rng,
                            const uint8_t* dup, Spec sp) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < o.elite || s >= o.P || !dup[s]) return;
  Cand child;
  load_cand(next, s, child);
  uint64_t h = next.h[s];
  Rng r = kid_rng[s - o.elite];
  retry_chain(o, r, child, h, tabu, t, next, s, nullptr, nullptr, 0, next);
  store_cand(sp.seq, s, child, h);
  int32_t later;
  first_before(t, next, child.c, child.n, h, s, &later);
  sp.disp[s] = later;
}

// Phase B (one warp, slots in order): a duplicate slot takes its phase-A result unless an earlier
// slot took the same replacement, in which case (and for a slot that a replacement displaced) lane
// 0 runs the chain again with the replacements taken so far counted as taken. The replacements
// are kept in shared memory (up to kAccMax; a longer list is read from the population itself).
constexpr uint32_t kAccMax = 1024;
constexpr uint32_t kFlagsMax = 16384;  // duplicate flags kept in shared memory up to this population
constexpr uint32_t kListMax = 512;     // duplicate slots walked from a list up to this many
constexpr uint32_t kExtraMax = 256;    // displaced slots waiting in the side list
__global__ void settle_kernel(Ops o, SlotTable t, Pop next, SeqSet tabu, const Rng* kid_rng,
                              uint8_t* dup_g, Spec sp, uint32_t* acc_slot_g, uint64_t* acc_h_g) {
  __shared__ uint64_t acc_h[kAccMax];
  __shared__ uint32_t acc_slot[kAccMax];
  __shared__ uint8_t dup_s[kFlagsMax];
  const int lane = threadIdx.x;
  const bool in_smem = o.P <= kFlagsMax;
  uint8_t* dup = in_smem ? dup_s : dup_g;
  if (in_smem) {  // 16 flags per load (the flag buffers are padded to 16 bytes)
    const uint32_t nv = (o.P + 15) / 16;
#pragma unroll 4
    for (uint32_t k = lane; k < nv; k += 32)
      reinterpret_cast<uint4*>(dup_s)[k] = reinterpret_cast<const uint4*>(dup_g)[k];
  }
  __syncwarp();
  uint32_t n_acc = 0;
  // Slot s (kind 1: phase A ran, with its key h_j, length n_j and displacement disp_j; kind 2:
  // displaced during this walk): the whole warp calls this; returns the slot it displaces, or -1.
  auto settle_slot = [&](uint32_t s, uint8_t kind, uint64_t h_j, uint32_t n_j,
                         int32_t disp_j) -> int32_t {
    // does the phase-A result repeat a replacement taken before?
    bool clash = false;
    if (kind == 1) {
      for (uint32_t k = lane; k < n_acc; k += 32) {
        const uint64_t ah = k < kAccMax ? acc_h[k] : acc_h_g[k];
        if (ah != h_j) continue;
        const uint32_t as = k < kAccMax ? acc_slot[k] : acc_slot_g[k];
        uint32_t na;
        const uint16_t* ca = accepted_seq(as, next, sp.seq, na);
        if (seq_equal(ca, na, sp.seq.c + (size_t)s * kMaxLen, n_j)) clash = true;
      }
      clash = __any_sync(0xFFFFFFFFu, clash);
    }
    int32_t displaced = -1;
    uint64_t h_acc = h_j;
    uint32_t slot_acc = s | kInSpec;
    if (kind == 1 && !clash) {
      displaced = disp_j;  // the phase-A result stands; copied into place after the walk
    } else if (lane == 0) {
      Cand child;
      load_cand(next, s, child);
      uint64_t h = next.h[s];
      Rng r = kid_rng[s - o.elite];
      retry_chain(o, r, child, h, tabu, t, next, s, n_acc <= kAccMax ? acc_h : acc_h_g,
                  n_acc <= kAccMax ? acc_slot : acc_slot_g, n_acc, sp.seq);
      first_before(t, next, child.c, child.n, h, s, &displaced);
      store_cand(next, s, child, h);
      dup[s] = 3;  // settled here: no copy from the phase-A buffer
      h_acc = h;
      slot_acc = s;
    }
    h_acc = __shfl_sync(0xFFFFFFFFu, h_acc, 0);
    slot_acc = __shfl_sync(0xFFFFFFFFu, slot_acc, 0);
    displaced = __shfl_sync(0xFFFFFFFFu, displaced, 0);
    if (lane == 0) {
      if (n_acc < kAccMax) {
        acc_h[n_acc] = h_acc;
        acc_slot[n_acc] = slot_acc;
      }
      acc_h_g[n_acc] = h_acc;
      acc_slot_g[n_acc] = slot_acc;
    }
    ++n_acc;
    __syncwarp();
    return displaced;
  };
  // the duplicate slots in order, compacted from the flags (shared memory), their phase-A keys
  // loaded together; slots displaced on the way are merged from a small side list
  __shared__ uint32_t list[kListMax];
  __shared__ uint64_t list_h[kListMax];
  __shared__ uint32_t list_n[kListMax];
  __shared__ int32_t list_d[kListMax];
  __shared__ uint32_t extra[kExtraMax];
  uint32_t count = 0;
  uint32_t walk_from = o.elite;
  if (in_smem) {
    for (uint32_t base = o.elite; base < o.P; base += 32) {
      const uint32_t s0 = base + lane;
      const bool d = s0 < o.P && dup[s0] == 1;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, d);
      const uint32_t pos = count + __popc(m & ((1u << lane) - 1u));
      if (d && pos < kListMax) list[pos] = s0;
      count += __popc(m);
    }
  }
  __syncwarp();
  if (in_smem && count <= kListMax) {
#pragma unroll 4
    for (uint32_t k = lane; k < count; k += 32) {
      const uint32_t s0 = list[k];
      list_h[k] = sp.seq.h[s0];
      list_n[k] = sp.seq.n[s0];
      list_d[k] = sp.disp[s0];
    }
    uint32_t n_extra = 0;  // displaced slots not settled yet (unordered; usually none)
    uint32_t i = 0;
    bool overflow = false;
    uint32_t resume = o.P;  // after an overflow: the slot the window walk resumes from
    __syncwarp();
    while (i < count || n_extra > 0) {
      // the next slot: the list's next one or the smallest displaced one
      uint32_t e_min = 0xFFFFFFFFu, e_at = 0;
      for (uint32_t k = lane; k < n_extra; k += 32)
        if (extra[k] < e_min) {
          e_min = extra[k];
          e_at = k;
        }
      for (int d = 16; d > 0; d >>= 1) {
        const uint32_t om = __shfl_xor_sync(0xFFFFFFFFu, e_min, d);
        const uint32_t oa = __shfl_xor_sync(0xFFFFFFFFu, e_at, d);
        if (om < e_min) {
          e_min = om;
          e_at = oa;
        }
      }
      const uint32_t l_next = i < count ? list[i] : 0xFFFFFFFFu;
      int32_t displaced;
      uint32_t cur;
      if (l_next < e_min) {
        cur = l_next;
        displaced = settle_slot(l_next, 1, list_h[i], list_n[i], list_d[i]);
        ++i;
      } else {
        cur = e_min;
        if (lane == 0) extra[e_at] = extra[n_extra - 1];
        --n_extra;
        __syncwarp();
        displaced = settle_slot(e_min, 2, 0, 0, -1);
      }
      // a displaced slot's own sequence is now held by an earlier slot: settled in turn
      if (displaced >= 0 && dup[displaced] != 2) {
        if (lane == 0) {
          dup[displaced] = 2;
          if (n_extra < kExtraMax) extra[n_extra] = (uint32_t)displaced;
        }
        if (n_extra < kExtraMax) ++n_extra;
        else overflow = true;
      }
      __syncwarp();
      if (overflow) {  // every slot up to cur is settled; the rest are flagged 1 or 2
        resume = cur + 1;
        break;
      }
    }
    if (!overflow) {
      __syncwarp();
      if (in_smem) {
        const uint32_t nv = (o.P + 15) / 16;
        for (uint32_t k = lane; k < nv; k += 32)
          reinterpret_cast<uint4*>(dup_g)[k] = reinterpret_cast<const uint4*>(dup_s)[k];
      }
      return;
    }
    // more displaced slots than the side list holds: the window walk below settles the slots
    // after `resume` in order (the flags say which: 1 or 2)
    walk_from = resume;
  }
  // the window walk: every slot in order, the window's phase-A keys one slot per lane
  for (uint32_t base = walk_from; base < o.P; base += 32) {
    __syncwarp();
    const uint32_t s0 = base + lane;
    uint32_t mask = __ballot_sync(0xFFFFFFFFu, s0 < o.P && (dup[s0] == 1 || dup[s0] == 2));
    if (!mask) continue;
    uint64_t my_h = 0;
    uint32_t my_n = 0;
    int32_t my_disp = -1;
    if (s0 < o.P && dup[s0] == 1) {
      my_h = sp.seq.h[s0];
      my_n = sp.seq.n[s0];
      my_disp = sp.disp[s0];
    }
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t s = base + (uint32_t)j;
      const uint8_t kind = dup[s];
      const uint64_t h_j = __shfl_sync(0xFFFFFFFFu, my_h, j);
      const int32_t disp_j = __shfl_sync(0xFFFFFFFFu, my_disp, j);
      const uint32_t n_j = __shfl_sync(0xFFFFFFFFu, my_n, j);
      const int32_t displaced = settle_slot(s, kind, h_j, n_j, disp_j);
      if (displaced >= 0) {
        if (lane == 0) dup[displaced] = 2;
        __syncwarp();
        if (displaced >= (int32_t)base && displaced < (int32_t)(base + 32))
          mask |= 1u << (uint32_t)(displaced - (int32_t)base);
      }
    }
  }
  __syncwarp();
  if (in_smem) {  // the flags back: 1 marks a phase-A result that stood (copied by the next kernel)
    const uint32_t nv = (o.P + 15) / 16;
    for (uint32_t k = lane; k < nv; k += 32)
      reinterpret_cast<uint4*>(dup_g)[k] = reinterpret_cast<const uint4*>(dup_s)[k];
  }
}

// The phase-A results that stood, copied into the population: a thread per slot.
__global__ void commit_spec_kernel(uint32_t P, uint32_t elite, const uint8_t* dup, Spec sp,
                                   Pop next) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P || s < elite || dup[s] != 1) return;
  uint4 v[kChunks];
  const uint32_t n = sp.seq.n[s];
  if (n > (uint32_t)kMaxLen) return;  // never: phase A wrote this slot
  load_chunks(sp.seq.c + (size_t)s * kMaxLen, n, v);
  uint4* dst = reinterpret_cast<uint4*>(next.c + (size_t)s * kMaxLen);
  for (uint32_t k = 0; 8 * k < n; ++k) dst[k] = v[k];
  next.n[s] = n;
  next.h[s] = sp.seq.h[s];
}

__global__ void next_generation_kernel(uint32_t* gen) { ++*gen; }

// The next population as the list the scoring reads.
__global__ void pack_kernel(Pop pop, uint32_t P, uint16_t* cols, uint32_t* offs) {
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < P; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t n = i < P ? pop.n[i] : 0u;
    // block-wide exclusive scan of the lengths
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = n;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    __shared__ uint32_t wsum[32];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
        if (lane >= d) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const uint32_t start = carry + (warp ? wsum[warp - 1] : 0u) + x - n;
    if (i < P) {
      offs[i] = start;
      for (uint32_t k = 0; k < n; ++k) cols[start + k] = pop.c[(size_t)i * kMaxLen + k];
      if (i == P - 1) offs[P] = start + n;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = start + n;
    __syncthreads();
  }
}

struct AdmitArgs {
  Pop pop;
  uint32_t P, K, T;
  uint32_t set_words;         // (columns + 31) / 32: the words of a column set in use
  float threshold;
  const uint32_t* counts;
  const uint32_t* overlaps;   // [P][K] the population against the archive (padded to K)
  const uint32_t* pair;       // [T][T] the offers among themselves
  const uint32_t* offers;
  const uint32_t* n_offers;
  Archive cur, nxt;
  int32_t* gather_src;        // [K] rows of the new archive: population i, or -(a + 1)
};

// The archive update, one warp: offers in order; a lane per archive member, then per admitted
// offer; then the merged list ranked by the member order and cut to K.
__global__ void admit_kernel(AdmitArgs a) {
  __shared__ uint32_t oset[kMaxOffers][kSetWords], aset[kMaxArch][kSetWords];
  __shared__ uint32_t adm[kMaxOffers];
  __shared__ uint32_t alive_mask;
  // what the offers loop reads, loaded up front by all lanes
  __shared__ uint32_t s_off[kMaxOffers], s_cnt[kMaxOffers], s_ov[kMaxOffers][kMaxArch];
  __shared__ uint64_t s_q[kMaxOffers], s_aq[kMaxArch];
  __shared__ uint32_t s_pair[kMaxOffers][kMaxOffers];
  const int lane = threadIdx.x;
  const uint32_t ka = *a.cur.size, nt = *a.n_offers;
  for (uint32_t t = lane; t < nt; t += 32) {
    const uint32_t i = a.offers[t];
    s_off[t] = i;
    s_cnt[t] = a.counts[i];
    s_q[t] = quality_of(s_cnt[t], a.pop.n[i]);
  }
  if (lane < (int)ka) s_aq[lane] = a.cur.q[lane];
  __syncwarp();
#pragma unroll 8
  for (uint32_t k = lane; k < nt * ka; k += 32) {
    const uint32_t t = k / ka, m = k % ka;
    s_ov[t][m] = a.overlaps[(size_t)s_off[t] * a.K + m];
  }
#pragma unroll 8
  for (uint32_t k = lane; k < nt * nt; k += 32) {
    const uint32_t t = k / nt, u = k % nt;
    s_pair[t][u] = u < t ? a.pair[(size_t)t * a.T + u] : 0u;
  }
  for (uint32_t k = lane; k < kMaxOffers * kSetWords; k += 32) (&oset[0][0])[k] = 0u;
  for (uint32_t k = lane; k < kMaxArch * kSetWords; k += 32) (&aset[0][0])[k] = 0u;
  __syncwarp();
  for (uint32_t t = lane; t < nt; t += 32) {
    const uint32_t i = s_off[t];
    const uint32_t n = a.pop.n[i];
    uint4 v[kChunks];
    load_chunks(a.pop.c + (size_t)i * kMaxLen, n, v);
    for (uint32_t k = 0; k < n; ++k) {
      const uint16_t x = chunk_col(v, k);
      oset[t][x >> 5] |= 1u << (x & 31);
    }
  }
  if (lane < (int)ka) {
    const uint32_t n = a.cur.n[lane];
    uint4 v[kChunks];
    load_chunks(a.cur.c + (size_t)lane * kMaxLen, n, v);
    for (uint32_t k = 0; k < n; ++k) {
      const uint16_t x = chunk_col(v, k);
      aset[lane][x >> 5] |= 1u << (x & 31);
    }
  }
  __syncwarp();
  const uint32_t nsw = a.set_words;
  auto shares = [nsw](const uint32_t* x, const uint32_t* y) {
    uint32_t any = 0;
    for (uint32_t w = 0; w < nsw; ++w) any |= x[w] & y[w];
    return any != 0;
  };
  uint32_t alive = ka >= 32 ? 0xFFFFFFFFu : ((1u << ka) - 1u);
  uint32_t n_adm = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    const uint32_t cnt = s_cnt[t];
    const uint64_t q = s_q[t];
    const double limit = (double)a.threshold * (double)cnt;
    bool block = false, evict = false;
    if (lane < (int)ka && ((alive >> lane) & 1u) && shares(oset[t], aset[lane]) &&
        (double)s_ov[t][lane] > limit) {
      if (q > s_aq[lane]) evict = true;
      else block = true;
    }
    bool blocked = __any_sync(0xFFFFFFFFu, block);
    if (!blocked) {
      bool b2 = false;
      for (uint32_t u = lane; u < n_adm; u += 32) {
        const uint32_t tu = adm[u];
        if (shares(oset[t], oset[tu]) && (double)s_pair[t][tu] > limit) b2 = true;
      }
      blocked = __any_sync(0xFFFFFFFFu, b2);
    }
    if (!blocked) {
      alive &= ~__ballot_sync(0xFFFFFFFFu, evict);
      if (lane == 0) adm[n_adm] = t;
      ++n_adm;
      __syncwarp();
    }
  }
  if (lane == 0) alive_mask = alive;
  __syncwarp();
  // the merged list: alive members, then admitted offers; item x's position is the number of
  // items before it in the member order (quality, rows, length, sequence: all distinct)
  const uint32_t n_items = ka + n_adm;  // alive members are among the first ka
  auto item = [&](uint32_t x, const uint16_t*& c, uint32_t& n, uint32_t& cnt, uint64_t& q,
                  int32_t& src) {
    if (x < ka) {
      c = a.cur.c + (size_t)x * kMaxLen;
      n = a.cur.n[x];
      cnt = a.cur.count[x];
      q = a.cur.q[x];
      src = -(int32_t)x - 1;
    } else {
      const uint32_t i = a.offers[adm[x - ka]];
      c = a.pop.c + (size_t)i * kMaxLen;
      n = a.pop.n[i];
      cnt = a.counts[i];
      q = quality_of(cnt, n);
      src = (int32_t)i;
    }
  };
  auto live = [&](uint32_t x) { return x >= ka || ((alive_mask >> x) & 1u); };
  // the items' keys, loaded once
  __shared__ uint64_t m_q[kMaxArch + kMaxOffers];
  __shared__ uint32_t m_cnt[kMaxArch + kMaxOffers], m_n[kMaxArch + kMaxOffers];
  for (uint32_t x = lane; x < n_items; x += 32) {
    const uint16_t* cx;
    int32_t srcx;
    item(x, cx, m_n[x], m_cnt[x], m_q[x], srcx);
  }
  __syncwarp();
  uint32_t n_new = 0;
  for (uint32_t x = 0; x < n_items; ++x) n_new += live(x);
  n_new = n_new < a.K ? n_new : a.K;
  // every row's source starts as the zero row (the items are distinct, so every position below
  // n_new is then written; this only keeps the gather in bounds whatever happens)
  for (uint32_t r = lane; r < a.K; r += 32) a.gather_src[r] = -(int32_t)a.K - 1;
  __syncwarp();
  for (uint32_t x = lane; x < n_items; x += 32) {
    if (!live(x)) continue;
    const uint16_t* cx;
    uint32_t nx, cntx;
    uint64_t qx;
    int32_t srcx;
    item(x, cx, nx, cntx, qx, srcx);
    uint32_t pos = 0;
    for (uint32_t y = 0; y < n_items; ++y) {
      if (y == x || !live(y)) continue;
      bool before;
      if (m_q[y] != qx) before = m_q[y] > qx;
      else if (m_cnt[y] != cntx) before = m_cnt[y] > cntx;
      else if (m_n[y] != nx) before = m_n[y] > nx;
      else {  // the same quality, rows and length: the sequences decide
        const uint16_t* cy;
        uint32_t ny, cnty;
        uint64_t qy;
        int32_t srcy;
        item(y, cy, ny, cnty, qy, srcy);
        before = seq_less(cy, ny, cx, nx);
      }
      pos += before;
    }
    if (pos < a.K) {
      uint4 v[kChunks];
      load_chunks(cx, nx, v);
      uint4* dst = reinterpret_cast<uint4*>(a.nxt.c + (size_t)pos * kMaxLen);
      for (uint32_t k = 0; 8 * k < nx; ++k) dst[k] = v[k];
      a.nxt.n[pos] = nx;
      a.nxt.count[pos] = cntx;
      a.nxt.q[pos] = qx;
      a.gather_src[pos] = srcx;
    }
  }
  __syncwarp();
  // empty members to K: one column, no rows (the zero row after the K bitmap rows)
  for (uint32_t r = n_new + lane; r < a.K; r += 32) {
    a.nxt.c[(size_t)r * kMaxLen] = 0;
    a.nxt.n[r] = 1;
    a.nxt.count[r] = 0;
    a.nxt.q[r] = 0;
    a.gather_src[r] = -(int32_t)a.K - 1;
  }
  __syncwarp();
  // the padded list the scoring reads: member r = lane's offsets by a warp prefix sum (K <= 32),
  // its columns copied by its lane
  if (lane == 0) *a.nxt.size = n_new;
  {
    const uint32_t r = (uint32_t)lane;
    const uint32_t n = r < a.K ? a.nxt.n[r] : 0u;
    uint32_t x = n;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    const uint32_t start = x - n;
    if (r < a.K) {
      a.nxt.csr_offs[r] = start;
      uint4 v[kChunks];
      load_chunks(a.nxt.c + (size_t)r * kMaxLen, n, v);
      for (uint32_t k = 0; k < n; ++k) a.nxt.csr_cols[start + k] = chunk_col(v, k);
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
    if (lane == 0) a.nxt.csr_offs[a.K] = total;
  }
}

}  // namespace gadev
}  // namespace ebic

// ---- the host side of the device loop -----------------------------------------------------------
namespace ebic {
namespace {

#define GD_CUDA(expr)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      (void)cudaGetLastError();                                                            \
      return set_last_error(e_ == cudaErrorMemoryAllocation ? EBIC_ERR_OOM : EBIC_ERR_CUDA,  \
                            (std::string(#expr) + ": " + cudaGetErrorString(e_)).c_str()); \
    }                                                                                      \
  } while (0)

struct DeviceBuffers {
  std::vector<void*> all;
  ~DeviceBuffers() {
    for (void* p : all) cudaFree(p);
  }
  template <class X>
  cudaError_t get(X** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (n ? n : 1) * sizeof(X));
    if (e == cudaSuccess) all.push_back(v);
    *p = static_cast<X*>(v);
    return e;
  }
};

uint64_t pow2_at_least(uint64_t x) {
  uint64_t c = 64;
  while (c < x) c <<= 1;
  return c;
}

}  // namespace

namespace {
// The loop's own stream (it can be captured into a graph, which the legacy default stream cannot),
// started after the caller's stream's pending work; released when the run returns.
struct RunStream {
  cudaStream_t s = nullptr, s2 = nullptr;  // s2: the branch that runs beside s within a generation
  cudaEvent_t e = nullptr;
  cudaEvent_t fork0 = nullptr, tabu_done = nullptr, fork1 = nullptr, archive_done = nullptr;
  ~RunStream() {
    for (cudaStream_t x : {s, s2})
      if (x) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
      }
    for (cudaEvent_t x : {e, fork0, tabu_done, fork1, archive_done})
      if (x) cudaEventDestroy(x);
  }
};
}  // namespace

int run_ga_on_device(const ebic_matrix* m, int64_t rows, int32_t ncols, int64_t W,
                     const ebic_params& p, cudaStream_t caller, const uint16_t* init_cols,
                     const uint32_t* init_n, const uint64_t* init_h, ebic_result** out) {
  using namespace gadev;
  DeviceBuffers b;  // freed after the stream below is drained (declared first, destroyed last)
  RunStream rs;
  GD_CUDA(cudaStreamCreateWithFlags(&rs.s, cudaStreamNonBlocking));
  GD_CUDA(cudaStreamCreateWithFlags(&rs.s2, cudaStreamNonBlocking));
  for (cudaEvent_t* x : {&rs.e, &rs.fork0, &rs.tabu_done, &rs.fork1, &rs.archive_done})
    GD_CUDA(cudaEventCreateWithFlags(x, cudaEventDisableTiming));
  GD_CUDA(cudaEventRecord(rs.e, caller));
  GD_CUDA(cudaStreamWaitEvent(rs.s, rs.e, 0));
  cudaStream_t s = rs.s, s2 = rs.s2;
  const uint32_t P = p.population, K = p.archive_size, T = 2 * K, G = p.generations;
  if (K > kMaxArch)
    return set_last_error(EBIC_ERR_UNSUPPORTED, "the device loop takes archive_size <= 32");
  const uint32_t eflags = p.flags & EBIC_NEGATIVE_TRENDS;
  const uint64_t cap_e = (uint64_t)P * (G + 1);  // every evaluated sequence, at most
  const uint64_t cap_t = pow2_at_least(2 * cap_e), cap_n = pow2_at_least(2 * (uint64_t)P);
  if (cap_e >= 0xFFFFFFFFull)
    return set_last_error(EBIC_ERR_UNSUPPORTED, "population x generations too large for the device loop");
  int num_sms = 0;
  {
    int dev = 0;
    GD_CUDA(cudaGetDevice(&dev));
    GD_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  Pop pop, nxt;
  GD_CUDA(b.get(&pop.c, (size_t)P * kMaxLen));
  GD_CUDA(b.get(&pop.n, P));
  GD_CUDA(b.get(&pop.h, P));
  GD_CUDA(b.get(&nxt.c, (size_t)P * kMaxLen));
  GD_CUDA(b.get(&nxt.n, P));
  GD_CUDA(b.get(&nxt.h, P));
  uint16_t* dcols;
  uint32_t *doffs, *dcounts, *dov, *dbm, *rank, *elites, *offer_sorted, *n_offerable, *offers,
      *n_offers, *pov;
  uint64_t* dfit;
  int32_t* gather_src;
  Rng* kid_rng;
  uint8_t* dup;
  GD_CUDA(b.get(&dcols, (size_t)P * kMaxLen));
  GD_CUDA(b.get(&doffs, (size_t)P + 1));
  GD_CUDA(b.get(&dcounts, P));
  GD_CUDA(b.get(&dfit, P));
  GD_CUDA(b.get(&dov, (size_t)P * K));
  GD_CUDA(b.get(&dbm, (size_t)P * W));
  GD_CUDA(b.get(&rank, P));
  GD_CUDA(b.get(&elites, p.elite));
  GD_CUDA(b.get(&offer_sorted, P));
  GD_CUDA(b.get(&n_offerable, 1));
  GD_CUDA(b.get(&offers, T));
  GD_CUDA(b.get(&n_offers, 1));
  GD_CUDA(b.get(&pov, (size_t)T * T));
  GD_CUDA(b.get(&kid_rng, P));
  GD_CUDA(b.get(&dup, ((size_t)P + 15) / 16 * 16));
  GD_CUDA(cudaMemsetAsync(dup, 0, ((size_t)P + 15) / 16 * 16, s));
  Spec spec;
  GD_CUDA(b.get(&spec.seq.c, (size_t)P * kMaxLen));
  GD_CUDA(b.get(&spec.seq.n, P));
  GD_CUDA(b.get(&spec.seq.h, P));
  GD_CUDA(b.get(&spec.disp, P));
  uint32_t* acc_slot;
  uint64_t* acc_h;
  GD_CUDA(b.get(&acc_slot, P));
  GD_CUDA(b.get(&acc_h, P));
  SlotTable table;
  table.mask = cap_n - 1;
  GD_CUDA(b.get(&table.v, cap_n));
  SeqSet tabu;
  tabu.mask = cap_t - 1;
  GD_CUDA(b.get(&tabu.slots, cap_t));
  GD_CUDA(b.get(&tabu.ent_n, cap_e));
  GD_CUDA(b.get(&tabu.arena, cap_e * kMaxLen));
  GD_CUDA(b.get(&tabu.n_ent, 1));
  Archive arch[2];
  uint32_t* abm[2];
  for (int k = 0; k < 2; ++k) {
    GD_CUDA(b.get(&arch[k].c, (size_t)K * kMaxLen));
    GD_CUDA(b.get(&arch[k].n, K));
    GD_CUDA(b.get(&arch[k].count, K));
    GD_CUDA(b.get(&arch[k].q, K));
    GD_CUDA(b.get(&arch[k].size, 1));
    GD_CUDA(b.get(&arch[k].csr_cols, (size_t)K * kMaxLen));
    GD_CUDA(b.get(&arch[k].csr_offs, (size_t)K + 1));
    GD_CUDA(b.get(&abm[k], (size_t)(K + 1) * W));  // row K stays zero: the empty members' row
    GD_CUDA(cudaMemsetAsync(abm[k], 0, (size_t)(K + 1) * W * 4, s));
  }
  GD_CUDA(b.get(&gather_src, K));
  GD_CUDA(cudaMemsetAsync(tabu.slots, 0, cap_t * 8, s));
  GD_CUDA(cudaMemsetAsync(tabu.n_ent, 0, 4, s));
  // the initial population and the empty archive (K members of one column, no rows)
  GD_CUDA(cudaMemcpyAsync(pop.c, init_cols, (size_t)P * kMaxLen * 2, cudaMemcpyHostToDevice, s));
  GD_CUDA(cudaMemcpyAsync(pop.n, init_n, (size_t)P * 4, cudaMemcpyHostToDevice, s));
  GD_CUDA(cudaMemcpyAsync(pop.h, init_h, (size_t)P * 8, cudaMemcpyHostToDevice, s));
  {
    std::vector<uint16_t> c((size_t)K * kMaxLen, 0);
    std::vector<uint32_t> n(K, 1u), zeros(K, 0u), offs(K + 1);
    std::vector<uint64_t> q(K, 0ull);
    for (uint32_t r = 0; r <= K; ++r) offs[r] = r;
    const uint32_t size0 = 0;
    for (int k = 0; k < 2; ++k) {
      // synchronous copies: the host vectors go out of scope
      GD_CUDA(cudaMemcpy(arch[k].c, c.data(), c.size() * 2, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].n, n.data(), K * 4, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].count, zeros.data(), K * 4, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].q, q.data(), K * 8, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].size, &size0, 4, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].csr_cols, c.data(), (size_t)K * 2, cudaMemcpyHostToDevice));
      GD_CUDA(cudaMemcpy(arch[k].csr_offs, offs.data(), (K + 1) * 4, cudaMemcpyHostToDevice));
    }
  }
  Ops o;
  o.P = P;
  o.min_len = p.min_len;
  o.max_init_len = p.max_init_len;
  o.max_len = p.max_len;
  o.tournament = p.tournament;
  o.tabu_retries = p.tabu_retries;
  o.elite = p.elite;
  o.ncols = ncols;
  o.p_crossover = p.p_crossover;
  o.p_mutation = p.p_mutation;
  o.seed = p.seed;
  uint32_t* dgen;
  GD_CUDA(b.get(&dgen, 1));
  GD_CUDA(cudaMemsetAsync(dgen, 0, 4, s));
  Pop pops[2] = {pop, nxt};
  // One generation's work on the stream; the buffers alternate with the generation's parity, so
  // two generations return to the same buffers (a graph of two replays unchanged).
  // Within a generation two branches run side by side: on s2 the tabu insert (beside the
  // scoring), then, after the ranks, the archive chain (offers, their overlaps, admission, the
  // new archive's rows); on s the scoring, the ranks and the breeding chain. They touch disjoint
  // buffers; s waits for s2 before the generation ends.
  auto issue = [&](int par, bool breed) -> int {
    const Pop& cp = pops[par];
    const Pop& np = pops[1 - par];
    GD_CUDA(cudaEventRecord(rs.fork0, s));
    GD_CUDA(cudaStreamWaitEvent(s2, rs.fork0, 0));
    count_launch();
    tabu_insert_kernel<<<(P + 255) / 256, 256, 0, s2>>>(tabu, cp, P);
    GD_CUDA(cudaEventRecord(rs.tabu_done, s2));
    int rc = ebic_eval_fitness(m, dcols, doffs, P, eflags, arch[par].csr_cols, arch[par].csr_offs,
                               abm[par], K, dcounts, dbm, dfit, dov, s);
    if (rc != EBIC_OK) return rc;
    GD_CUDA(cudaMemsetAsync(n_offerable, 0, 4, s));
    OrderArgs oa{cp, P, p.elite, dfit, dcounts, rank, elites, offer_sorted, n_offerable};
    count_launch();
    order_kernel<<<(unsigned)(((uint64_t)P * 32 + 255) / 256), 256, 0, s>>>(oa);
    GD_CUDA(cudaEventRecord(rs.fork1, s));
    // the archive chain, on s2
    GD_CUDA(cudaStreamWaitEvent(s2, rs.fork1, 0));
    count_launch();
    offers_kernel<<<1, 32, 0, s2>>>(cp, offer_sorted, n_offerable, arch[par], T, offers, n_offers);
    GD_CUDA(cudaMemsetAsync(pov, 0, (size_t)T * T * 4, s2));
    count_launch();
    offer_overlap_kernel<<<(unsigned)num_sms, 256, 0, s2>>>(dbm, W, offers, n_offers, T, pov);
    AdmitArgs aa{cp, P, K, T, (uint32_t)(ncols + 31) / 32, p.overlap_threshold, dcounts, dov,
                 pov, offers, n_offers, arch[par], arch[1 - par], gather_src};
    count_launch();
    admit_kernel<<<1, 32, 0, s2>>>(aa);
    GD_CUDA(launch_gather_rows(dbm, abm[par], gather_src, K, W, abm[1 - par], s2));
    GD_CUDA(cudaEventRecord(rs.archive_done, s2));
    // the breeding chain, on s (after the tabu insert)
    if (breed) {
      GD_CUDA(cudaStreamWaitEvent(s, rs.tabu_done, 0));
      BreedArgs ba{o, dgen, cp, np, rank, elites, tabu, kid_rng};
      count_launch();
      breed_kernel<<<(P + 127) / 128, 128, 0, s>>>(ba);
      GD_CUDA(cudaMemsetAsync(table.v, 0, cap_n * 4, s));
      count_launch();
      first_slot_kernel<<<(P + 255) / 256, 256, 0, s>>>(table, np, P);
      count_launch();
      dup_flag_kernel<<<(P + 255) / 256, 256, 0, s>>>(table, np, P, p.elite, dup);
      count_launch();
      spec_kernel<<<(P + 63) / 64, 64, 0, s>>>(o, table, np, tabu, kid_rng, dup, spec);
      count_launch();
      settle_kernel<<<1, 32, 0, s>>>(o, table, np, tabu, kid_rng, dup, spec, acc_slot, acc_h);
      count_launch();
      commit_spec_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, p.elite, dup, spec, np);
      count_launch();
      pack_kernel<<<1, 1024, 0, s>>>(np, P, dcols, doffs);
      count_launch();
      next_generation_kernel<<<1, 1, 0, s>>>(dgen);
    } else {
      GD_CUDA(cudaStreamWaitEvent(s, rs.tabu_done, 0));
    }
    GD_CUDA(cudaStreamWaitEvent(s, rs.archive_done, 0));  // the generation ends on s
    GD_CUDA(cudaGetLastError());
    return EBIC_OK;
  };
  pack_kernel<<<1, 1024, 0, s>>>(pops[0], P, dcols, doffs);
  GD_CUDA(cudaGetLastError());
  // the breeding generations 0 .. G-2 (two at a time from a captured graph when the stream can be
  // captured), then the last one without breeding
  uint32_t gen = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_launches = 0;  // kernels in the two-generation graph
  if (G >= 5) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const int64_t c0 = ebic_launch_count();
      const int rc0 = issue(0, true);
      const int rc1 = rc0 == EBIC_OK ? issue(1, true) : rc0;
      graph_launches = ebic_launch_count() - c0;
      count_launches(-graph_launches);  // nothing ran while capturing
      const cudaError_t ec = cudaStreamEndCapture(s, &graph);
      if (rc1 == EBIC_OK && ec == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    (void)cudaGetLastError();  // a failed capture leaves the direct launches below
  }
  if (exec) {
    for (; gen + 2 <= G - 1; gen += 2) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        GD_CUDA(e);
      }
      count_launches(graph_launches);
    }
    cudaGraphExecDestroy(exec);
  }
  for (; gen + 1 < G; ++gen) {
    const int rc = issue((int)(gen & 1u), true);
    if (rc != EBIC_OK) return rc;
  }
  {
    const int rc = issue((int)(gen & 1u), false);  // the last generation
    if (rc != EBIC_OK) return rc;
    ++gen;
  }
  const int cur = (int)(gen & 1u);  // the archive the last generation wrote
  const uint64_t evaluated = (uint64_t)P * gen;
  GD_CUDA(cudaStreamSynchronize(s));
  int st = ebic_matrix_status(const_cast<ebic_matrix*>(m), s);
  if (st != EBIC_OK) return st;
  // the archive, best first
  uint32_t n = 0;
  GD_CUDA(cudaMemcpy(&n, arch[cur].size, 4, cudaMemcpyDeviceToHost));
  std::vector<uint16_t> c((size_t)K * kMaxLen);
  std::vector<uint32_t> len(K), cnt(K);
  std::vector<uint64_t> q(K);
  GD_CUDA(cudaMemcpy(c.data(), arch[cur].c, c.size() * 2, cudaMemcpyDeviceToHost));
  GD_CUDA(cudaMemcpy(len.data(), arch[cur].n, K * 4, cudaMemcpyDeviceToHost));
  GD_CUDA(cudaMemcpy(cnt.data(), arch[cur].count, K * 4, cudaMemcpyDeviceToHost));
  GD_CUDA(cudaMemcpy(q.data(), arch[cur].q, K * 8, cudaMemcpyDeviceToHost));
  ebic_result* r = new ebic_result();
  std::memset(r, 0, sizeof(*r));
  r->n = n;
  r->words = (rows + 31) / 32;
  r->generations_run = gen;
  r->candidates_evaluated = evaluated;
  size_t tot = 0;
  for (uint32_t i = 0; i < n; ++i) tot += len[i];
  r->cols = new uint16_t[tot > 0 ? tot : 1];
  r->offsets = new uint32_t[n + 1];
  r->counts = new uint32_t[n > 0 ? n : 1];
  r->quality = new uint64_t[n > 0 ? n : 1];
  r->bitmaps = new uint32_t[(size_t)n * (size_t)W + 1];
  r->offsets[0] = 0;
  size_t pos = 0;
  for (uint32_t i = 0; i < n; ++i) {
    std::copy(c.begin() + (size_t)i * kMaxLen, c.begin() + (size_t)i * kMaxLen + len[i],
              r->cols + pos);
    pos += len[i];
    r->offsets[i + 1] = (uint32_t)pos;
    r->counts[i] = cnt[i];
    r->quality[i] = q[i];
  }
  cudaError_t e = n ? cudaMemcpy(r->bitmaps, abm[cur], (size_t)n * W * 4, cudaMemcpyDeviceToHost)
                    : cudaSuccess;
  if (e != cudaSuccess) {
    ebic_free_result(r);
    GD_CUDA(e);
  }
  *out = r;
  return EBIC_OK;
}

}  // namespace ebic
