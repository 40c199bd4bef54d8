// Device code of the pair-table pass shared by the single-population pass (pairs.cu) and the
// batched pass (batch.cu): item shape, a candidate's term list, the chain walk over the table
// rows, and the per-item epilogue (counts, bitmap words, archive overlaps). The file comment of
// pairs.cu describes the encoding and the work order.
#pragma once

#include "device_common.cuh"
#include "ebic_internal.h"

namespace ebic {
namespace pairdev {

constexpr int kPairThreads = 768;
constexpr int kPairWarps = kPairThreads / 32;
constexpr int kParts = 4;        // 128-word parts per item (four words per lane each)
constexpr int kStepTerms = 2;    // terms per chain step (one with negative trends)
constexpr int kRangeWords = 128;             // words per part (4,096 rows)
constexpr int kItemWords = kParts * kRangeWords;
static_assert(kPairRangeWords % kItemWords == 0, "table stride must hold whole items");
constexpr int kFewWords = 12;  // at most this many non-zero words: a lane per archive member

__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ uint32_t popc4(uint4 v) {
  // carry-save: popc(a) + popc(b) + popc(c) = popc(a ^ b ^ c) + 2 popc(maj(a, b, c))
  const uint32_t s = v.x ^ v.y ^ v.z;
  const uint32_t c = (v.x & v.y) | (v.z & (v.x ^ v.y));
  return __popc(s) + 2u * __popc(c) + __popc(v.w);
}

// One candidate's term list as the warp holds it: lane i has the row offsets of terms i and
// 32 + i (forward; reversed in blo/bhi), lane 31's hi word is the length L.
struct Terms {
  uint32_t lo = 0, hi = 0, blo = 0, bhi = 0;
};

template <bool NEG>
__device__ __forceinline__ void load_terms(const PairArgs& p, uint32_t cand, int lane,
                                           Terms& t) {
  const uint32_t* tp = p.terms + (uint64_t)cand * (NEG ? 2 * kTermSlots : kTermSlots);
  t.lo = __ldg(tp + lane);
  t.hi = __ldg(tp + 32 + lane);
  if (NEG) {
    t.blo = __ldg(tp + 64 + lane);
    t.bhi = __ldg(tp + 96 + lane);
  }
}

// The term list of candidate `cand` of a checked CSR list, computed in registers (the batched
// pass has no preparation kernel to build it): the same words the preparation writes, lane i
// holding terms i and 32 + i, lane 31's hi word the length L.
// From the candidate's L columns in registers (lane i: columns i and 32 + i).
template <bool NEG>
__device__ __forceinline__ void terms_from_cols(uint32_t c_lo, uint32_t c_hi, int L, uint32_t C,
                                                uint32_t S, int lane, Terms& t) {
  const uint32_t n_lo = __shfl_down_sync(0xFFFFFFFFu, c_lo, 1);
  const uint32_t n_hi = __shfl_down_sync(0xFFFFFFFFu, c_hi, 1);
  const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, c_hi, 0);
  const uint32_t next_lo = lane == 31 ? h0 : n_lo;  // c_{i+1} for i = lane
  const int n_terms = L == 1 ? 1 : L - 1;
  const bool t_lo = lane < n_terms, t_hi = lane + 32 < n_terms;
  t.lo = t_lo ? (L == 1 ? c_lo * C + c_lo : c_lo * C + next_lo) * S : 0u;
  t.hi = lane == 31 ? (uint32_t)L : (t_hi ? (c_hi * C + n_hi) * S : 0u);
  if (NEG) {
    t.blo = t_lo && L > 1 ? (next_lo * C + c_lo) * S : 0u;
    t.bhi = t_hi ? (n_hi * C + c_hi) * S : 0u;
  }
}

template <bool NEG>
__device__ __forceinline__ void terms_from_list(const uint16_t* __restrict__ cols,
                                                const uint32_t* __restrict__ offs, uint32_t cand,
                                                uint32_t C, uint32_t S, int lane, Terms& t) {
  const uint32_t o = offs[cand];
  const int L = (int)(offs[cand + 1] - o);
  const uint32_t c_lo = lane < L ? cols[o + lane] : 0u;
  const uint32_t c_hi = lane + 32 < L ? cols[o + 32 + lane] : 0u;
  terms_from_cols<NEG>(c_lo, c_hi, L, C, S, lane, t);
}

// L2 prefetch of the item segments (kParts parts of kRangeWords words: 2 KB, sixteen 128-byte
// lines) of two table rows, at word offsets off_a and off_b from `item` (the item's first table
// word): lanes 0-15 take row a's lines, lanes 16-31 row b's, one line per lane, only in the parts
// whose bit is set in part_mask. A prefetch holds no register: the pass issues one for the next
// candidate's first step before the current candidate's epilogue. (Prefetching each chain
// step's next rows as well measured slower, most for long candidates.)
__device__ __forceinline__ void prefetch_rows2(const uint32_t* item, uint32_t off_a, bool has_a,
                                               uint32_t off_b, bool has_b, uint32_t part_mask,
                                               int lane) {
  const int line = lane & 15;
  const bool b = lane >= 16;
  if ((b ? has_b : has_a) && ((part_mask >> (line >> 2)) & 1u)) {
    const uint32_t* ptr = item + (b ? off_b : off_a) + line * 32;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
  }
}

// The candidate's bitmap words 4*lane .. 4*lane+3 of each 128-word part of the item whose first
// table word is `base` (table + item*kItemWords): AND of its consecutive pairs' table rows, OR
// the reversed pairs' AND with negative trends. Each step keeps the rows of several terms of
// every part in flight. A lane whose own words of a part are all zero (they stay zero) reads the
// table's all-ones chunk `ones` instead of its segment: every lane doing so reads the same 16
// bytes, so the step's requests shrink to the lanes that still match rows, with no branch. The
// walk stops when no lane has a non-zero word left (long chains match no row of most ranges).
template <bool NEG>
__device__ __forceinline__ void pair_chain(const Terms& t, const uint32_t* base,
                                           const uint32_t* ones, int lane,
                                           uint4 (&out)[kParts]) {
  constexpr int kStep = NEG ? kStepTerms / 2 : kStepTerms;
  const int L = (int)__shfl_sync(0xFFFFFFFFu, t.hi, 31);
  const int n_terms = L == 1 ? 1 : L - 1;
  const bool two = NEG && L > 1;  // warp-uniform
  const uint4 all = make_uint4(~0u, ~0u, ~0u, ~0u);
  uint4 x[kParts], y[kParts];
  bool nzx[kParts], nzy[kParts];  // this lane's words of the part are not all zero
#pragma unroll
  for (int q = 0; q < kParts; ++q) {
    x[q] = y[q] = all;
    nzx[q] = nzy[q] = true;
  }
  // terms [t0, t1) with t0 in {0, 32}: lane (i - t0) holds term i's offsets
  auto walk = [&](uint32_t offf, uint32_t offb, int t0, int t1) -> bool {
    for (int i0 = t0; i0 < t1; i0 += kStep) {
      // the next step's rows, prefetched while this step's are loaded (the parts still alive
      // after the previous step: at most one step's rows are fetched in vain)
      uint4 v[kStep][kParts], u[kStep][kParts];
#pragma unroll
      for (int k = 0; k < kStep; ++k) {
        const int i = i0 + k;
        const bool has = i < t1;  // warp-uniform
        const uint32_t* rf = base + __shfl_sync(0xFFFFFFFFu, offf, i & 31);
#pragma unroll
        for (int q = 0; q < kParts; ++q)
          v[k][q] = __ldg(reinterpret_cast<const uint4*>(has && nzx[q] ? rf + q * kRangeWords
                                                                       : ones));
        if (NEG) {
          const uint32_t* rb = base + __shfl_sync(0xFFFFFFFFu, offb, i & 31);
#pragma unroll
          for (int q = 0; q < kParts; ++q)
            u[k][q] = __ldg(reinterpret_cast<const uint4*>(two && has && nzy[q]
                                                               ? rb + q * kRangeWords
                                                               : ones));
        }
      }
      bool lane_any = false;
#pragma unroll
      for (int q = 0; q < kParts; ++q) {
#pragma unroll
        for (int k = 0; k < kStep; ++k) x[q] = and4(x[q], v[k][q]);
        nzx[q] = (x[q].x | x[q].y | x[q].z | x[q].w) != 0u;
        lane_any |= nzx[q];
        if (NEG && two) {
#pragma unroll
          for (int k = 0; k < kStep; ++k) y[q] = and4(y[q], u[k][q]);
          nzy[q] = (y[q].x | y[q].y | y[q].z | y[q].w) != 0u;
          lane_any |= nzy[q];
        }
      }
      if (!__any_sync(0xFFFFFFFFu, lane_any)) return false;  // all zero from here on
    }
    return true;
  };
  if (walk(t.lo, t.blo, 0, n_terms < 32 ? n_terms : 32) && n_terms > 32)
    walk(t.hi, t.bhi, 32, n_terms);
#pragma unroll
  for (int q = 0; q < kParts; ++q)
    out[q] = two ? make_uint4(x[q].x | y[q].x, x[q].y | y[q].y, x[q].z | y[q].z, x[q].w | y[q].w)
                 : x[q];
}

// An archive row segment: re-read by every warp of the CTA that scores a candidate of the same
// range, so it is kept in L1 in preference to the streamed table rows. Archive rows are padded
// with zero words to the table's stride, an even number of rows.
__device__ __forceinline__ uint32_t ld_keep1(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ uint4 ld_arch4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::evict_last.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Adds a packed pair of warp sums (member 2k in the low 16 bits, 2k+1 in the high 16 bits) to
// the two adjacent 32-bit overlap counters of the pair with one 64-bit atomic (no carry crosses
// from the low counter: each total is at most the row count, below 2^32).
__device__ __forceinline__ void add_pair(unsigned long long* ov2, int k, uint32_t r, int lane) {
  if (lane == 0 && r)
    atomicAdd(&ov2[k], (unsigned long long)(r & 0xFFFFu) | ((unsigned long long)(r >> 16) << 32));
}

// Bitmap words and archive overlaps of candidate `cand` for the item at `rword`, from its words
// x (lane holds words 4*lane .. 4*lane+3 of part q, i.e. item words 128q + 4*lane + j, in x[q])
// and their warp total cnt.
// `members`: the archive members whose overlaps are wanted (a bit per member below n_arch).
template <bool BITMAPS, bool OVERLAP>
__device__ __forceinline__ void item_epilogue(const PairArgs& p, uint32_t cand, uint64_t rword,
                                              const uint4 (&x)[kParts], uint32_t cnt, uint32_t* st,
                                              int lane, uint32_t n_arch, int n_pairs,
                                              uint64_t members) {
  if constexpr (BITMAPS) {  // through shared memory, so each store instruction is coalesced
    uint32_t* out = p.bitmaps + (uint64_t)cand * (uint64_t)p.W;
#pragma unroll
    for (int h = 0; h < kParts; ++h) {
      *reinterpret_cast<uint4*>(st + 4 * lane) = x[h];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t w = rword + kRangeWords * h + 32 * j + lane;
        if (w < (uint64_t)p.W) out[w] = st[32 * j + lane];
      }
      __syncwarp();
    }
  }
  if constexpr (OVERLAP) {
    if (cnt == 0 || members == 0) return;  // warp-uniform: nothing to add
    const uint64_t astride = p.stride;
    const uint32_t* abase = p.arch + rword;
    uint32_t* ov = p.overlaps + (uint64_t)cand * p.ov_stride;
    // the lane's eight words and where they sit in the item
    uint32_t xw[4 * kParts];
#pragma unroll
    for (int q = 0; q < kParts; ++q) {
      xw[4 * q] = x[q].x;
      xw[4 * q + 1] = x[q].y;
      xw[4 * q + 2] = x[q].z;
      xw[4 * q + 3] = x[q].w;
    }
    uint32_t bal[4 * kParts];
    int nz = 0;
#pragma unroll
    for (int j = 0; j < 4 * kParts; ++j) {
      bal[j] = __ballot_sync(0xFFFFFFFFu, xw[j] != 0u);
      nz += __popc(bal[j]);
    }
    if (nz <= 32) {
      // compact the non-zero words: lane i takes the i-th one (value and word offset)
      uint32_t* sv = st;
      uint32_t* si = st + 32;
      const uint32_t lt = (1u << lane) - 1u;
      int base = 0;
#pragma unroll
      for (int j = 0; j < 4 * kParts; ++j) {
        if (xw[j]) {
          const int q = base + __popc(bal[j] & lt);
          sv[q] = xw[j];
          si[q] = (uint32_t)(kRangeWords * (j / 4)) + 4u * lane + (j & 3);
        }
        base += __popc(bal[j]);
      }
      __syncwarp();
      if (nz <= kFewWords) {
        // few non-zero words: a lane per archive member (two for members 32..63) walks them
        // all, gathering its member's word at each; no warp reduction, one atomic per member
        const bool a0 = (members >> lane) & 1ull;
        const bool a1 = (members >> (lane + 32)) & 1ull;
        const uint32_t* ar0 = abase + (uint64_t)lane * astride;
        const uint32_t* ar1 = abase + (uint64_t)(lane + 32) * astride;
        uint32_t o0 = 0, o1 = 0;
#pragma unroll 4
        for (int i = 0; i < nz; ++i) {
          const uint32_t v = sv[i], w = si[i];
          if (a0) o0 += __popc(v & ld_keep1(ar0 + w));
          if (a1) o1 += __popc(v & ld_keep1(ar1 + w));
        }
        __syncwarp();
        if (o0) atomicAdd(&ov[lane], o0);
        if (o1) atomicAdd(&ov[lane + 32], o1);
      } else {
        // a word per lane, two members per warp reduction (sums <= 1,024), one 64-bit atomic
        // per member pair
        unsigned long long* ov2 = reinterpret_cast<unsigned long long*>(ov);
        const uint64_t S2 = 2ull * astride;  // from member 2k to 2k+2
        const uint32_t mv = lane < nz ? sv[lane] : 0u;
        const uint32_t* ab = abase + (lane < nz ? si[lane] : 0u);
        __syncwarp();
        for (int k = 0; k < n_pairs; ++k, ab += S2) {
          if (((members >> (2 * k)) & 3ull) == 0) continue;  // warp-uniform
          // (an odd archive's last pair reads the zero padding row)
          const uint32_t w0 = ld_keep1(ab), w1 = ld_keep1(ab + astride);
          const uint32_t r =
              __reduce_add_sync(0xFFFFFFFFu, __popc(mv & w0) + (__popc(mv & w1) << 16));
          add_pair(ov2, k, r, lane);
        }
      }
    } else {
      // dense: the wanted members two at a time (no unwanted partner), one packed reduction
      // (each sum <= 128 * 4 * kParts * 32 / 4 < 2^16), lanes 0 and 1 add the two totals
      const uint32_t* ab = abase + 4 * lane;
      uint64_t mm = members;
      while (mm) {  // warp-uniform
        const int ma = __ffsll((long long)mm) - 1;
        mm &= mm - 1ull;
        const int mb = mm ? __ffsll((long long)mm) - 1 : ma;
        const bool has_b = mm != 0ull;
        mm &= mm - 1ull;
        const uint32_t* pa = ab + (uint64_t)ma * astride;
        const uint32_t* pb = ab + (uint64_t)mb * astride;
        uint32_t sa = 0, sb = 0;
#pragma unroll
        for (int q = 0; q < kParts; ++q) {
          sa += popc4(and4(x[q], ld_arch4(pa + q * kRangeWords)));
          sb += popc4(and4(x[q], ld_arch4(pb + q * kRangeWords)));
        }
        if (!has_b) sb = 0u;
        const uint32_t r = __reduce_add_sync(0xFFFFFFFFu, sa + (sb << 16));
        const uint32_t v = lane == 0 ? (r & 0xFFFFu) : (r >> 16);
        if (lane < 2 && v) atomicAdd(&ov[lane == 0 ? ma : mb], v);
      }
    }
  }
}

// The pass over all (range, candidate group) items of one population, by a persistent grid of
// kPairThreads-thread CTAs (see pairs.cu for the work order); `st` is the warp's kRangeWords-word
// shared staging buffer. CTA b owns items b, b + G, b + 2G, ... (G = gridDim.x); an item's
// kPairWarps candidates are its units, and the CTA's warps take units in that order from the
// CTA's shared counter `next_unit` (zero at entry) as each becomes free, so a warp that drew
// short candidates takes more of them and the CTA ends when its work ends, not when its unluckiest
// warp does. The units of one item still run side by side on one SM, so the table rows they
// share meet in its L1.
// `valid()` (warp-uniform) is asked after the warp's first term list is requested and before any
// table row is read; false ends the pass.
template <bool NEG, bool BITMAPS, bool OVERLAP, class Valid>
__device__ __forceinline__ void pair_items(const PairArgs& p, uint32_t* st, uint32_t* next_unit,
                                           Valid valid) {
  const int lane = threadIdx.x & 31;
  const uint32_t n_ranges = (uint32_t)((p.W + kItemWords - 1) / kItemWords);
  const uint32_t n_groups = (p.n_cand + kPairWarps - 1) / kPairWarps;
  const uint64_t n_items = (uint64_t)n_ranges * n_groups;
  const bool narrow = n_items <= 0xFFFFFFFFull;  // 32-bit item arithmetic suffices
  const uint32_t n_arch = OVERLAP ? p.n_arch : 0u;
  const int n_pairs = (int)(n_arch + 1) >> 1;
  const uint64_t all_members = n_arch >= 64 ? ~0ull : ((1ull << n_arch) - 1ull);
  const uint32_t* ones = pair_ones(p.table, (uint64_t)p.C, p.stride);
  struct Unit {
    uint64_t it;
    uint32_t range, grp, slot, cand;
  };
  // the CTA's next unit: its item, range, group, slot and candidate
  auto take = [&]() {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(next_unit, 1u);
    u = __shfl_sync(0xFFFFFFFFu, u, 0);
    Unit x;
    x.slot = u % kPairWarps;
    x.it = blockIdx.x + (uint64_t)(u / kPairWarps) * gridDim.x;
    x.range = x.grp = x.cand = 0;
    if (x.it < n_items) {
      if (narrow) {
        x.range = (uint32_t)x.it / n_groups;
        x.grp = (uint32_t)x.it - x.range * n_groups;
      } else {
        x.range = (uint32_t)(x.it / n_groups);
        x.grp = (uint32_t)(x.it - (uint64_t)x.range * n_groups);
      }
      x.cand = x.grp * kPairWarps + x.slot;
    }
    return x;
  };
  Unit cur = take();
  Terms next;
  if (cur.it < n_items && cur.cand < p.n_cand) load_terms<NEG>(p, cur.cand, lane, next);
  if (!valid()) return;
  while (cur.it < n_items) {
    const uint64_t rword = (uint64_t)cur.range * kItemWords;  // first word of the item
    const uint32_t cand = cur.cand;
    const Terms t = next;
    const bool arch_share = OVERLAP && cur.grp == 0;  // this range's archive counts, slot's share
    const uint32_t slot = cur.slot;
    // the next unit, and its term list, requested before this one is walked
    cur = take();
    if (cur.it < n_items && cur.cand < p.n_cand) load_terms<NEG>(p, cur.cand, lane, next);
    if (arch_share) {  // the archive members' own row counts, once per range
      for (uint32_t a = slot; a < n_arch; a += kPairWarps) {
        const uint32_t* ar = p.arch + (uint64_t)a * p.stride + rword + 4 * lane;
        uint32_t pa = 0;
#pragma unroll
        for (int q = 0; q < kParts; ++q) pa += popc4(ld_arch4(ar + q * kRangeWords));
        const uint32_t n = __reduce_add_sync(0xFFFFFFFFu, pa);
        if (lane == 0 && n) atomicAdd(&p.arch_counts[a], n);
      }
    }
    if (cand >= p.n_cand) continue;  // warp-uniform
    uint4 x[kParts];
    pair_chain<NEG>(t, p.table + rword + 4 * lane, ones, lane, x);
    // the next unit's first step, prefetched while this unit's epilogue runs (its term list has
    // arrived during the walk)
    if (!NEG && cur.it < n_items && cur.cand < p.n_cand) {
      const int Ln = (int)__shfl_sync(0xFFFFFFFFu, next.hi, 31);
      const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, next.lo, 0);
      const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, next.lo, 1);
      prefetch_rows2(p.table + (uint64_t)cur.range * kItemWords, a0, true, a1, Ln > 2,
                     (1u << kParts) - 1u, lane);
    }
    uint32_t pc = 0;
#pragma unroll
    for (int q = 0; q < kParts; ++q) pc += popc4(x[q]);
    const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, pc);
    if (lane == 0 && c) atomicAdd(&p.counts[cand], c);
    const uint64_t members = OVERLAP && p.score ? p.score[cand] & all_members : all_members;
    item_epilogue<BITMAPS, OVERLAP>(p, cand, rword, x, c, st, lane, n_arch, n_pairs, members);
  }
}

}  // namespace pairdev
}  // namespace ebic
