// Device code of the population preparation and of the fused pass's fitness: candidate checks,
// term lists, share masks, the padded archive copy, the fused preparation's work for one block,
// and F_c of one candidate.
#pragma once

#include "device_common.cuh"
#include "ebic_internal.h"

namespace ebic {
namespace prepdev {

constexpr int kSetWords = (kMaxCols + 31) / 32;  // a column set as a bitset

// Warp-cooperative check of candidate i of a CSR list of n: offsets[0] == 0, 1 <= L <= 64, the
// candidate ends at or before offsets[n] (so its columns lie inside cols[0 .. offsets[n]), the
// caller's buffer), its columns are < ncols and distinct. Columns are read only when the offsets
// pass, so reads stay in bounds whatever the other candidates' offsets are. Leaves the
// candidate's column set in `set` (the warp's own shared-memory bitset; empty when the offsets
// fail). Returns true on every lane when the candidate is invalid.
__device__ inline bool check_candidate_span(const uint16_t* __restrict__ cols, uint32_t lo, uint32_t hi,
                                     uint32_t total, bool first, int32_t ncols, uint32_t* set,
                                     int lane) {
  const bool bad = (first && lo != 0u) || hi <= lo || hi - lo > (uint32_t)kMaxLen || hi > total;
  const int nw = (ncols + 31) / 32;
  for (int w = lane; w < nw; w += 32) set[w] = 0u;
  __syncwarp();
  bool b = false;
  if (!bad) {
    for (uint32_t j = lo + lane; j < hi; j += 32) {
      const uint32_t c = cols[j];
      if (c >= (uint32_t)ncols) {
        b = true;
        continue;
      }
      const uint32_t bit = 1u << (c & 31u);
      b |= (atomicOr(&set[c >> 5], bit) & bit) != 0u;  // seen before: a repeated column
    }
  }
  __syncwarp();
  return __any_sync(0xFFFFFFFFu, bad || b);
}

__device__ inline bool check_candidate_warp(const uint16_t* __restrict__ cols,
                                     const uint32_t* __restrict__ offs, uint32_t n, uint32_t i,
                                     int32_t ncols, uint32_t* set, int lane) {
  return check_candidate_span(cols, offs[i], offs[i + 1], offs[n], i == 0, ncols, set, lane);
}

// The term list of one candidate (see kTermSlots), a warp per candidate. Its offsets must have
// passed the check (lo < hi <= lo + 64, inside the caller's columns); a column >= C makes a
// garbage offset, but the call is then rejected and no later kernel reads the list.
__device__ inline void build_terms_warp(const uint16_t* __restrict__ cols, uint32_t lo, uint32_t hi,
                                 uint32_t C, uint32_t S, bool negative, uint32_t* out,
                                 int lane) {
  const int L = (int)(hi - lo);
  const uint32_t c_lo = lane < L ? cols[lo + lane] : 0u;
  const uint32_t c_hi = lane + 32 < L ? cols[lo + 32 + lane] : 0u;
  const uint32_t n_lo = __shfl_down_sync(0xFFFFFFFFu, c_lo, 1);
  const uint32_t n_hi = __shfl_down_sync(0xFFFFFFFFu, c_hi, 1);
  const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, c_hi, 0);
  const uint32_t next_lo = lane == 31 ? h0 : n_lo;  // c_{i+1} for i = lane
  const int n_terms = L == 1 ? 1 : L - 1;
  const bool t_lo = lane < n_terms, t_hi = lane + 32 < n_terms;
  out[lane] = t_lo ? (L == 1 ? c_lo * C + c_lo : c_lo * C + next_lo) * S : 0u;
  out[32 + lane] = lane == 31 ? (uint32_t)L : (t_hi ? (c_hi * C + n_hi) * S : 0u);
  if (negative) {
    out[64 + lane] = t_lo && L > 1 ? (next_lo * C + c_lo) * S : 0u;
    out[96 + lane] = t_hi ? (n_hi * C + c_hi) * S : 0u;
  }
}

__device__ __forceinline__ bool offsets_sane(uint32_t lo, uint32_t hi, uint32_t total,
                                             bool first) {
  return !(first && lo != 0u) && hi > lo && hi - lo <= (uint32_t)kMaxLen && hi <= total;
}

__device__ __forceinline__ void report_invalid(bool bad, uint32_t* err, uint32_t* status) {
  if (bad) {
    atomicOr(err, kErrInvalid);
    if (status) atomicOr(status, kErrInvalid);
  }
}


// Shared memory of the fused preparation in a block of WARPS warps.
template <int WARPS>
struct PrepShared {
  uint32_t msets[kPairMaxArch][kSetWords];  // archive members' column sets
  uint32_t sets[WARPS][kSetWords];          // a warp's candidate column set
  uint32_t aoff[kPairMaxArch + 1];          // archive offsets
};

// The columns of a candidate whose offsets passed offsets_sane, lane i holding columns i and
// 32 + i (0 past the end).
__device__ __forceinline__ void load_cols_regs(const uint16_t* __restrict__ cols, uint32_t lo,
                                               uint32_t hi, int lane, uint32_t& c_lo,
                                               uint32_t& c_hi) {
  const uint32_t L = hi - lo;
  c_lo = (uint32_t)lane < L ? cols[lo + lane] : 0u;
  c_hi = (uint32_t)lane + 32u < L ? cols[lo + 32 + lane] : 0u;
}

// True on every lane unless the L columns held as load_cols_regs leaves them are all < ncols and
// distinct; `set` (the warp's bitset, zero on entry) is left holding the column set.
__device__ __forceinline__ bool cols_bad_regs(uint32_t c_lo, uint32_t c_hi, uint32_t L,
                                              int32_t ncols, uint32_t* set, int lane) {
  bool b = false;
  auto add = [&](uint32_t c) {
    if (c >= (uint32_t)ncols) {
      b = true;
      return;
    }
    const uint32_t bit = 1u << (c & 31u);
    b |= (atomicOr(&set[c >> 5], bit) & bit) != 0u;  // seen before: a repeated column
  };
  if ((uint32_t)lane < L) add(c_lo);
  if ((uint32_t)lane + 32u < L) add(c_hi);
  __syncwarp();
  return __any_sync(0xFFFFFFFFu, b);
}

// The term list of a checked candidate from its columns in registers (see build_terms_warp).
__device__ __forceinline__ void build_terms_regs(uint32_t c_lo, uint32_t c_hi, int L, uint32_t C,
                                                 uint32_t S, bool negative, uint32_t* out,
                                                 int lane) {
  const uint32_t n_lo = __shfl_down_sync(0xFFFFFFFFu, c_lo, 1);
  const uint32_t n_hi = __shfl_down_sync(0xFFFFFFFFu, c_hi, 1);
  const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, c_hi, 0);
  const uint32_t next_lo = lane == 31 ? h0 : n_lo;  // c_{i+1} for i = lane
  const int n_terms = L == 1 ? 1 : L - 1;
  const bool t_lo = lane < n_terms, t_hi = lane + 32 < n_terms;
  out[lane] = t_lo ? (L == 1 ? c_lo * C + c_lo : c_lo * C + next_lo) * S : 0u;
  out[32 + lane] = lane == 31 ? (uint32_t)L : (t_hi ? (c_hi * C + n_hi) * S : 0u);
  if (negative) {
    out[64 + lane] = t_lo && L > 1 ? (next_lo * C + c_lo) * S : 0u;
    out[96 + lane] = t_hi ? (n_hi * C + c_hi) * S : 0u;
  }
}

// The mask of archive members (column sets in msets) sharing a column with the warp's set.
__device__ __forceinline__ uint64_t share_mask(const uint32_t* set,
                                               const uint32_t (*msets)[kSetWords], uint32_t na,
                                               int nw, int lane) {
  uint32_t s0 = 0u, s1 = 0u;
  for (int w = 0; w < nw; ++w) {
    const uint32_t cw = set[w];
    if ((uint32_t)lane < na) s0 |= cw & msets[lane][w];
    if ((uint32_t)lane + 32u < na) s1 |= cw & msets[lane + 32][w];
  }
  const uint32_t lo_mask = __ballot_sync(0xFFFFFFFFu, s0 != 0u);
  const uint32_t hi_mask = __ballot_sync(0xFFFFFFFFu, s1 != 0u);
  return ((uint64_t)hi_mask << 32) | lo_mask;
}

// The archive's rows (src, [na][W]) copied into rows of `stride` words with zero padding, an
// even number of rows (dst), by threads tid of nthreads, eight loads in flight each (so a
// preparation grid copies a 20-member archive of 436,444 rows in one round of loads).
__device__ __forceinline__ void copy_archive_padded(const uint32_t* __restrict__ src,
                                                    uint32_t* __restrict__ dst, uint32_t na,
                                                    int64_t W, uint32_t stride, size_t tid,
                                                    size_t nthreads) {
  constexpr int kInFlight = 8;
  const uint64_t n_pad = (uint64_t)((na + 1u) & ~1u) * stride;
  const bool narrow = n_pad < (1ull << 32);  // 32-bit index arithmetic suffices
  for (uint64_t i0 = tid; i0 < n_pad; i0 += kInFlight * nthreads) {
    uint32_t v[kInFlight];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) {
      const uint64_t i = i0 + k * nthreads;
      uint64_t m, w;
      if (narrow) {
        const uint32_t i32 = (uint32_t)i;
        m = i32 / stride;
        w = i32 - (uint32_t)m * stride;
      } else {
        m = i / stride;
        w = i - m * stride;
      }
      v[k] = i < n_pad && m < na && w < (uint64_t)W ? src[m * (uint64_t)W + w] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) {
      const uint64_t i = i0 + k * nthreads;
      if (i < n_pad) dst[i] = v[k];
    }
  }
}

// The fused preparation's work for block `blk` of `nblk` blocks of WARPS warps (see
// FusedPrepareArgs): checks, term lists, share masks, zeroed outputs and the padded archive copy.
// Two rounds of global loads: (A) archive offsets, the warp's first candidate's offsets and the
// archive copy, with every zeroing store; (B) the archive members' columns (checked there, when
// the caller keeps the archive list on the device) and the first candidate's columns together,
// then its check and term list from registers; (C) share masks
// (shared memory only), then any further candidates of the warp one by one. Every thread of the
// block calls it; returns true on a thread that found an invalid list (the caller reduces the
// verdict over the block).
template <int WARPS>
__device__ bool fused_prepare_body(const FusedPrepareArgs& a, PrepShared<WARPS>& sh,
                                   uint32_t blk, uint32_t nblk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t tid = (size_t)blk * blockDim.x + threadIdx.x;
  const size_t nthreads = (size_t)nblk * blockDim.x;
  const uint32_t gw = blk * WARPS + warp, nwarps = nblk * WARPS;
  const int nw = (a.ncols + 31) / 32;
  const uint32_t na = a.n_arch;
  uint32_t* const set = sh.sets[warp];
  const int slots = term_slots(a.negative);

  // (A)
  if (threadIdx.x <= na && na) sh.aoff[threadIdx.x] = a.aoffsets[threadIdx.x];
  for (int i = threadIdx.x; i < (int)na * kSetWords; i += blockDim.x) (&sh.msets[0][0])[i] = 0u;
  for (int w = lane; w < nw; w += 32) set[w] = 0u;
  uint32_t lo0 = 0, hi0 = 0, tot0 = 0;
  if (gw < a.n_cand) {
    lo0 = a.offsets[gw];
    hi0 = a.offsets[gw + 1];
    tot0 = a.offsets[a.n_cand];
  }
  for (uint32_t i = gw; i < a.n_cand; i += nwarps) {  // the warp's candidates' counters
    if (lane == 0) a.counts[i] = 0u;
    for (uint32_t m = lane; m < a.ov_stride; m += 32) a.overlaps[(size_t)i * a.ov_stride + m] = 0u;
  }
  copy_archive_padded(a.arch_src, a.arch_pad, na, a.W, a.stride, tid, nthreads);
  for (size_t i = tid; i < na; i += nthreads) a.arch_counts[i] = 0u;
  __syncthreads();

  // (B) the first candidate's columns are requested first, then every block builds the
  // members' column sets, one (member, position) per thread; a member whose offsets fail
  // contributes none (the list is rejected below, and the pass that follows does nothing)
  const bool first_sane = gw < a.n_cand && offsets_sane(lo0, hi0, tot0, gw == 0);
  uint32_t c_lo = 0, c_hi = 0;
  if (first_sane) load_cols_regs(a.cols, lo0, hi0, lane, c_lo, c_hi);
  const uint32_t atotal = na ? sh.aoff[na] : 0u;
  // the archive list is checked on the way (when the caller keeps it on the device): offsets, a
  // column out of range, a column repeated within a member (seen by the atomic OR)
  bool abad = false;
  if (a.check_arch)
    for (uint32_t m = threadIdx.x; m < na; m += blockDim.x) {
      const uint32_t lo = sh.aoff[m], hi = sh.aoff[m + 1];
      abad |= !offsets_sane(lo, hi, atotal, m == 0);
    }
  for (uint32_t t0 = threadIdx.x; t0 < na * (uint32_t)kMaxLen; t0 += 4 * blockDim.x) {
    uint32_t c[4], m[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t t = t0 + k * blockDim.x;
      m[k] = t / kMaxLen;
      const uint32_t j = t % kMaxLen;
      ok[k] = false;
      c[k] = 0u;
      if (m[k] < na) {
        const uint32_t lo = sh.aoff[m[k]], hi = sh.aoff[m[k] + 1];
        const bool sane = !(m[k] == 0 && lo != 0u) && hi > lo && hi - lo <= (uint32_t)kMaxLen &&
                          hi <= atotal;
        ok[k] = sane && j < hi - lo;
        if (ok[k]) c[k] = a.acols[lo + j];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (ok[k]) {
        if (c[k] < (uint32_t)a.ncols) {
          const uint32_t bit = 1u << (c[k] & 31u);
          const bool seen = (atomicOr(&sh.msets[m[k]][c[k] >> 5], bit) & bit) != 0u;
          abad |= a.check_arch && seen;
        } else {
          abad |= a.check_arch;
        }
      }
  }
  bool bad = false;
  if (gw < a.n_cand) {
    bad = !first_sane;
    if (first_sane) {
      const uint32_t L = hi0 - lo0;
      bad = cols_bad_regs(c_lo, c_hi, L, a.ncols, set, lane);
      build_terms_regs(c_lo, c_hi, (int)L, (uint32_t)a.ncols, a.stride, a.negative,
                       a.terms + (size_t)gw * slots, lane);
      if (a.table && !bad && !a.negative) {
        // the first chain step (terms 0 and 1) of the candidate's first two 16,384-row ranges:
        // lanes 0-15 the lines of term 0's rows, lanes 16-31 term 1's (the pass reads them first)
        const uint32_t n_lo = __shfl_down_sync(0xFFFFFFFFu, c_lo, 1);
        const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, c_hi, 0);
        const uint32_t nxt = lane == 31 ? h0 : n_lo;
        const uint32_t term = (L == 1 ? c_lo * (uint32_t)a.ncols + c_lo
                                      : c_lo * (uint32_t)a.ncols + nxt) * a.stride;
        const uint32_t t0 = __shfl_sync(0xFFFFFFFFu, term, 0);
        const uint32_t t1 = __shfl_sync(0xFFFFFFFFu, term, 1);
        const bool has = lane < 16 || L > 2;
        const uint32_t* row = a.table + (lane < 16 ? t0 : t1) + (lane & 15) * 32;
        if (has) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
          if (a.W > 512) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 512));
        }
      }
    }
  }
  __syncthreads();

  // (C) share masks; then the warp's further candidates (when there are more than warps)
  for (uint32_t i = gw; i < a.n_cand; i += nwarps) {
    if (i != gw) {
      const uint32_t lo = a.offsets[i], hi = a.offsets[i + 1];
      for (int w = lane; w < nw; w += 32) set[w] = 0u;
      __syncwarp();
      if (offsets_sane(lo, hi, tot0, false)) {
        load_cols_regs(a.cols, lo, hi, lane, c_lo, c_hi);
        bad |= cols_bad_regs(c_lo, c_hi, hi - lo, a.ncols, set, lane);
        build_terms_regs(c_lo, c_hi, (int)(hi - lo), (uint32_t)a.ncols, a.stride, a.negative,
                         a.terms + (size_t)i * slots, lane);
      } else {
        bad = true;
      }
    }
    if (a.share) {
      const uint64_t mask = share_mask(set, sh.msets, na, nw, lane);
      if (lane == 0) a.share[i] = mask;
    }
    __syncwarp();  // the set is rebuilt for the next candidate
  }
  // a failure reaches the deferred status only for a list that the caller keeps on the device
  // (a host list's failure is the host check's to report); the archive verdict was found by
  // single threads, so the warp agrees on it first
  abad = __any_sync(0xFFFFFFFFu, abad);
  if (lane == 0) {
    if (bad && a.status_cand) atomicOr(a.status_cand, kErrInvalid);
    if (abad && a.status_arch) atomicOr(a.status_arch, kErrInvalid);
  }
  return bad || abad;
}

// F_c of candidate c of the fused pass (at most 64 archive members), a lane per member (two for
// members 32..63); `sh` (the members sharing a column with the candidate) stands for the
// column-set test. L is the candidate's length and al0 / al1 the lengths of members `lane` and
// `lane + 32` (0 when absent). Every load is issued before any comparison (none depends on
// another), so the warp waits for one round of loads. Returns F_c in every lane, and the
// candidate's row count in n.
__device__ __forceinline__ uint64_t fused_fitness_value(uint32_t c, uint32_t L, uint32_t al0,
                                                        uint32_t al1, uint32_t n_arch,
                                                        uint64_t sh, const uint32_t* counts,
                                                        const uint32_t* overlaps,
                                                        uint32_t ov_stride,
                                                        const uint32_t* arch_counts, int lane,
                                                        uint32_t& n) {
  const uint32_t m0 = (uint32_t)lane, m1 = (uint32_t)lane + 32u;
  const bool in0 = m0 < n_arch, in1 = m1 < n_arch;
  const size_t row = (size_t)c * ov_stride;
  n = counts[c];
  const uint32_t ac0 = in0 ? arch_counts[m0] : 0u, ac1 = in1 ? arch_counts[m1] : 0u;
  const uint32_t ov0 = in0 ? overlaps[row + m0] : 0u, ov1 = in1 ? overlaps[row + m1] : 0u;
  const bool has0 = in0 && ((sh >> m0) & 1ull), has1 = in1 && ((sh >> m1) & 1ull);
  const uint32_t shift = (L < 33u ? L : 33u) - 1u;
  const uint64_t qc = (uint64_t)n << shift;
  // a strictly worse member (q(a) < q(c)) does not penalise the candidate
  uint32_t best = 0;
  if (has0 && ((uint64_t)ac0 << ((al0 < 33u ? al0 : 33u) - 1u)) >= qc) best = ov0;
  if (has1 && ((uint64_t)ac1 << ((al1 < 33u ? al1 : 33u) - 1u)) >= qc) best = ov1 > best ? ov1 : best;
  best = __reduce_max_sync(0xFFFFFFFFu, best);
  return (uint64_t)(n - best) << shift;
}

// The same, stored by lane 0.
__device__ __forceinline__ void fused_fitness_mask(uint32_t c, uint32_t L, uint32_t al0,
                                                   uint32_t al1, uint32_t n_arch, uint64_t sh,
                                                   const uint32_t* counts,
                                                   const uint32_t* overlaps, uint32_t ov_stride,
                                                   const uint32_t* arch_counts, uint64_t* fitness,
                                                   int lane) {
  uint32_t n;
  const uint64_t f = fused_fitness_value(c, L, al0, al1, n_arch, sh, counts, overlaps, ov_stride,
                                         arch_counts, lane, n);
  if (lane == 0) fitness[c] = f;
}

}  // namespace prepdev
}  // namespace ebic
