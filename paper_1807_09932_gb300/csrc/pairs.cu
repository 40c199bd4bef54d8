// Pair-table evaluation: an exact alternative encoding of the same trend rule, with the archive
// overlaps of the fitness optionally computed in the same pass.
//
// For a loaded matrix, the pair table holds one row bitmap per ordered column pair (a, b):
//   T[a*C + b] = rows where a is not missing and code[b] >= code[a]   (a != b)
//   T[a*C + a] = rows where a is not missing
// It is built once per matrix by the population evaluator itself, run on the population of all
// C*C pairs and singles (its bitmaps output is the table), so it carries exactly the evaluator's
// semantics. Then, for a candidate (c_1..c_L), with the "greater or equal" relation of arXiv
// 1807.09932 (Methods, "Handling missing values"):
//   increasing: AND_i T[c_i*C + c_{i+1}]       (each factor also says c_i is present; c_L is
//               present because code[c_L] >= code[c_{L-1}] >= 1)
//   decreasing: AND_i T[c_{i+1}*C + c_i]       (each factor says c_{i+1} is present and
//               code[c_i] >= code[c_{i+1}]; so c_1 is present too)
//   L = 1:      T[c_1*C + c_1]
// so a candidate costs one 32-bit AND per 32 rows per column, streamed from the table.
//
// Table rows are stored with a stride of ceil(W / 512) * 512 words whose padding words are zero,
// so a lane reads four consecutive words of each 128-word part of an item with one 16-byte load
// and never tests a bound: a padding word ANDs to zero and counts nothing.
//
// Work order: items are (range of 512 words = 16,384 rows, group of 24 candidates), taken
// round-robin by a persistent grid in range-major order, so all CTAs work on the same few row
// ranges at a time and the table rows of those ranges stay in L2 while every candidate reads
// them; each table word comes from HBM about once per evaluation. A CTA's items are fixed
// (round-robin), but its warps take the items' candidates in order from a counter of the CTA as
// each warp becomes free, so a warp that drew short candidates takes more of them. The
// preparation kernel has already turned the candidate into its term list (the table-row offsets
// of its consecutive pairs), which the warp loads while it walks its previous candidate. The
// chain goes two pairs per step, each step keeping eight 512-byte warp loads in flight (two
// pairs x four parts; with negative trends one pair, both orders); the next candidate's first
// step is prefetched into L2 before the epilogue (a prefetch holds no registers), and the
// preparation kernel, which builds the term lists while DRAM is otherwise idle, prefetches every
// candidate's first step in the first two ranges, the rows of the pass's first wave. A part stops
// loading once all its words are zero and the walk
// stops when all are: long chains match no row of most ranges. Larger items amortise the
// per-item work (the term list, the reductions and atomics of the epilogue) over more rows.
//
// Fused overlaps (the fitness's o(c, a) = popcount(M_c & M_a), Methods, "Handling missing
// values" and the archive rule of the fitness): the warp that has just built a candidate's words
// of an item ANDs them with the archive members' words of the same rows (archive rows padded to
// the same stride) and adds the popcounts, so candidate bitmaps never go through HBM. Items
// where the candidate matches no row are skipped, and so are archive members that the caller
// does not need (those sharing no column with the candidate cannot penalise it). By the number
// of non-zero words in the item: up to 12 are walked by a lane per member (no reductions); up
// to 32 are compacted to one per lane and members go two per warp reduction; denser items
// take the wanted members two at a time over all words.
#include "pair_chain.cuh"

namespace ebic {
namespace {

using namespace pairdev;

template <bool NEG, bool BITMAPS, bool OVERLAP>
__global__ void __launch_bounds__(kPairThreads, 1) pair_eval_kernel(const PairArgs p) {
  // per warp: 128 words for the coalesced bitmap store, or its compacted non-zero words
  __shared__ __align__(16) uint32_t stage[kPairWarps][kRangeWords];
  __shared__ uint32_t next_unit;  // the CTA's next (item, candidate) unit
  if (threadIdx.x == 0) next_unit = 0u;
  dev::pdl_wait();     // the preparation (checks, zeroed outputs) is complete and visible
  dev::pdl_trigger();  // the finalize launch may be scheduled now; it waits for this grid itself
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the preparation's verdicts (per block, or the call's error word), requested here and checked
  // once the warp's first term list is requested too: the two loads are in flight together, and
  // no table row is read before the check
  uint32_t f = 0;
  if (p.flags) {
    for (uint32_t i = lane; i < p.n_flags; i += 32) f |= p.flags[i];
  } else if (lane == 0) {
    f = *reinterpret_cast<const volatile uint32_t*>(p.err);
  }
  __syncthreads();  // next_unit is set
  pair_items<NEG, BITMAPS, OVERLAP>(p, stage[warp], &next_unit, [&]() {
    f = __reduce_or_sync(0xFFFFFFFFu, f);
    if (p.flags && blockIdx.x == 0 && threadIdx.x == 0) *p.err_out = f;  // CTA 0 records it
    return f == 0u;  // else invalid input: nothing is evaluated
  });
}

template <bool NEG, bool BITMAPS>
cudaError_t launch_variant(const PairArgs& p, int grid, bool pdl, cudaStream_t s) {
  if (p.arch)
    return launch_maybe_pdl(pdl, pair_eval_kernel<NEG, BITMAPS, true>, dim3(grid),
                            dim3(kPairThreads), 0, s, p);
  return launch_maybe_pdl(pdl, pair_eval_kernel<NEG, BITMAPS, false>, dim3(grid),
                          dim3(kPairThreads), 0, s, p);
}

}  // namespace

cudaError_t launch_pair_eval(const PairArgs& p, bool negative, int grid, bool pdl,
                             cudaStream_t s) {
  if (p.n_cand == 0) return cudaSuccess;
  if (p.arch && p.n_arch > (uint32_t)kPairMaxArch) return cudaErrorInvalidValue;
  if (p.stride % kItemWords != 0 || (int64_t)p.stride < p.W) return cudaErrorInvalidValue;
  if ((uint64_t)p.C * (uint64_t)p.C * p.stride > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  if (p.arch && (p.ov_stride % 2 != 0 || p.ov_stride < p.n_arch)) return cudaErrorInvalidValue;
  count_launch();
  const bool bm = p.bitmaps != nullptr;
  if (negative)
    return bm ? launch_variant<true, true>(p, grid, pdl, s)
              : launch_variant<true, false>(p, grid, pdl, s);
  return bm ? launch_variant<false, true>(p, grid, pdl, s)
            : launch_variant<false, false>(p, grid, pdl, s);
}

}  // namespace ebic
