// Pair-table evaluation: an exact alternative encoding of the same trend rule.
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
// Work order: items are (range of 4 row tiles of 32 words, group of 32 candidates), taken
// round-robin by a persistent grid in range-major order, so all CTAs work on the same few row
// ranges at a time and the table rows of those ranges stay in L2 while every candidate reads
// them; each table word comes from HBM about once per evaluation. Each warp takes one candidate
// of its item: it reads the column list once (a lane per column), turns it into the table rows
// of the consecutive pairs (a lane per pair), and walks the chain four pairs at a time, each
// step issuing 16 independent 128-byte loads (one per pair and tile; 32 with negative trends).
#include "ebic_internal.h"

namespace ebic {
namespace {

constexpr int kPairThreads = 1024;
constexpr int kPairWarps = kPairThreads / 32;

constexpr int kPairTiles = 4;  // 32-word row tiles per item (4,096 rows)

template <bool NEG, bool BITMAPS>
__global__ void __launch_bounds__(kPairThreads, 1)
    pair_eval_kernel(const uint32_t* __restrict__ table, int32_t C, int64_t W,
                     const uint16_t* __restrict__ cols, const uint32_t* __restrict__ offsets,
                     uint32_t n_cand, uint32_t* __restrict__ counts,
                     uint32_t* __restrict__ bitmaps, const uint32_t* err) {
  if (*reinterpret_cast<const volatile uint32_t*>(err) != 0) return;  // invalid input
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t span = 32 * kPairTiles;  // words per item
  const int64_t n_ranges = (W + span - 1) / span;
  const int64_t n_groups = (n_cand + kPairWarps - 1) / kPairWarps;
  const int64_t n_items = n_ranges * n_groups;
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int64_t range = it / n_groups, grp = it - range * n_groups;
    const uint32_t cand = (uint32_t)(grp * kPairWarps + warp);
    if (cand >= n_cand) continue;  // warp-uniform
    const uint32_t o = offsets[cand];
    const int L = (int)(offsets[cand + 1] - o);
    // lane i holds column i and 32 + i, then the table rows of its consecutive pairs:
    // fwd(i) = c_i*C + c_{i+1} (increasing), bwd(i) = c_{i+1}*C + c_i (decreasing)
    const uint32_t c_lo = lane < L ? cols[o + lane] : 0u;
    const uint32_t c_hi = lane + 32 < L ? cols[o + 32 + lane] : 0u;
    const uint32_t n_lo = __shfl_down_sync(0xFFFFFFFFu, c_lo, 1);
    const uint32_t n_hi = __shfl_down_sync(0xFFFFFFFFu, c_hi, 1);
    const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, c_hi, 0);
    const uint32_t next_lo = lane == 31 ? h0 : n_lo;   // c_{i+1} for i = lane
    const uint32_t fwd_lo = L == 1 ? c_lo * C + c_lo : c_lo * C + next_lo;
    const uint32_t fwd_hi = c_hi * C + n_hi;
    const uint32_t bwd_lo = next_lo * C + c_lo, bwd_hi = n_hi * C + c_hi;
    const int n_terms = L == 1 ? 1 : L - 1;
    const int64_t w0 = range * span + lane;
    uint32_t x[kPairTiles], y[kPairTiles];
#pragma unroll
    for (int j = 0; j < kPairTiles; ++j) x[j] = y[j] = 0xFFFFFFFFu;
    for (int i0 = 0; i0 < n_terms; i0 += 4) {
      uint32_t v[4][kPairTiles], u[4][kPairTiles];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k;
#pragma unroll
        for (int j = 0; j < kPairTiles; ++j) v[k][j] = u[k][j] = 0xFFFFFFFFu;
        if (i < n_terms) {  // warp-uniform
          const uint32_t pf = i < 32 ? __shfl_sync(0xFFFFFFFFu, fwd_lo, i)
                                     : __shfl_sync(0xFFFFFFFFu, fwd_hi, i - 32);
          const uint32_t* rf = table + (size_t)pf * W;
          uint32_t pb = 0;
          if (NEG && L > 1)
            pb = i < 32 ? __shfl_sync(0xFFFFFFFFu, bwd_lo, i)
                        : __shfl_sync(0xFFFFFFFFu, bwd_hi, i - 32);
          const uint32_t* rb = table + (size_t)pb * W;
#pragma unroll
          for (int j = 0; j < kPairTiles; ++j) {
            const int64_t w = w0 + 32 * j;
            if (w < W) {
              v[k][j] = __ldg(rf + w);
              if (NEG && L > 1) u[k][j] = __ldg(rb + w);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kPairTiles; ++j) {
        x[j] &= (v[0][j] & v[1][j]) & (v[2][j] & v[3][j]);
        if (NEG) y[j] &= (u[0][j] & u[1][j]) & (u[2][j] & u[3][j]);
      }
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kPairTiles; ++j) {
      const int64_t w = w0 + 32 * j;
      uint32_t r = x[j];
      if (NEG && L > 1) r |= y[j];
      if (w < W) {
        if (BITMAPS) bitmaps[(size_t)cand * W + w] = r;
        cnt += __popc(r);
      }
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (lane == 0 && cnt) atomicAdd(&counts[cand], cnt);
  }
}

}  // namespace

cudaError_t launch_pair_eval(const uint32_t* table, int32_t C, int64_t W, const uint16_t* cols,
                             const uint32_t* offsets, uint32_t n_cand, bool negative,
                             uint32_t* counts, uint32_t* bitmaps, const uint32_t* err,
                             int num_sms, cudaStream_t s) {
  if (n_cand == 0) return cudaSuccess;
  const int grid = num_sms;
  count_launch();
  if (negative) {
    if (bitmaps)
      pair_eval_kernel<true, true><<<grid, kPairThreads, 0, s>>>(table, C, W, cols, offsets,
                                                                  n_cand, counts, bitmaps, err);
    else
      pair_eval_kernel<true, false><<<grid, kPairThreads, 0, s>>>(table, C, W, cols, offsets,
                                                                   n_cand, counts, bitmaps, err);
  } else {
    if (bitmaps)
      pair_eval_kernel<false, true><<<grid, kPairThreads, 0, s>>>(table, C, W, cols, offsets,
                                                                   n_cand, counts, bitmaps, err);
    else
      pair_eval_kernel<false, false><<<grid, kPairThreads, 0, s>>>(table, C, W, cols, offsets,
                                                                    n_cand, counts, bitmaps, err);
  }
  return cudaGetLastError();
}

}  // namespace ebic
