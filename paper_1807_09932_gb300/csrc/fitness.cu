// Population preparation (device-side argument checks, zeroing) and the overlap-penalised
// fitness.
//
// Fitness (the project's reading of "EBIC search is driven by counting of rows", arXiv
// 1807.09932, Methods, "Handling missing values"): for candidate c with row count n_c and row
// bitmap M_c, and archive members a with column sets A_a and bitmaps M_a,
//   q(x)   = (uint64) n_x << (min(L_x, 33) - 1)               (raw quality)
//   o(c,a) = popcount(M_c & M_a)                              (rows c shares with a)
//   p_c    = n_c - max{ o(c,a) : a shares a column with c and q(a) >= q(c) }   (0 if none)
//   F_c    = (uint64) p_c << (min(L_c, 33) - 1)
// Only archive members at least as good as the candidate penalise it, so a candidate that
// improves on an archived bicluster is not pushed away from it.
// The overlap pass reads every candidate bitmap from HBM once, against archive words staged in
// shared memory; the finalize pass builds the candidate's column set as a shared-memory bitset and
// tests each archive member's columns against it.
#include <algorithm>

#include "prep_dev.cuh"

namespace ebic {
namespace {

using namespace prepdev;

constexpr int kPrepWarps = 8;

// Device-side check of up to two CSR candidate lists (a warp per candidate) and zeroing of up to
// two outputs, in one launch.
__global__ void __launch_bounds__(kPrepWarps * 32) prepare_kernel(PrepareArgs a) {
  __shared__ uint32_t sets[kPrepWarps][kSetWords];
  dev::pdl_trigger();  // a following pair-table pass may be scheduled; it waits for this grid
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nthreads = (size_t)gridDim.x * blockDim.x;
  if (a.zero)
    for (size_t i = tid; i < a.n_zero; i += nthreads) a.zero[i] = 0u;
  if (a.zero2)
    for (size_t i = tid; i < a.n_zero2; i += nthreads) a.zero2[i] = 0u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t gw = blockIdx.x * kPrepWarps + warp, nwarps = gridDim.x * kPrepWarps;
  bool bad = false;
#pragma unroll
  for (int l = 0; l < 2; ++l)
    for (uint32_t i = gw; i < a.n[l]; i += nwarps)
      bad |= check_candidate_warp(a.cols[l], a.offsets[l], a.n[l], i, a.ncols, sets[warp], lane);
  if (a.terms) {
    const uint32_t total = a.offsets[0][a.n_terms_cand];
    const int slots = term_slots(a.negative);
    for (uint32_t i = gw; i < a.n_terms_cand; i += nwarps) {
      const uint32_t lo = a.offsets[0][i], hi = a.offsets[0][i + 1];
      if (offsets_sane(lo, hi, total, i == 0))
        build_terms_warp(a.cols[0], lo, hi, (uint32_t)a.pair_cols, a.pair_stride, a.negative,
                         a.terms + (size_t)i * slots, lane);
    }
  }
  if (lane == 0) report_invalid(bad, a.err, a.status);
}

// Preparation of the fused evaluation + overlap pass (see launch_fused_prepare).
__global__ void __launch_bounds__(kPrepWarps * 32) fused_prepare_kernel(FusedPrepareArgs a) {
  __shared__ PrepShared<kPrepWarps> sh;
  dev::pdl_trigger();  // the pair-table pass may be scheduled; it waits for this grid
  const bool bad = fused_prepare_body<kPrepWarps>(a, sh, blockIdx.x, gridDim.x);
  // the block's verdict, stored (not accumulated) in its own flag: nothing needs zeroing first
  const bool block_bad = __syncthreads_or(bad) != 0;
  if (threadIdx.x == 0) a.flags[blockIdx.x] = block_bad ? kErrInvalid : 0u;
}

// F_c for the fused pass: a warp per candidate, a lane per archive member.
__global__ void __launch_bounds__(kPrepWarps * 32)
    fused_finalize_kernel(const uint32_t* __restrict__ offsets, uint32_t n_cand,
                          const uint32_t* __restrict__ counts,
                          const uint32_t* __restrict__ aoffsets, uint32_t n_arch,
                          const uint32_t* __restrict__ overlaps, uint32_t ov_stride,
                          const uint32_t* __restrict__ arch_counts,
                          const uint64_t* __restrict__ share, uint64_t* __restrict__ fitness,
                          const uint32_t* err, uint32_t* __restrict__ counts_out,
                          uint32_t* err_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x * kPrepWarps + warp;
  // the call's inputs (written before the preparation ran) are read before the wait
  const bool live = c < n_cand;
  const uint32_t L = live ? offsets[c + 1] - offsets[c] : 1u;
  const uint32_t al0 = lane < (int)n_arch ? aoffsets[lane + 1] - aoffsets[lane] : 0u;
  const uint32_t al1 = lane + 32 < (int)n_arch ? aoffsets[lane + 33] - aoffsets[lane + 32] : 0u;
  dev::pdl_wait();  // the pair-table pass is complete and visible
  // the error word is read alongside the scores; a failed call's scores are read but not stored
  const uint32_t e = *reinterpret_cast<const volatile uint32_t*>(err);
  uint32_t n = 0;
  uint64_t f = 0;
  if (live) {
    const uint64_t sh = n_arch ? share[c] : 0ull;
    f = fused_fitness_value(c, L, al0, al1, n_arch, sh, counts, overlaps, ov_stride, arch_counts,
                            lane, n);
  }
  if (err_out && blockIdx.x == 0 && threadIdx.x == 0) *err_out = e;
  if (!live || e != 0 || lane != 0) return;
  fitness[c] = f;
  if (counts_out) counts_out[c] = n;
}

// Carry-save adder: a + b + c = 2 * carry + sum, bit by bit (two 3-input logic ops).
__device__ __forceinline__ void csa(uint32_t& carry, uint32_t& sum, uint32_t a, uint32_t b,
                                    uint32_t c) {
  sum = a ^ b ^ c;
  carry = (a & b) | (c & (a ^ b));
}

// Total population count of 8 words with a carry-save tree (Harley and Seal): the words are
// summed bit-parallel into ones/twos/fours/eights, and only those four are popcounted, so the
// popcount pipe does 4 operations instead of 8 and the ALU pipe absorbs the rest.
__device__ __forceinline__ uint32_t popc8(const uint32_t (&w)[8]) {
  uint32_t t1, t2, t3, o1, o2, ones, f1, tw1;
  csa(t1, o1, w[0], w[1], w[2]);
  csa(t2, o2, o1, w[3], w[4]);
  csa(t3, ones, o2, w[5], w[6]);
  const uint32_t t4 = ones & w[7];
  ones ^= w[7];
  csa(f1, tw1, t1, t2, t3);
  const uint32_t f2 = tw1 & t4;
  const uint32_t twos = tw1 ^ t4;
  const uint32_t eights = f1 & f2;
  const uint32_t fours = f1 ^ f2;
  return __popc(ones) + 2u * __popc(twos) + 4u * __popc(fours) + 8u * __popc(eights);
}

constexpr int kOverlapWarps = 8;
constexpr int kOvCPW = 4;                          // candidates per warp (register blocking)
constexpr int kOvCands = kOverlapWarps * kOvCPW;   // candidates per block
constexpr int kOvNPL = 8;                          // words per lane per sub-segment
constexpr int kOvSub = 32 * kOvNPL;                // words per sub-segment (256)
constexpr int kOvSubs = 2;                         // sub-segments per block (512 words)
constexpr int kOvArch = 32;                        // archive members staged per pass

// overlaps[c][a] += popcount(M_c & M_a) over this block's words, for the block's 32 candidates
// and every archive member. The archive's words of each 256-word sub-segment are staged in
// shared memory once per block and read by all warps; each warp keeps 4 candidates' words in
// registers, so an archive word read from shared memory serves 4 AND+popc. Partial sums live in
// shared memory per (candidate, member) and reach HBM as one atomicAdd each per block.
__global__ void __launch_bounds__(kOverlapWarps * 32)
    overlap_kernel(const uint32_t* __restrict__ bitmaps, uint32_t n_cand,
                   const uint32_t* __restrict__ arch, uint32_t n_arch, int64_t W,
                   uint32_t* __restrict__ overlaps, uint32_t* __restrict__ arch_counts,
                   const uint32_t* err) {
  __shared__ uint32_t arch_s[kOvArch][kOvSub];
  __shared__ uint32_t part_s[kOvCands][kOvArch];
  if (*reinterpret_cast<const volatile uint32_t*>(err) != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t c0 = blockIdx.x * kOvCands + warp * kOvCPW;  // this warp's first candidate
  const int64_t wblk = (int64_t)blockIdx.y * kOvSub * kOvSubs;
  for (uint32_t a0 = 0; a0 < n_arch; a0 += kOvArch) {
    const int na = n_arch - a0 < (uint32_t)kOvArch ? (int)(n_arch - a0) : kOvArch;
    for (int i = tid; i < kOvCands * kOvArch; i += blockDim.x) (&part_s[0][0])[i] = 0u;
    for (int sub = 0; sub < kOvSubs; ++sub) {
      const int64_t ws = wblk + (int64_t)sub * kOvSub;
      if (ws >= W) break;
      __syncthreads();
      for (int i = tid; i < na * kOvSub; i += blockDim.x) {
        const int a = i / kOvSub, w = i % kOvSub;
        arch_s[a][w] = ws + w < W ? __ldg(arch + (size_t)(a0 + a) * W + ws + w) : 0u;
      }
      __syncthreads();
      if (blockIdx.x == 0) {  // the archive's own row counts, once per word segment
        for (int a = warp; a < na; a += kOverlapWarps) {
          uint32_t n = 0;
#pragma unroll
          for (int t = 0; t < kOvNPL; ++t) n += __popc(arch_s[a][lane + 32 * t]);
          n = __reduce_add_sync(0xFFFFFFFFu, n);
          if (lane == 0 && n) atomicAdd(&arch_counts[a0 + a], n);
        }
      }
      uint32_t cw[kOvCPW][kOvNPL];
#pragma unroll
      for (int c = 0; c < kOvCPW; ++c)
#pragma unroll
        for (int t = 0; t < kOvNPL; ++t) {
          const int64_t w = ws + lane + 32 * t;
          cw[c][t] = (c0 + c < n_cand && w < W) ? __ldg(bitmaps + (size_t)(c0 + c) * W + w) : 0u;
        }
      // a candidate whose 256 words here are all zero contributes nothing to any overlap: long
      // chains match few rows, so most of their sub-segments are skipped (warp-uniform flags)
      bool nz[kOvCPW];
      bool any = false;
#pragma unroll
      for (int c = 0; c < kOvCPW; ++c) {
        uint32_t o = 0;
#pragma unroll
        for (int t = 0; t < kOvNPL; ++t) o |= cw[c][t];
        nz[c] = __any_sync(0xFFFFFFFFu, o != 0u);
        any |= nz[c];
      }
      if (any) {
        for (int a = 0; a < na; ++a) {
          uint32_t x[kOvNPL];
#pragma unroll
          for (int t = 0; t < kOvNPL; ++t) x[t] = arch_s[a][lane + 32 * t];
#pragma unroll
          for (int c = 0; c < kOvCPW; ++c) {
            if (!nz[c]) continue;
            uint32_t w[kOvNPL];
#pragma unroll
            for (int t = 0; t < kOvNPL; ++t) w[t] = cw[c][t] & x[t];
            const uint32_t v = __reduce_add_sync(0xFFFFFFFFu, popc8(w));
            if (lane == 0) part_s[warp * kOvCPW + c][a] += v;
          }
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < kOvCands * na; i += blockDim.x) {
      const int c = i / na, a = i % na;
      const uint32_t v = part_s[c][a];
      const uint32_t cand = blockIdx.x * kOvCands + c;
      if (v && cand < n_cand) atomicAdd(&overlaps[(size_t)cand * n_arch + a0 + a], v);
    }
    __syncthreads();
  }
}

constexpr int kFinalizeWarps = 8;

__global__ void __launch_bounds__(kFinalizeWarps * 32)
    fitness_finalize_kernel(const uint16_t* __restrict__ cols,
                            const uint32_t* __restrict__ offsets, uint32_t n_cand,
                            const uint32_t* __restrict__ counts,
                            const uint16_t* __restrict__ acols,
                            const uint32_t* __restrict__ aoffsets, uint32_t n_arch,
                            const uint32_t* __restrict__ overlaps,
                            const uint32_t* __restrict__ arch_counts,
                            uint64_t* __restrict__ fitness, const uint32_t* err) {
  __shared__ uint32_t colset[kFinalizeWarps][(kMaxCols + 31) / 32];
  if (*reinterpret_cast<const volatile uint32_t*>(err) != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x * kFinalizeWarps + warp;
  if (c >= n_cand) return;
  uint32_t* set = colset[warp];
  for (int i = lane; i < (kMaxCols + 31) / 32; i += 32) set[i] = 0u;
  __syncwarp();
  const uint32_t o = offsets[c], L = offsets[c + 1] - o;
  for (uint32_t i = lane; i < L; i += 32) {
    const uint32_t col = cols[o + i];
    atomicOr(&set[col >> 5], 1u << (col & 31));
  }
  __syncwarp();
  const uint64_t qc = (uint64_t)counts[c] << ((L < 33u ? L : 33u) - 1u);
  uint32_t best = 0;
  for (uint32_t a = lane; a < n_arch; a += 32) {
    const uint32_t ao = aoffsets[a], al = aoffsets[a + 1] - ao;
    const uint64_t qa = (uint64_t)arch_counts[a] << ((al < 33u ? al : 33u) - 1u);
    if (qa < qc) continue;  // a strictly worse member does not penalise the candidate
    bool share = false;
    for (uint32_t j = 0; j < al && !share; ++j) {
      const uint32_t col = acols[ao + j];
      share = (set[col >> 5] >> (col & 31)) & 1u;
    }
    if (share) {
      const uint32_t ov = overlaps[(size_t)c * n_arch + a];
      best = ov > best ? ov : best;
    }
  }
  best = __reduce_max_sync(0xFFFFFFFFu, best);
  if (lane == 0) {
    const uint32_t shift = (L < 33u ? L : 33u) - 1u;
    fitness[c] = (uint64_t)(counts[c] - best) << shift;
  }
}

__global__ void gather_rows_kernel(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                                   const int32_t* __restrict__ idx, uint32_t n, int64_t W,
                                   uint32_t* __restrict__ dst) {
  const uint64_t total = (uint64_t)n * (uint64_t)W;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = i / (uint64_t)W, w = i - k * (uint64_t)W;
    const int32_t r = idx[k];
    dst[i] = r >= 0 ? a[(uint64_t)r * W + w] : b[(uint64_t)(-r - 1) * W + w];
  }
}

}  // namespace

cudaError_t launch_gather_rows(const uint32_t* a, const uint32_t* b, const int32_t* idx,
                               uint32_t n, int64_t W, uint32_t* dst, cudaStream_t s) {
  if (n == 0 || W == 0) return cudaSuccess;
  const uint64_t total = (uint64_t)n * (uint64_t)W;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  gather_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, b, idx, n, W, dst);
  return cudaGetLastError();
}

cudaError_t ready_prepare() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, prepare_kernel);
}

cudaError_t launch_prepare(const PrepareArgs& a, cudaStream_t s) {
  size_t warps = a.n[0] > a.n[1] ? a.n[0] : a.n[1];
  if (a.terms && a.n_terms_cand > warps) warps = a.n_terms_cand;
  const size_t zero = a.n_zero > a.n_zero2 ? a.n_zero : a.n_zero2;
  size_t blocks = (warps + kPrepWarps - 1) / kPrepWarps;
  const size_t zb = (zero + kPrepWarps * 32 * 4 - 1) / (kPrepWarps * 32 * 4);
  blocks = blocks > zb ? blocks : zb;
  if (blocks == 0) return cudaSuccess;
  if (blocks > 4096) blocks = 4096;  // grid-stride beyond
  count_launch();
  prepare_kernel<<<(unsigned)blocks, kPrepWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

uint32_t fused_prepare_blocks(uint32_t n_cand, uint32_t n_arch, uint32_t stride, int num_sms) {
  size_t blocks = (n_cand + kPrepWarps - 1) / kPrepWarps;
  const size_t cb = ((size_t)(n_arch + 1) * stride + kPrepWarps * 32 * 8 - 1) /
                    (kPrepWarps * 32 * 8);
  blocks = blocks > cb ? blocks : cb;
  const size_t cap = (size_t)(num_sms > 0 ? num_sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  return (uint32_t)blocks;
}

cudaError_t launch_fused_prepare(const FusedPrepareArgs& a, uint32_t blocks, cudaStream_t s) {
  if (a.n_arch > (uint32_t)kPairMaxArch) return cudaErrorInvalidValue;
  count_launch();
  fused_prepare_kernel<<<blocks, kPrepWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused_finalize(const uint32_t* offsets, uint32_t n_cand, const uint32_t* counts,
                                  const uint32_t* arch_offsets, uint32_t n_arch,
                                  const uint32_t* overlaps, uint32_t ov_stride,
                                  const uint32_t* arch_counts, const uint64_t* share,
                                  uint64_t* fitness, const uint32_t* err, uint32_t* counts_out,
                                  uint32_t* err_out, bool pdl, cudaStream_t s) {
  if (n_cand == 0) return cudaSuccess;
  count_launch();
  return launch_maybe_pdl(pdl, fused_finalize_kernel,
                          dim3((n_cand + kPrepWarps - 1) / kPrepWarps), dim3(kPrepWarps * 32), 0,
                          s, offsets, n_cand, counts, arch_offsets, n_arch, overlaps, ov_stride,
                          arch_counts, share, fitness, err, counts_out, err_out);
}

cudaError_t launch_overlap(const uint32_t* bitmaps, uint32_t n_cand, const uint32_t* arch_bitmaps,
                           uint32_t n_arch, int64_t words, uint32_t* overlaps,
                           uint32_t* arch_counts, const uint32_t* err, int num_sms,
                           cudaStream_t s) {
  (void)num_sms;
  if (n_cand == 0 || n_arch == 0) return cudaSuccess;
  const int64_t per_block = (int64_t)kOvSub * kOvSubs;
  const int64_t gy = (words + per_block - 1) / per_block;
  if (gy > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((n_cand + kOvCands - 1) / kOvCands, (unsigned)gy);
  count_launch();
  overlap_kernel<<<grid, kOverlapWarps * 32, 0, s>>>(bitmaps, n_cand, arch_bitmaps, n_arch, words,
                                                     overlaps, arch_counts, err);
  return cudaGetLastError();
}

cudaError_t launch_fitness_finalize(const uint16_t* cols, const uint32_t* offsets, uint32_t n_cand,
                                    const uint32_t* counts, const uint16_t* arch_cols,
                                    const uint32_t* arch_offsets, uint32_t n_arch,
                                    const uint32_t* overlaps, const uint32_t* arch_counts,
                                    uint64_t* fitness, const uint32_t* err, cudaStream_t s) {
  if (n_cand == 0) return cudaSuccess;
  const unsigned grid = (n_cand + kFinalizeWarps - 1) / kFinalizeWarps;
  count_launch();
  fitness_finalize_kernel<<<grid, kFinalizeWarps * 32, 0, s>>>(
      cols, offsets, n_cand, counts, arch_cols, arch_offsets, n_arch, overlaps, arch_counts,
      fitness, err);
  return cudaGetLastError();
}

}  // namespace ebic
