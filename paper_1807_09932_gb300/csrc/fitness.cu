// Population preparation (device-side argument checks, zeroing) and the overlap-penalised
// fitness.
//
// Fitness (the project's reading of "EBIC search is driven by counting of rows", arXiv
// 1807.09932, Methods, "Handling missing values"): for candidate c with row count n_c and row
// bitmap M_c, and archive members a with column sets A_a and bitmaps M_a,
//   o(c,a) = popcount(M_c & M_a)                           (rows c shares with a)
//   p_c    = n_c - max{ o(c,a) : c and a share a column }  (0 when there is none)
//   F_c    = (uint64) p_c << (min(L_c, 33) - 1)
// The overlap pass streams each candidate bitmap once per archive member out of L1/L2 with
// 32-bit AND + popc per word and a warp reduction; the finalize pass builds the candidate's
// column set as a shared-memory bitset and tests each archive member's columns against it.
#include "ebic_internal.h"

namespace ebic {
namespace {

// A valid CSR list: offsets[0] == 0, every length in [1, 64].
__global__ void check_offsets_kernel(const uint32_t* __restrict__ offsets, uint32_t n,
                                     uint32_t* err, uint32_t* status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool bad = (i == 0 && offsets[0] != 0u);
  const uint32_t a = offsets[i], b = offsets[i + 1];
  bad |= b <= a || b - a > (uint32_t)kMaxLen;
  if (bad) {
    atomicOr(err, kErrInvalid);
    if (status) atomicOr(status, kErrInvalid);
  }
}

// Columns in range and distinct within each candidate. Runs only after the offsets passed, so
// every read stays inside cols[0 .. offsets[n]).
__global__ void check_columns_kernel(const uint16_t* __restrict__ cols,
                                     const uint32_t* __restrict__ offsets, uint32_t n,
                                     int32_t ncols, bool check, uint32_t* __restrict__ zero,
                                     size_t n_zero, uint32_t* err, uint32_t* status) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (zero && i < n_zero) zero[i] = 0u;
  if (!check || i >= n) return;
  if (*reinterpret_cast<const volatile uint32_t*>(err) != 0) return;
  const uint32_t a = offsets[i], L = offsets[i + 1] - a;
  bool bad = false;
  for (uint32_t j = 0; j < L; ++j) {
    const uint16_t c = cols[a + j];
    bad |= c >= (uint32_t)ncols;
    for (uint32_t t = 0; t < j; ++t) bad |= cols[a + t] == c;
  }
  if (bad) {
    atomicOr(err, kErrInvalid);
    if (status) atomicOr(status, kErrInvalid);
  }
}

constexpr int kOverlapWarps = 8;
constexpr int kWordsPerSegment = 2048;

// overlaps[c][a] += popcount(M_c & M_a) over the words of this block's segment.
__global__ void __launch_bounds__(kOverlapWarps * 32)
    overlap_kernel(const uint32_t* __restrict__ bitmaps, uint32_t n_cand,
                   const uint32_t* __restrict__ arch, uint32_t n_arch, int64_t W,
                   int64_t seg_words, uint32_t* __restrict__ overlaps, const uint32_t* err) {
  if (*reinterpret_cast<const volatile uint32_t*>(err) != 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x * kOverlapWarps + warp;
  if (c >= n_cand) return;
  const int64_t w0 = (int64_t)blockIdx.y * seg_words;
  const int64_t w1 = w0 + seg_words < W ? w0 + seg_words : W;
  const uint32_t* mc = bitmaps + (size_t)c * W;
  for (uint32_t a = 0; a < n_arch; ++a) {
    const uint32_t* ma = arch + (size_t)a * W;
    uint32_t part = 0;
    for (int64_t w = w0 + lane; w < w1; w += 32) part += __popc(__ldg(mc + w) & __ldg(ma + w));
    part = __reduce_add_sync(0xFFFFFFFFu, part);
    if (lane == 0 && part) atomicAdd(&overlaps[(size_t)c * n_arch + a], part);
  }
}

constexpr int kFinalizeWarps = 8;

__global__ void __launch_bounds__(kFinalizeWarps * 32)
    fitness_finalize_kernel(const uint16_t* __restrict__ cols,
                            const uint32_t* __restrict__ offsets, uint32_t n_cand,
                            const uint32_t* __restrict__ counts,
                            const uint16_t* __restrict__ acols,
                            const uint32_t* __restrict__ aoffsets, uint32_t n_arch,
                            const uint32_t* __restrict__ overlaps, uint64_t* __restrict__ fitness,
                            const uint32_t* err) {
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
  uint32_t best = 0;
  for (uint32_t a = lane; a < n_arch; a += 32) {
    const uint32_t ao = aoffsets[a], al = aoffsets[a + 1] - ao;
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

}  // namespace

cudaError_t launch_prepare(const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                           int32_t ncols, bool check, uint32_t* zero, size_t n_zero,
                           uint32_t* err, uint32_t* status, cudaStream_t s) {
  const int T = 256;
  if (check && n > 0) {
    check_offsets_kernel<<<(n + T - 1) / T, T, 0, s>>>(offsets, n, err, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t work = (check ? n : 0) > n_zero ? (check ? n : 0) : n_zero;
  if (work == 0) return cudaSuccess;
  check_columns_kernel<<<(unsigned)((work + T - 1) / T), T, 0, s>>>(cols, offsets, n, ncols,
                                                                     check, zero, n_zero, err,
                                                                     status);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const uint32_t* bitmaps, uint32_t n_cand, const uint32_t* arch_bitmaps,
                           uint32_t n_arch, int64_t words, uint32_t* overlaps, const uint32_t* err,
                           int num_sms, cudaStream_t s) {
  if (n_cand == 0 || n_arch == 0) return cudaSuccess;
  const unsigned gx = (n_cand + kOverlapWarps - 1) / kOverlapWarps;
  int64_t nseg = (words + kWordsPerSegment - 1) / kWordsPerSegment;
  const int64_t want = (4 * (int64_t)num_sms + gx - 1) / gx;  // about 4 blocks per SM
  if (nseg > want) nseg = want;
  if (nseg < 1) nseg = 1;
  if (nseg > 65535) nseg = 65535;
  int64_t seg = (words + nseg - 1) / nseg;
  seg = (seg + 31) / 32 * 32;
  nseg = (words + seg - 1) / seg;
  dim3 grid(gx, (unsigned)nseg);
  overlap_kernel<<<grid, kOverlapWarps * 32, 0, s>>>(bitmaps, n_cand, arch_bitmaps, n_arch, words,
                                                     seg, overlaps, err);
  return cudaGetLastError();
}

cudaError_t launch_fitness_finalize(const uint16_t* cols, const uint32_t* offsets, uint32_t n_cand,
                                    const uint32_t* counts, const uint16_t* arch_cols,
                                    const uint32_t* arch_offsets, uint32_t n_arch,
                                    const uint32_t* overlaps, int32_t ncols, uint64_t* fitness,
                                    const uint32_t* err, cudaStream_t s) {
  (void)ncols;
  if (n_cand == 0) return cudaSuccess;
  const unsigned grid = (n_cand + kFinalizeWarps - 1) / kFinalizeWarps;
  fitness_finalize_kernel<<<grid, kFinalizeWarps * 32, 0, s>>>(
      cols, offsets, n_cand, counts, arch_cols, arch_offsets, n_arch, overlaps, fitness, err);
  return cudaGetLastError();
}

}  // namespace ebic
