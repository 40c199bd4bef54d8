// Rank transform: float32 matrix -> per-row dense ranks in the evaluator's layout (one pass).
//
// The evaluator only ever asks whether one value of a row is >= another value of the same row
// (arXiv 1807.09932, Methods, "Handling missing values": the "greater or equal" relation between
// the values in the candidate's columns). A per-row dense rank, rank(x) = number of distinct
// non-missing values of the row strictly below x, keeps that relation exactly:
// x <= y  <=>  rank(x) <= rank(y). Stored codes are rank + 1 (1..C); missing values (NaN,
// exclusion on) and padding rows get code 0, below every real code; with exclusion off NaN is
// first replaced by the fill value.
//
// Float order without float compares: the IEEE bit pattern is mapped to an unsigned key that
// orders like the value (-0 folded onto +0, negatives bit-inverted, positives given the top bit),
// so ties, signed zeros, infinities and subnormals are exact whatever the FTZ mode.
//
// One CTA per slab of rows (VEC row groups). Each warp takes one row at a time: it loads the
// row's keys into its own shared buffer as (key << 32 | column) pairs, sorts them with a bitonic
// network, and walks the sorted run with a warp prefix count of "first of a new key" flags to get
// the dense rank of every column. Ranks are written as bytes/halves into a shared slab tile
// laid out as the HBM layout (with one padding word per column against bank conflicts), then the
// tile is copied out with coalesced 32-bit stores, 128*VEC contiguous bytes per column.
#include "ebic_internal.h"

namespace ebic {
namespace {

constexpr uint32_t kMissingKey = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t order_key(float x, int exclude, float fill) {
  uint32_t b = __float_as_uint(x);
  if ((b & 0x7FFFFFFFu) > 0x7F800000u) {  // NaN: a missing value
    if (exclude) return kMissingKey;
    b = __float_as_uint(fill);
  }
  if (b == 0x80000000u) b = 0u;  // -0 == +0
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

template <int WIDTH, int VEC>
__global__ void __launch_bounds__(512) rank_transform_kernel(const float* __restrict__ X,
                                                            int64_t R, int C, int64_t ld,
                                                            int exclude, float fill,
                                                            uint32_t* __restrict__ out,
                                                            int64_t Q, int N, int nwarps) {
  constexpr int RPG = WIDTH == 8 ? 128 : 64;  // rows per group
  constexpr int RPS = RPG * VEC;              // rows per slab
  constexpr uint32_t MISSING = 0u;  // code of a missing value and of padding rows
  constexpr int TROW = 32 * VEC + 1;          // padded words per column in the tile
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* tile = reinterpret_cast<uint32_t*>(smem);
  unsigned long long* sortbuf =
      reinterpret_cast<unsigned long long*>(smem + (((size_t)C * TROW * 4 + 15) & ~(size_t)15));

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  unsigned long long* buf = sortbuf + (size_t)warp * N;
  const int npl = N / 32;  // sorted positions per lane in the ranking pass

  for (int rho = warp; rho < RPS; rho += nwarps) {
    const int64_t r = q * RPS + rho;
    const int j = rho / RPG, rr = rho % RPG, l = rr & 31, k = rr >> 5;
    uint8_t* cell0 = reinterpret_cast<uint8_t*>(tile) + ((size_t)l * VEC + j) * 4 +
                     (WIDTH == 8 ? k : 2 * k);
    if (r >= R) {  // padding rows hold the missing code in every column
      for (int c = lane; c < C; c += 32) {
        uint8_t* cell = cell0 + (size_t)c * TROW * 4;
        if (WIDTH == 8) *cell = (uint8_t)MISSING;
        else *reinterpret_cast<uint16_t*>(cell) = (uint16_t)MISSING;
      }
      continue;
    }
    const float* row = X + r * ld;
    for (int i = lane; i < N; i += 32)
      buf[i] = i < C ? ((unsigned long long)order_key(row[i], exclude, fill) << 32) | (uint32_t)i
                     : ~0ull;
    __syncwarp();
    // bitonic sort, ascending, N a power of two
    for (int kk = 2; kk <= N; kk <<= 1) {
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int p = lane; p < N / 2; p += 32) {
          const int i = 2 * jj * (p / jj) + (p % jj);
          const int ixj = i + jj;
          const unsigned long long x = buf[i], y = buf[ixj];
          const bool up = (i & kk) == 0;
          if ((x > y) == up) { buf[i] = y; buf[ixj] = x; }
        }
        __syncwarp();
      }
    }
    // dense rank: number of distinct keys up to and including this position, minus one
    const int p0 = lane * npl;
    uint32_t cnt = 0;
    for (int t = 0; t < npl; ++t) {
      const int p = p0 + t;
      const uint32_t key = (uint32_t)(buf[p] >> 32);
      const bool fresh = key != kMissingKey && (p == 0 || (uint32_t)(buf[p - 1] >> 32) != key);
      cnt += fresh;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= d) incl += v;
    }
    uint32_t run = incl - cnt;
    for (int t = 0; t < npl; ++t) {
      const int p = p0 + t;
      const unsigned long long e = buf[p];
      const uint32_t key = (uint32_t)(e >> 32), c = (uint32_t)e;
      const bool fresh = key != kMissingKey && (p == 0 || (uint32_t)(buf[p - 1] >> 32) != key);
      run += fresh;
      if (c < (uint32_t)C) {
        const uint32_t rank = key == kMissingKey ? MISSING : run;  // 1-based dense rank
        uint8_t* cell = cell0 + (size_t)c * TROW * 4;
        if (WIDTH == 8) *cell = (uint8_t)rank;
        else *reinterpret_cast<uint16_t*>(cell) = (uint16_t)rank;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // copy out: column c of slab q is 32*VEC contiguous words in HBM
  const int wpc = 32 * VEC;
  for (int64_t idx = threadIdx.x; idx < (int64_t)C * wpc; idx += blockDim.x) {
    const int64_t c = idx / wpc, i = idx % wpc;
    out[(c * Q + q) * wpc + i] = tile[c * TROW + i];
  }
}

template <int WIDTH, int VEC>
cudaError_t launch_rank_layout(const Layout& L, const float* dX, int64_t ld, int exclude,
                               float fill, uint32_t* ranks, cudaStream_t s) {
  int N = 32;
  while (N < L.cols) N <<= 1;
  const size_t tile_bytes = (((size_t)L.cols * (32 * VEC + 1) * 4) + 15) & ~(size_t)15;
  const size_t per_warp = (size_t)N * 8;
  int nwarps = (int)((kSmemDynMax - tile_bytes) / per_warp);
  if (nwarps > 16) nwarps = 16;
  if (nwarps < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = tile_bytes + per_warp * nwarps;
  auto kern = rank_transform_kernel<WIDTH, VEC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  kern<<<(unsigned)L.slabs, nwarps * 32, smem, s>>>(dX, L.rows, L.cols, ld, exclude, fill, ranks,
                                                    L.slabs, N, nwarps);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rank_transform(const Layout& L, const float* dX, int64_t ld, int exclude,
                                  float fill, uint32_t* ranks, cudaStream_t s) {
  if (L.width == 8) return launch_rank_layout<8, 4>(L, dX, ld, exclude, fill, ranks, s);
  switch (L.vec) {
    case 4: return launch_rank_layout<16, 4>(L, dX, ld, exclude, fill, ranks, s);
    case 2: return launch_rank_layout<16, 2>(L, dX, ld, exclude, fill, ranks, s);
    case 1: return launch_rank_layout<16, 1>(L, dX, ld, exclude, fill, ranks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ebic
