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
// One CTA per slab of rows (VEC row groups). Rows of up to 64 columns: one thread per row sorts
// its (key, column) pairs with a compare-exchange network in registers and walks the sorted run.
// Wider rows: each warp takes one row at a time. Up to 256 columns the keys are sorted in
// registers and shuffles, and each column looks its key up in the sorted run; wider still,
// (key << 32 | column) pairs are sorted in the warp's shared buffer and walked. In the warp forms
// a warp prefix count of "first of a new key" flags over the sorted run gives the dense ranks. Ranks are written as bytes/halves into a shared slab tile
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

// The same transform for rows of at most 32*E columns with the sort in registers: lane l holds
// the row's sorted keys at positions l*E .. l*E+E-1 ("blocked" layout) after a bitonic network
// whose exchanges are register min/max when partners share a lane (distance < E) and shuffles
// otherwise. Only the 32-bit keys are sorted: the warp then writes the sorted keys and their
// dense ranks to its shared buffer, and every lane finds the rank of each of its own columns by a
// binary search of its key there. Each warp loads its next row while it ranks the current one.
template <int E>
__device__ __forceinline__ void bitonic_sort_keys(uint32_t (&x)[E], int lane) {
  constexpr int N = 32 * E;
#pragma unroll
  for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      if (jj < E) {  // partners in this lane: elements e and e | jj
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (e & jj) continue;
          const bool up = ((lane * E + e) & kk) == 0;
          const uint32_t a = x[e], b = x[e | jj];
          const uint32_t lo = min(a, b), hi = max(a, b);
          x[e] = up ? lo : hi;
          x[e | jj] = up ? hi : lo;
        }
      } else {  // partner in lane ^ (jj / E), same element
        const int d = jj / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = lane * E + e;
          const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x[e], d);
          // the lower index of an ascending pair keeps the smaller key, and so on
          const bool keep_min = ((i & jj) == 0) == ((i & kk) == 0);
          x[e] = keep_min ? min(x[e], y) : max(x[e], y);
        }
      }
    }
  }
}

template <int WIDTH, int VEC, int E>
__global__ void __launch_bounds__(512) rank_transform_reg_kernel(const float* __restrict__ X,
                                                                int64_t R, int C, int64_t ld,
                                                                int exclude, float fill,
                                                                uint32_t* __restrict__ out,
                                                                int64_t Q, int nwarps) {
  constexpr int RPG = WIDTH == 8 ? 128 : 64;  // rows per group
  constexpr int RPS = RPG * VEC;              // rows per slab
  constexpr int N = 32 * E;
  constexpr uint32_t MISSING = 0u;
  constexpr int TROW = 32 * VEC + 1;
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* tile = reinterpret_cast<uint32_t*>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the warp's sorted keys and their dense ranks
  uint32_t* skey = reinterpret_cast<uint32_t*>(
                       smem + (((size_t)C * TROW * 4 + 15) & ~(size_t)15)) + (size_t)warp * 2 * N;
  uint32_t* srank = skey + N;
  const int64_t q = blockIdx.x;
  // the row's values as loaded: element e of lane l is column e*32 + l (coalesced)
  auto load_row = [&](int rho, float (&v)[E]) {
    const int64_t r = q * RPS + rho;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = e * 32 + lane;
      v[e] = (rho < RPS && r < R && c < C) ? __ldg(X + r * ld + c) : 0.0f;
    }
  };
  float cur[E];
  load_row(warp, cur);
  for (int rho = warp; rho < RPS; rho += nwarps) {
    const int64_t r = q * RPS + rho;
    float nxt[E];
    load_row(rho + nwarps, nxt);  // the warp's next row, while this one is ranked
    const int j = rho / RPG, rr = rho % RPG, l = rr & 31, k = rr >> 5;
    uint8_t* cell0 = reinterpret_cast<uint8_t*>(tile) + ((size_t)l * VEC + j) * 4 +
                     (WIDTH == 8 ? k : 2 * k);
    if (r >= R) {  // padding rows hold the missing code in every column
      for (int c = lane; c < C; c += 32) {
        uint8_t* cell = cell0 + (size_t)c * TROW * 4;
        if (WIDTH == 8) *cell = (uint8_t)MISSING;
        else *reinterpret_cast<uint16_t*>(cell) = (uint16_t)MISSING;
      }
    } else {
      uint32_t v[E], x[E];  // keys of the lane's columns; the same, to be sorted
#pragma unroll
      for (int e = 0; e < E; ++e) {
        v[e] = e * 32 + lane < C ? order_key(cur[e], exclude, fill) : kMissingKey;
        x[e] = v[e];
      }
      bitonic_sort_keys<E>(x, lane);
      // dense rank of each sorted position: distinct keys up to and including it (the missing
      // key, which also pads the row, sorts last and is never counted)
      const uint32_t prev_last = __shfl_up_sync(0xFFFFFFFFu, x[E - 1], 1);
      uint32_t fresh = 0, cnt = 0;  // fresh: bit e = position lane*E+e starts a new key
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const uint32_t before = e > 0 ? x[e - 1] : prev_last;
        const bool f = x[e] != kMissingKey && ((lane == 0 && e == 0) || before != x[e]);
        fresh |= (uint32_t)f << e;
        cnt += f;
      }
      uint32_t incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
      }
      uint32_t run = incl - cnt;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        run += (fresh >> e) & 1u;
        skey[lane * E + e] = x[e];
        srank[lane * E + e] = run;
      }
      __syncwarp();
      // each column's rank: the first sorted position holding its key (lower bound)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int c = e * 32 + lane;
        if (c >= C) continue;
        uint32_t rank = MISSING;
        if (v[e] != kMissingKey) {
          int pos = 0;
#pragma unroll
          for (int step = N / 2; step >= 1; step >>= 1)
            if (skey[pos + step - 1] < v[e]) pos += step;
          rank = srank[pos];  // 1-based dense rank
        }
        uint8_t* cell = cell0 + (size_t)c * TROW * 4;
        if (WIDTH == 8) *cell = (uint8_t)rank;
        else *reinterpret_cast<uint16_t*>(cell) = (uint16_t)rank;
      }
      __syncwarp();  // the buffer is rewritten for the next row
    }
#pragma unroll
    for (int e = 0; e < E; ++e) cur[e] = nxt[e];
  }
  __syncthreads();
  // copy out: column c of slab q is 32*VEC contiguous words in HBM
  const int wpc = 32 * VEC;
  for (int64_t idx = threadIdx.x; idx < (int64_t)C * wpc; idx += blockDim.x) {
    const int64_t c = idx / wpc, i = idx % wpc;
    out[(c * Q + q) * wpc + i] = tile[c * TROW + i];
  }
}

// Rows of at most 64 columns (8-bit codes): one thread per row. A compare-exchange network
// sorts the thread's (key, column) pairs in registers: Batcher's odd-even merge sort (Batcher,
// "Sorting networks and their applications", AFIPS 1968), 543 exchanges for 64 keys, 191 for 32,
// each a compare, a min, a max and two selects, every index fixed at compile time so that the
// arrays stay in registers. A walk over the sorted run then counts distinct keys and drops each
// column's dense rank into the slab tile. Each chunk of 128 rows is staged in shared memory by
// 4-byte cp.async copies (row stride N + 1 words, so that thread t reading its column c hits bank
// (t + c) mod 32), the next chunk's copies in flight while the current one is sorted.
__device__ __forceinline__ void compare_exchange(uint32_t& ka, uint32_t& kb, uint32_t& ca,
                                                 uint32_t& cb) {
  const bool swap = ka > kb;
  const uint32_t lo = min(ka, kb), hi = max(ka, kb);
  const uint32_t c0 = swap ? cb : ca, c1 = swap ? ca : cb;
  ka = lo;
  kb = hi;
  ca = c0;
  cb = c1;
}

// Batcher's merge of the elements at LO, LO+R, LO+2R, ... below LO+NN, whose two halves are each
// sorted: merge the even and the odd subsequences (stride 2R), then exchange the neighbours
// (i, i+R) for i = LO+R, LO+3R, ...
template <int LO, int NN, int R, int N>
struct OddEvenMerge {
  static __device__ __forceinline__ void run(uint32_t (&k)[N], uint32_t (&c)[N]) {
    if constexpr (2 * R < NN) {
      OddEvenMerge<LO, NN, 2 * R, N>::run(k, c);
      OddEvenMerge<LO + R, NN, 2 * R, N>::run(k, c);
#pragma unroll
      for (int i = LO + R; i + R < LO + NN; i += 2 * R) compare_exchange(k[i], k[i + R], c[i], c[i + R]);
    } else {
      compare_exchange(k[LO], k[LO + R], c[LO], c[LO + R]);
    }
  }
};

template <int LO, int NN, int N>
struct OddEvenSort {
  static __device__ __forceinline__ void run(uint32_t (&k)[N], uint32_t (&c)[N]) {
    if constexpr (NN > 1) {
      OddEvenSort<LO, NN / 2, N>::run(k, c);
      OddEvenSort<LO + NN / 2, NN / 2, N>::run(k, c);
      OddEvenMerge<LO, NN, 1, N>::run(k, c);
    }
  }
};

template <int N>
__device__ __forceinline__ void oddeven_merge_sort(uint32_t (&k)[N], uint32_t (&c)[N]) {
  OddEvenSort<0, N, N>::run(k, c);
}

__device__ __forceinline__ void cp_async4(uint32_t* dst, const float* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

constexpr int kRowThreads = 128;  // rows per chunk, one per thread

template <int N>
__global__ void __launch_bounds__(kRowThreads, 3) rank_transform_row_kernel(
    const float* __restrict__ X, int64_t R, int C, int64_t ld, int exclude, float fill,
    uint32_t* __restrict__ out, int64_t Q) {
  constexpr int VEC = 4, RPG = 128, RPS = RPG * VEC;  // 8-bit codes: 512 rows per slab
  constexpr int TROW = 32 * VEC + 1;
  constexpr int SROW = N + 1;
  constexpr int T = kRowThreads;
  constexpr uint32_t MISSING = 0u;
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* tile = reinterpret_cast<uint32_t*>(smem);
  uint32_t* stage =
      reinterpret_cast<uint32_t*>(smem + (((size_t)C * TROW * 4 + 15) & ~(size_t)15));
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t q = blockIdx.x;
  const int64_t r_base = q * RPS;
  // chunk copies: warp w stages rows w, w+4, ..., columns lane, lane+32 (coalesced per row)
  auto stage_chunk = [&](int cb) {
    for (int rr = warp; rr < T; rr += T / 32) {
      const int64_t r = r_base + cb + rr;
      if (r >= R) break;
      const float* row = X + r * ld;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 32)
        if (c0 + lane < C) cp_async4(stage + rr * SROW + c0 + lane, row + c0 + lane);
    }
    cp_async_commit();
  };
  stage_chunk(0);
  for (int cb = 0; cb < RPS; cb += T) {
    const int rho = cb + t;
    const int64_t r = r_base + rho;
    cp_async_wait_all();
    __syncthreads();
    uint32_t key[N], col[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      key[c] = (c < C && r < R) ? order_key(__uint_as_float(stage[t * SROW + c]), exclude, fill)
                                : kMissingKey;
      col[c] = c;
    }
    __syncthreads();  // the stage is free: the next chunk's copies overlap this one's sort
    if (cb + T < RPS) stage_chunk(cb + T);
    const int j = rho / RPG, rr = rho % RPG, l = rr & 31, k = rr >> 5;
    uint8_t* cell0 = reinterpret_cast<uint8_t*>(tile) + ((size_t)l * VEC + j) * 4 + k;
    if (r >= R) {  // padding rows hold the missing code in every column
      for (int c = 0; c < C; ++c) cell0[(size_t)c * TROW * 4] = (uint8_t)MISSING;
      continue;
    }
    oddeven_merge_sort<N>(key, col);
    uint32_t run = 0;  // distinct non-missing keys so far: the 1-based dense rank
#pragma unroll
    for (int p = 0; p < N; ++p) {
      run += key[p] != kMissingKey && (p == 0 || key[p] != key[p - 1]);
      if (col[p] < (uint32_t)C)
        cell0[(size_t)col[p] * TROW * 4] = (uint8_t)(key[p] == kMissingKey ? MISSING : run);
    }
  }
  __syncthreads();
  // copy out: column c of slab q is 32*VEC contiguous words in HBM
  constexpr int wpc = 32 * VEC;
  for (int idx = t; idx < C * wpc; idx += T) {
    const int c = idx / wpc, i = idx % wpc;
    out[((int64_t)c * Q + q) * wpc + i] = tile[c * TROW + i];
  }
}

template <int N>
cudaError_t launch_rank_row(const Layout& L, const float* dX, int64_t ld, int exclude, float fill,
                            uint32_t* ranks, cudaStream_t s) {
  const size_t tile = (((size_t)L.cols * (32 * 4 + 1) * 4) + 15) & ~(size_t)15;
  const size_t smem = tile + (size_t)kRowThreads * (N + 1) * 4;
  auto kern = rank_transform_row_kernel<N>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  kern<<<(unsigned)L.slabs, kRowThreads, smem, s>>>(dX, L.rows, L.cols, ld, exclude, fill, ranks,
                                                    L.slabs);
  return cudaGetLastError();
}

template <int WIDTH, int VEC, int E>
cudaError_t launch_rank_reg(const Layout& L, const float* dX, int64_t ld, int exclude, float fill,
                            uint32_t* ranks, cudaStream_t s) {
  const size_t tile = (((size_t)L.cols * (32 * VEC + 1) * 4) + 15) & ~(size_t)15;
  const size_t per_warp = (size_t)2 * 32 * E * 4;  // sorted keys and their ranks
  int nwarps = (int)((kSmemDynMax - tile) / per_warp);
  if (nwarps > 16) nwarps = 16;
  if (nwarps < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = tile + per_warp * nwarps;
  auto kern = rank_transform_reg_kernel<WIDTH, VEC, E>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  kern<<<(unsigned)L.slabs, nwarps * 32, smem, s>>>(dX, L.rows, L.cols, ld, exclude, fill, ranks,
                                                    L.slabs, nwarps);
  return cudaGetLastError();
}

template <int WIDTH, int VEC>
cudaError_t launch_rank_layout(const Layout& L, const float* dX, int64_t ld, int exclude,
                               float fill, uint32_t* ranks, cudaStream_t s) {
  if (WIDTH == 8 && VEC == 4) {
    if (L.cols <= 32) return launch_rank_row<32>(L, dX, ld, exclude, fill, ranks, s);
    if (L.cols <= 64) return launch_rank_row<64>(L, dX, ld, exclude, fill, ranks, s);
  }
  if (L.cols <= 32) return launch_rank_reg<WIDTH, VEC, 1>(L, dX, ld, exclude, fill, ranks, s);
  if (L.cols <= 64) return launch_rank_reg<WIDTH, VEC, 2>(L, dX, ld, exclude, fill, ranks, s);
  if (L.cols <= 128) return launch_rank_reg<WIDTH, VEC, 4>(L, dX, ld, exclude, fill, ranks, s);
  if (L.cols <= 256) return launch_rank_reg<WIDTH, VEC, 8>(L, dX, ld, exclude, fill, ranks, s);
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
