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
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "device_common.cuh"
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

// Rows of at most 64 columns (8-bit codes): one thread per row sorts single words, each value's
// order key with its low B bits (B = log2 N: 6 for 64 columns, 5 for 32) replaced by its column,
// so that a compare-exchange is one min and one max and the sorted words still carry their
// columns. The network is Batcher's odd-even merge sort (Batcher, "Sorting networks and their
// applications", AFIPS 1968): 543 exchanges for 64 keys, 191 for 32, every index fixed at
// compile time so that the words stay in registers. Words whose top 32 - B bits differ are in
// the values' order, so the walk over the sorted words gives each column its code, the number of
// distinct top-bit values up to its word. Two adjacent words with the same top bits hold one
// value twice (a tie: one code, as the walk gives) or two values within 2^B key units, whose
// order the sort did not see. A lane whose walk met such a pair hands its sorted words to its
// warp, which recounts that row from the full keys: lane l takes sorted positions l and 32 + l,
// a ballot marks each key's first position within its group of equal top bits, and a position's
// code is 1 + the first positions of lower groups (a popcount) + the distinct keys of its own
// group below its key (a walk over the group, a few words long). About 1.2 % of the rows of a
// methylation-shaped matrix (beta values) are recounted, at about a hundred warp instructions
// each.
//
// Keys: adding +0.0 (round to nearest, subnormals kept) folds -0 onto +0 and turns every NaN into
// the canonical NaN 0x7FFFFFFF, whose key 0xFFFFFFFF is the missing key (exclusion on; with
// exclusion off it is replaced by the fill value). A negative value's key is its bits inverted,
// a positive value's its bits with the top bit set. Missing values sort last; the walk counts
// them as one more value, and their columns, known from a bit mask, get code 0 afterwards.
//
// Work: each CTA ranks whole slabs of 512 rows, 16 batches of 32 rows (batch b: rows
// 128 (b / 4) + 32 (b % 4) + lane), and drops the codes as bytes into a shared slab tile laid out
// [column][chunk][lane], so that lane l always writes bank l, whatever the column; columns C..N-1
// take the padding words. The tile is copied out with 16-byte stores into the HBM layout (word
// 4 l + chunk of a column's 128 words of the slab); two tiles, one barrier per slab. Rows of at
// least 32 columns on 16-byte boundaries (a multiple of four columns) take the TMA form: one CTA
// of 16 warps per SM, each warp's next batch brought into shared memory by TMA while the current
// one is sorted. Other rows are loaded by each lane straight into registers (8 warps, two CTAs
// per SM).
__device__ __forceinline__ void compare_exchange(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b);
  b = max(a, b);
  a = lo;
}

// Batcher's merge of the elements at LO, LO+R, LO+2R, ... below LO+NN, whose two halves are each
// sorted: merge the even and the odd subsequences (stride 2R), then exchange the neighbours
// (i, i+R) for i = LO+R, LO+3R, ...
template <int LO, int NN, int R, int N>
struct OddEvenMerge {
  static __device__ __forceinline__ void run(uint32_t (&k)[N]) {
    if constexpr (2 * R < NN) {
      OddEvenMerge<LO, NN, 2 * R, N>::run(k);
      OddEvenMerge<LO + R, NN, 2 * R, N>::run(k);
#pragma unroll
      for (int i = LO + R; i + R < LO + NN; i += 2 * R) compare_exchange(k[i], k[i + R]);
    } else {
      compare_exchange(k[LO], k[LO + R]);
    }
  }
};

template <int LO, int NN, int N>
struct OddEvenSort {
  static __device__ __forceinline__ void run(uint32_t (&k)[N]) {
    if constexpr (NN > 1) {
      OddEvenSort<LO, NN / 2, N>::run(k);
      OddEvenSort<LO + NN / 2, NN / 2, N>::run(k);
      OddEvenMerge<LO, NN, 1, N>::run(k);
    }
  }
};

constexpr int kRankThreads = 256;   // 8 warps a CTA, two CTAs an SM (rows in any alignment)
constexpr int kRankBlocksPerSM = 2;
constexpr int kStagedThreads = 512;  // 16 warps, one CTA an SM (16-byte aligned rows)
constexpr int kStagedWarps = kStagedThreads / 32;
constexpr int kRankSlabRows = 512;  // the 8-bit layout's slab: 4 chunks of 128 rows

// A value's bits as its key sees them: -0 folded onto +0 and every NaN made 0x7FFFFFFF (the sum
// with +0.0 in round-to-nearest without flushing subnormals), then a NaN replaced by the fill
// value when exclusion is off. `nan` says whether the value was a NaN.
template <bool EXCL>
__device__ __forceinline__ uint32_t value_bits(float x, uint32_t fill_bits, bool& nan) {
  float y;
  asm("add.rn.f32 %0, %1, 0f00000000;" : "=f"(y) : "f"(x));
  const uint32_t b = __float_as_uint(y);
  nan = b == 0x7FFFFFFFu;
  return !EXCL && nan ? fill_bits : b;
}

template <bool EXCL>
__device__ __forceinline__ uint32_t full_key(float x, uint32_t fill_bits) {
  bool nan;
  const uint32_t b = value_bits<EXCL>(x, fill_bits, nan);
  return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
}

// A value's packed word: (key & ~CM) | c, key = bits ^ (sign ? 0xFFFFFFFF : 0x80000000), with the
// sign taken by the multiply pipe (the high word of 2 * bits); a missing value sets its column's
// bit in `missing`.
template <int N, bool EXCL>
__device__ __forceinline__ uint32_t packed_word(float x, int c, uint32_t fill_bits,
                                                uint64_t& missing) {
  constexpr uint32_t CM = N == 64 ? 63u : 31u;
  bool nan;
  const uint32_t bits = value_bits<EXCL>(x, fill_bits, nan);
  if (EXCL && nan) missing |= 1ull << c;
  const uint32_t sign = __umulhi(bits, 2u);
  return (bits & ~CM) ^ (sign * (0x7FFFFFFFu & ~CM)) ^ (0x80000000u | (uint32_t)c);
}

// One lane's row, its packed words v in registers (columns C..N-1 and a padding row's columns as
// missing words): sort, walk, the warp's recount of rows whose words repeat top bits, and code 0
// for missing columns. `cell` is the lane's byte of the slab tile (+ 512 per column); `sw`, `sk`
// the warp's two N-word buffers; `srow0` the warp's first row.
template <int N, bool EXCL>
__device__ __forceinline__ void rank_lane_row(uint32_t (&v)[N], uint64_t missing, int C,
                                              const float* __restrict__ srow0, int64_t ld,
                                              uint32_t fill_bits, uint8_t* cell0, int lane,
                                              uint32_t* sw, uint32_t* sk) {
  constexpr int B = N == 64 ? 6 : 5;  // column bits of a word
  constexpr uint32_t CM = (1u << B) - 1u;
  constexpr uint32_t kTopMissing = kMissingKey >> B;
  uint8_t* cell = cell0 + lane * 4;
  OddEvenSort<0, N, N>::run(v);
  // the walk: code = distinct top-bit values up to this word
  uint32_t run = 1;
  cell[(v[0] & CM) * 512] = 1u;
#pragma unroll
  for (int p = 1; p < N; ++p) {
    run += (v[p] ^ v[p - 1]) > CM;
    cell[(v[p] & CM) * 512] = (uint8_t)run;
  }
  // words that repeated their predecessor's top bits: the missing and padding words after the
  // first of them, and any pair of values within 2^B key units
  const int n_last = (N - C) + __popcll(missing);
  const int repeats = N - (int)run - (n_last > 1 ? n_last - 1 : 0);
  // rare: a lane whose row repeated top bits hands its sorted words to the warp, which
  // recounts that row from the full keys (a group of words with the same top bits may hold ties
  // and values the sort could not order)
  uint32_t need = __ballot_sync(0xFFFFFFFFu, repeats > 0);
  while (need) {
    const int src = __ffs(need) - 1;
    need &= need - 1u;
    if (lane == src) {
#pragma unroll
      for (int p = 0; p < N; ++p) sw[p] = v[p];
    }
    __syncwarp();
    const float* srow = srow0 + src * ld;
    uint32_t wp[N / 32], kp[N / 32];
#pragma unroll
    for (int h = 0; h < N / 32; ++h) {
      wp[h] = sw[lane + 32 * h];
      kp[h] = (wp[h] >> B) == kTopMissing
                  ? kMissingKey
                  : full_key<EXCL>(__ldg(srow + (wp[h] & CM)), fill_bits);
      sk[lane + 32 * h] = kp[h];
    }
    __syncwarp();
    // each position's group (same top bits) start, and whether its key first occurs there
    int g0[N / 32];
    uint64_t first = 0;
#pragma unroll
    for (int h = 0; h < N / 32; ++h) {
      const int p = lane + 32 * h;
      int g = p;
      while (g > 0 && (sw[g - 1] ^ wp[h]) <= CM) --g;
      bool f = kp[h] != kMissingKey;
      for (int i = g; i < p && f; ++i) f = sk[i] != kp[h];
      g0[h] = g;
      first |= (uint64_t)__ballot_sync(0xFFFFFFFFu, f) << (32 * h);
    }
    uint8_t* scell = cell0 + src * 4;
#pragma unroll
    for (int h = 0; h < N / 32; ++h) {
      // 1 + distinct keys in lower groups + distinct keys of its group below its own
      uint32_t code = 1u + (uint32_t)__popcll(first & ((1ull << g0[h]) - 1ull));
      for (int i = g0[h]; i < N && (sw[i] ^ wp[h]) <= CM; ++i)
        code += ((first >> i) & 1ull) && sk[i] < kp[h];
      scell[(wp[h] & CM) * 512] = (uint8_t)(kp[h] == kMissingKey ? 0u : code);
    }
    __syncwarp();  // the buffers are rewritten for the next lane
  }
  while (missing) {
    const int c = __ffsll((long long)missing) - 1;
    missing &= missing - 1ull;
    cell[c * 512] = 0u;
  }
}

// A lane's words for a padding row (exclusion off; with exclusion on its NaN values are missing
// already): every column missing.
template <int N>
__device__ __forceinline__ void padding_words(uint32_t (&v)[N], uint64_t& missing, int C) {
  constexpr uint32_t CM = N == 64 ? 63u : 31u;
#pragma unroll
  for (int c = 0; c < N; ++c) v[c] = ~CM | (uint32_t)c;
  missing = C >= 64 ? ~0ull : ((1ull << C) - 1ull);
}

// Column c of slab q is 128 contiguous words; word 4 l + j is tile word 32 j + l.
__device__ __forceinline__ void copy_out_tile(const uint32_t* tile, uint32_t* __restrict__ out,
                                              int C, int64_t Q, int64_t q, int tid, int nthreads) {
  for (int i = tid; i < C * 32; i += nthreads) {
    const int c = i >> 5, l = i & 31;
    const uint32_t* t = tile + c * 128 + l;
    const uint4 w = make_uint4(t[0], t[32], t[64], t[96]);
    *reinterpret_cast<uint4*>(out + ((int64_t)c * Q + q) * 128 + 4 * l) = w;
  }
}

// Rows in any alignment: each lane loads its row with 4-byte loads straight into registers; warp
// w takes the slab's batches w and w + 8.
template <int N, bool EXCL>
__global__ void __launch_bounds__(kRankThreads, kRankBlocksPerSM) rank_rows_packed_kernel(
    const float* __restrict__ X, int64_t R, int C, int64_t ld, uint32_t fill_bits,
    uint32_t* __restrict__ out, int64_t Q) {
  constexpr int kWarps = kRankThreads / 32;
  constexpr int tile_words = N * 128;
  constexpr uint32_t CM = N == 64 ? 63u : 31u;
  static_assert(N == 32 || N == 64, "packed words carry a 5- or 6-bit column");
  extern __shared__ __align__(16) uint32_t tiles[];  // two tiles of [N][4 chunks][32 lanes] words
  __shared__ uint32_t sorted_w[kWarps][N];  // one lane's sorted words, for its warp
  __shared__ uint32_t sorted_k[kWarps][N];  // the full keys of those words' values
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int buf = 0;
  for (int64_t q = blockIdx.x; q < Q; q += gridDim.x, buf ^= 1) {
    uint32_t* tile = tiles + buf * tile_words;
    for (int b = warp; b < kRankSlabRows / 32; b += kWarps) {
      const int j = b >> 2, k = b & 3;  // chunk, and the byte of the word
      const int64_t r0 = q * kRankSlabRows + j * 128 + k * 32;
      const bool live = r0 + lane < R;  // a padding row is ranked as a row of missing values
      const float* row = X + (live ? r0 + lane : 0) * ld;
      uint32_t v[N];
      uint64_t missing = 0;
#pragma unroll
      for (int c = 0; c < N; ++c)
        v[c] = c < C ? packed_word<N, EXCL>(live ? __ldg(row + c) : NAN, c, fill_bits, missing)
                     : (~CM | (uint32_t)c);
      if (!EXCL && !live) padding_words<N>(v, missing, C);
      rank_lane_row<N, EXCL>(v, missing, C, X + r0 * ld, ld, fill_bits,
                             reinterpret_cast<uint8_t*>(tile + j * 32) + k, lane, sorted_w[warp],
                             sorted_k[warp]);
    }
    __syncthreads();
    copy_out_tile(tile, out, C, Q, q, threadIdx.x, kRankThreads);
  }
}

// Rows of at least 32 columns on 16-byte boundaries, a multiple of four columns: one CTA of 16
// warps per SM, warp w always taking batch w of its slabs. The warp's next batch (32 rows) is
// brought into its stage by TMA while the current one is sorted: one lane issues a 32 x 32-float
// box per 32 columns (128-byte swizzle: 16-byte chunk c of row rr at chunk c ^ (rr % 8) of the
// row's 128 bytes, so the eight lanes of a 16-byte read phase hit distinct banks), completion on
// the warp's mbarrier. With the loads off the critical path (and no per-lane copies to issue) the
// integer pipe is the bound. Every wait is bounded; a wait that expires records kErrTimeout in
// *status, and the warp stops staging (its later rows are ranked from whatever the stage holds,
// and the load that reads *status fails).
template <int N, bool EXCL>
__global__ void __launch_bounds__(kStagedThreads, 1) rank_rows_tma_kernel(
    const __grid_constant__ CUtensorMap xmap, const float* __restrict__ X, int64_t R, int C,
    int64_t ld, uint32_t fill_bits, uint32_t* __restrict__ out, int64_t Q,
    uint32_t* __restrict__ status, uint64_t timeout_ns) {
  constexpr int NB = N / 32;                       // 32-column boxes per row
  constexpr uint32_t kBoxBytes = 32u * 128u;        // 32 rows of 128 bytes
  constexpr uint32_t kStageBytes = NB * kBoxBytes;
  constexpr int tile_words = N * 128;
  constexpr uint32_t CM = N == 64 ? 63u : 31u;
  static_assert(N == 32 || N == 64, "packed words carry a 5- or 6-bit column");
  extern __shared__ __align__(1024) uint8_t sraw[];  // stages (1024-byte aligned), then two tiles
  __shared__ uint64_t bars[kStagedWarps];
  __shared__ uint32_t sorted_w[kStagedWarps][N];
  __shared__ uint32_t sorted_k[kStagedWarps][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = warp >> 2, k = warp & 3;  // the warp's chunk and byte in every slab
  uint8_t* sbase = sraw + ((1024u - (dev::smem_addr(sraw) & 1023u)) & 1023u);
  uint8_t* stage = sbase + warp * kStageBytes;
  uint32_t* tiles = reinterpret_cast<uint32_t*>(sbase + kStagedWarps * kStageBytes);
  uint64_t* bar = &bars[warp];
  if (lane == 0) {
    dev::mbar_init(bar, 1);
    dev::fence_barrier_init();
  }
  __syncwarp();
  auto issue = [&](int64_t q) {  // lane 0: the warp's batch of slab q
    const int32_t y = (int32_t)(q * kRankSlabRows + j * 128 + k * 32);
    dev::mbar_arrive_expect_tx(bar, kStageBytes);
#pragma unroll
    for (int bx = 0; bx < NB; ++bx) dev::tma_load_2d(stage + bx * kBoxBytes, &xmap, bar, bx * 32, y);
  };
  // a batch whose rows are all padding is not staged (its rows are never read)
  auto staged = [&](int64_t q) { return q * kRankSlabRows + j * 128 + k * 32 < R; };
  int64_t q = blockIdx.x;
  uint32_t parity = 0;
  bool pending = false, bad = false;  // a copy is in flight; a wait of this warp expired
  if (q < Q && staged(q)) {
    if (lane == 0) issue(q);
    pending = true;
  }
  int buf = 0;
  for (; q < Q; q += gridDim.x, buf ^= 1) {
    uint32_t* tile = tiles + buf * tile_words;
    const int64_t r0 = q * kRankSlabRows + j * 128 + k * 32;
    const bool live = r0 + lane < R;
    if (pending && !bad) {
      if (dev::mbar_wait_bounded(bar, parity, timeout_ns)) {
        parity ^= 1u;
        pending = false;
      } else {
        bad = true;
      }
    }
    uint32_t v[N];
    uint64_t missing = 0;
    const uint8_t* srow = stage + lane * 128;
#pragma unroll
    for (int c4 = 0; c4 < N / 4; ++c4) {
      if (4 * c4 < C) {
        const float4 f =
            live ? *reinterpret_cast<const float4*>(srow + (c4 >> 3) * kBoxBytes +
                                                    (((c4 & 7) ^ (lane & 7)) << 4))
                 : make_float4(NAN, NAN, NAN, NAN);
        v[4 * c4] = packed_word<N, EXCL>(f.x, 4 * c4, fill_bits, missing);
        v[4 * c4 + 1] = packed_word<N, EXCL>(f.y, 4 * c4 + 1, fill_bits, missing);
        v[4 * c4 + 2] = packed_word<N, EXCL>(f.z, 4 * c4 + 2, fill_bits, missing);
        v[4 * c4 + 3] = packed_word<N, EXCL>(f.w, 4 * c4 + 3, fill_bits, missing);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[4 * c4 + e] = ~CM | (uint32_t)(4 * c4 + e);
      }
    }
    if (!EXCL && !live) padding_words<N>(v, missing, C);
    __syncwarp();  // every lane has read its row: the stage takes the next batch
    if (!bad && q + gridDim.x < Q && staged(q + gridDim.x)) {
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads before the copy
        issue(q + gridDim.x);
      }
      pending = true;
    }
    rank_lane_row<N, EXCL>(v, missing, C, X + r0 * ld, ld, fill_bits,
                           reinterpret_cast<uint8_t*>(tile + j * 32) + k, lane, sorted_w[warp],
                           sorted_k[warp]);
    __syncthreads();
    copy_out_tile(tile, out, C, Q, q, threadIdx.x, kStagedThreads);
  }
  if (pending) (void)dev::mbar_wait_bounded(bar, parity, timeout_ns);  // none outlives the CTA
  if (bad && lane == 0) atomicOr(status, kErrTimeout);
}

uint32_t fill_bits_host(float fill) {
  uint32_t b;
  std::memcpy(&b, &fill, 4);
  return b == 0x80000000u ? 0u : b;  // -0 -> +0 (fill is never NaN)
}


// A tensor map over the float matrix for the TMA form: dims {C, R}, row stride ld floats, boxes of
// 32 x 32 floats with the 128-byte swizzle. False when the driver cannot make one.
bool encode_matrix_map(CUtensorMap* map, const float* dX, int64_t R, int C, int64_t ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      (void)cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)R};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4ull};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(dX), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N, bool EXCL>
cudaError_t launch_rank_packed_as(const Layout& L, const float* dX, int64_t ld, float fill,
                                  uint32_t* ranks, uint32_t* status, int num_sms,
                                  cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  const uint32_t fb = fill_bits_host(fill);
  CUtensorMap map;
  const bool tma = L.cols >= 32 && L.rows >= 32 && ld % 4 == 0 && L.cols % 4 == 0 &&
                   (reinterpret_cast<uintptr_t>(dX) & 15u) == 0 &&
                   encode_matrix_map(&map, dX, L.rows, L.cols, ld);
  if (tma) {
    constexpr size_t smem = 1024 + (size_t)kStagedWarps * (N / 32) * 32 * 128 + (size_t)2 * N * 128 * 4;
    auto kern = rank_rows_tma_kernel<N, EXCL>;
    static std::atomic<uint64_t> ready{0};  // a bit per device: the attribute is set
    if (!((ready.load() >> dev) & 1u)) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      ready.fetch_or(1ull << dev);
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(L.slabs, num_sms));
    count_launch();
    kern<<<grid, kStagedThreads, smem, s>>>(map, dX, L.rows, L.cols, ld, fb, ranks, L.slabs,
                                            status, 1000000000ull);
    return cudaGetLastError();
  }
  constexpr size_t smem = (size_t)2 * N * 128 * 4;
  auto kern = rank_rows_packed_kernel<N, EXCL>;
  static std::atomic<uint64_t> ready{0};
  if (!((ready.load() >> dev) & 1u)) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ready.fetch_or(1ull << dev);
  }
  const int grid =
      (int)std::max<int64_t>(1, std::min<int64_t>(L.slabs, kRankBlocksPerSM * (int64_t)num_sms));
  count_launch();
  kern<<<grid, kRankThreads, smem, s>>>(dX, L.rows, L.cols, ld, fb, ranks, L.slabs);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_rank_packed(const Layout& L, const float* dX, int64_t ld, int exclude,
                               float fill, uint32_t* ranks, uint32_t* status, int num_sms,
                               cudaStream_t s) {
  return exclude ? launch_rank_packed_as<N, true>(L, dX, ld, fill, ranks, status, num_sms, s)
                 : launch_rank_packed_as<N, false>(L, dX, ld, fill, ranks, status, num_sms, s);
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
                               float fill, uint32_t* ranks, uint32_t* status, int num_sms,
                               cudaStream_t s) {
  if (WIDTH == 8 && VEC == 4) {
    if (L.cols <= 32)
      return launch_rank_packed<32>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
    if (L.cols <= 64)
      return launch_rank_packed<64>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
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
                                  float fill, uint32_t* ranks, uint32_t* status, int num_sms,
                                  cudaStream_t s) {
  if (L.width == 8)
    return launch_rank_layout<8, 4>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
  switch (L.vec) {
    case 4: return launch_rank_layout<16, 4>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
    case 2: return launch_rank_layout<16, 2>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
    case 1: return launch_rank_layout<16, 1>(L, dX, ld, exclude, fill, ranks, status, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ebic
