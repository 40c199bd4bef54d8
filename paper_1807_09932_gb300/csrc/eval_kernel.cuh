// Population evaluator: scores every candidate of a population against every row.
//
// What it computes (arXiv 1807.09932, Methods, "Handling missing values"): a row follows a
// candidate (c_1..c_L) when its values satisfy the "greater or equal" relation along the
// candidate's column order; a row with a missing value in one of those columns no longer counts
// when exclusion is on; with the negative-trend option a non-increasing row also follows. The
// output is each candidate's matched-row count and, optionally, its row bitmap.
//
// How (GB300): the rank matrix (see ebic_internal.h for its layout) is streamed through shared
// memory in row tiles of TS slabs by a 2-stage TMA pipeline (one elected thread issues 3-D
// cp.async.bulk.tensor loads that complete on an mbarrier; every wait is bounded by the global
// timer). One CTA per SM is persistent over a contiguous range of work items (candidate chunk,
// row tile); the candidate chunk's column lists are staged in shared memory. Each warp takes one
// candidate at a time and checks all TS*VEC row groups of the tile:
//   * lane l loads one 32-bit word per group and column: 4 rows (8-bit ranks) or 2 rows
//     (16-bit ranks) of the column, as one 16-byte shared load for four groups (VEC = 4);
//   * packed-field compare without unpacking: every field is < 2^(WIDTH-1), so
//     (b | H) - a == b + H - a has no borrow between fields and its top field bit is set
//     exactly when b >= a (H = the top bit of every field). AND-ing these words along the
//     chain leaves the top bit of a field set iff that row is non-decreasing along the order;
//   * exclusion by code: a missing value has code 0, below every real rank (1..C). A
//     non-decreasing chain that contains a 0 starts with it, a non-increasing one ends with it,
//     so requiring first >= 1 (increasing) and last >= 1 (decreasing) removes exactly the rows
//     with a missing value among the candidate's columns; padded rows hold 0 and never match;
//   * bitmap words without ballots: each lane gathers the match bits of up to 8 (16) groups into
//     one word, and a 5-stage shuffle butterfly transposes the warp's 32x32 bit matrix, so that
//     every lane holds one LSB-first bitmap word; the words of a tile go to HBM as one coalesced
//     run per candidate; counts are __popc of those words, summed with a warp reduction and one
//     atomicAdd per candidate and tile.
#pragma once

#include <atomic>

#include "device_common.cuh"
#include "ebic_internal.h"

namespace ebic {

template <int WIDTH>
struct Swar;
template <>
struct Swar<8> {
  static constexpr uint32_t H = 0x80808080u;    // top bit of each 8-bit field
  static constexpr uint32_t LB = 0x7F7F7F7Fu;   // H - 1 per field: top bit of v + LB <=> v >= 1
  static constexpr int WPG = 4;                 // bitmap words per 128-row group
};
template <>
struct Swar<16> {
  static constexpr uint32_t H = 0x80008000u;
  static constexpr uint32_t LB = 0x7FFF7FFFu;
  static constexpr int WPG = 2;                 // bitmap words per 64-row group
};

template <int VEC>
__device__ __forceinline__ void load_vec(const uint8_t* p, uint32_t* out) {
  if constexpr (VEC == 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (VEC == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    out[0] = v.x; out[1] = v.y;
  } else {
    out[0] = *reinterpret_cast<const uint32_t*>(p);
  }
}

// The lane's TS*VEC words of one column of the staged tile.
template <int VEC, int TS>
__device__ __forceinline__ void load_col(const uint8_t* colbase, uint32_t (&v)[TS * VEC]) {
#pragma unroll
  for (int s = 0; s < TS; ++s) load_vec<VEC>(colbase + s * 128 * VEC, v + s * VEC);
}

// Trend accumulators of one candidate for the lane's rows of the tile: on return acc[g] holds,
// in the top bit of each field (and nowhere else), whether that row follows the candidate
// (increasing, or also decreasing when NEG).
// Codes: a missing value is 0 and real ranks are 1..C, so 0 is below every real rank. A
// non-decreasing chain that contains a 0 must start with it, and a non-increasing one must end
// with it; requiring first >= 1 (resp. last >= 1) excludes exactly the rows with a missing value
// among the candidate's columns. The increasing test starts from that bound (no extra step at
// the end), and the chain is walked four columns per iteration: a compare costs one 3-input add,
// and every two compares one 3-input AND.
template <int WIDTH, int VEC, int TS, bool NEG>
__device__ __forceinline__ void trend_masks(const uint8_t* lane_base, uint32_t col_stride,
                                            const uint16_t* ccols, int L,
                                            uint32_t (&acc)[TS * VEC]) {
  constexpr int GT = TS * VEC;
  constexpr uint32_t H = Swar<WIDTH>::H;
  constexpr uint32_t LB = Swar<WIDTH>::LB;
  uint32_t a[GT], accd[GT];
  load_col<VEC, TS>(lane_base + (uint32_t)ccols[0] * col_stride, a);
#pragma unroll
  for (int g = 0; g < GT; ++g) {
    acc[g] = a[g] + LB;  // first >= 1: no missing value at the head of an increasing chain
    if (NEG) accd[g] = 0xFFFFFFFFu;
  }
  int i = 1;
  // column indices are read one step ahead (the chunk buffer has slack past its last column,
  // so reading a few entries beyond a candidate stays inside it)
  uint32_t n0 = ccols[1], n1 = ccols[2];
  if constexpr (!NEG && GT <= 8) {
    uint32_t n2 = ccols[3], n3 = ccols[4];
#pragma unroll 1
    for (; i + 3 < L; i += 4) {
      uint32_t b[GT], c[GT], d[GT], e[GT];
      load_col<VEC, TS>(lane_base + n0 * col_stride, b);
      load_col<VEC, TS>(lane_base + n1 * col_stride, c);
      load_col<VEC, TS>(lane_base + n2 * col_stride, d);
      load_col<VEC, TS>(lane_base + n3 * col_stride, e);
      n0 = ccols[i + 4];
      n1 = ccols[i + 5];
      n2 = ccols[i + 6];
      n3 = ccols[i + 7];
#pragma unroll
      for (int g = 0; g < GT; ++g) {
        const uint32_t t = acc[g] & (b[g] + H - a[g]) & (c[g] + H - b[g]);
        acc[g] = t & (d[g] + H - c[g]) & (e[g] + H - d[g]);  // a <= b <= c <= d <= e
        a[g] = e[g];
      }
    }
  }
#pragma unroll 1
  for (; i + 1 < L; i += 2) {
    uint32_t b[GT], c[GT];
    load_col<VEC, TS>(lane_base + n0 * col_stride, b);
    load_col<VEC, TS>(lane_base + n1 * col_stride, c);
    n0 = ccols[i + 2];
    n1 = ccols[i + 3];
#pragma unroll
    for (int g = 0; g < GT; ++g) {
      acc[g] = acc[g] & (b[g] + H - a[g]) & (c[g] + H - b[g]);            // a <= b <= c
      if (NEG) accd[g] = accd[g] & (a[g] + H - b[g]) & (b[g] + H - c[g]);  // a >= b >= c
      a[g] = c[g];
    }
  }
  if (i < L) {
    uint32_t b[GT];
    load_col<VEC, TS>(lane_base + n0 * col_stride, b);
#pragma unroll
    for (int g = 0; g < GT; ++g) {
      acc[g] &= b[g] + H - a[g];
      if (NEG) accd[g] &= a[g] + H - b[g];
      a[g] = b[g];
    }
  }
#pragma unroll
  for (int g = 0; g < GT; ++g) {
    if (NEG) acc[g] |= accd[g] & (a[g] + LB);  // last >= 1 for the decreasing chain
    acc[g] &= H;
  }
}

// Gather the match bits of up to WIDTH groups into one word per lane: bit (k*WIDTH + gl) is the
// top bit of field k of acc[b*WIDTH + gl], i.e. row (group b*WIDTH+gl, sub-row k, this lane).
// acc holds only top-of-field bits, so shifting group gl's bits right by (WIDTH-1-gl) puts them
// at distinct positions; the shift is done as the high half of a multiply-add on the FMA pipe,
// which also accumulates (the bit sets are disjoint, so the sum is their union).
template <int WIDTH, int GT>
__device__ __forceinline__ uint32_t pack_block(const uint32_t (&acc)[GT], int b) {
  uint32_t x = 0;
#pragma unroll
  for (int gl = 0; gl < WIDTH; ++gl) {
    const int g = b * WIDTH + gl;
    if (g < GT) {
      if (gl == WIDTH - 1) {
        x |= acc[g];
      } else {
        const uint32_t mul = 1u << (32 - (WIDTH - 1 - gl));  // hi(acc * 2^(32-s)) = acc >> s
        asm("mad.hi.u32 %0, %1, %2, %0;" : "+r"(x) : "r"(acc[g]), "r"(mul));
      }
    }
  }
  return x;
}

// 32x32 bit transpose across the warp: afterwards bit i of lane j is what bit j of lane i was.
// Five butterfly stages; in stage s the off-diagonal s x s blocks of every 2s x 2s block swap.
// rot[t] / sel[t] are the lane's rotation amount and bit mask of stage t (transpose_consts).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, const uint32_t (&rot)[5],
                                                const uint32_t (&sel)[5]) {
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, 16 >> t);
    const uint32_t r = __funnelshift_l(y, y, rot[t]);  // rotate left
    x = (x & ~sel[t]) | (r & sel[t]);
  }
  return x;
}

__device__ __forceinline__ void transpose_consts(int lane, uint32_t (&rot)[5],
                                                 uint32_t (&sel)[5]) {
  // bits j with (j & s) != 0, for s = 16, 8, 4, 2, 1
  const uint32_t right[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int s = 16 >> t;
    const bool top = (lane & s) == 0;  // top lanes take the partner's left bits into the right
    rot[t] = top ? (uint32_t)s : (uint32_t)(32 - s);
    sel[t] = top ? right[t] : ~right[t];
  }
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t n, uint64_t v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if ((uint64_t)a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Threads per CTA: 32 warps when the variant's registers fit in 64 per thread (more warps hide
// the shared-memory load latency of the column chain), else 16.
template <int GT, bool NEG>
__host__ __device__ constexpr int eval_threads() { return GT * (NEG ? 3 : 2) <= 16 ? 1024 : 512; }

// Shared-memory plan (dynamic): [stage 0][stage 1][chunk columns][chunk offsets]
template <int WIDTH, int VEC, int TS, bool NEG, bool BITMAPS>
__global__ void __launch_bounds__(eval_threads<TS * VEC, NEG>(), 1)
    eval_population_kernel(const __grid_constant__ CUtensorMap tmap, const EvalArgs a) {
  constexpr int GT = TS * VEC;
  constexpr int THREADS = eval_threads<GT, NEG>();
  constexpr int WARPS = THREADS / 32;
  constexpr int WPT = GT * Swar<WIDTH>::WPG;  // bitmap words per tile
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full_bar[2];
  __shared__ uint32_t chunk_info[3];

  if (*reinterpret_cast<const volatile uint32_t*>(a.err) != 0) return;  // invalid input

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t trot[5], tsel[5];
  transpose_consts(lane, trot, tsel);
  const uint32_t total = a.cand_offsets[a.n_cand];
  const int64_t n_tiles = (a.slabs + TS - 1) / TS;
  const int64_t n_chunks = ((int64_t)total + a.chunk_cols - 1) / a.chunk_cols;
  const int64_t n_items = n_chunks * n_tiles;
  const int64_t i0 = n_items * blockIdx.x / gridDim.x;
  const int64_t i1 = n_items * (blockIdx.x + 1) / gridDim.x;
  if (i0 >= i1) return;

  uint8_t* const stage0 = smem;
  uint8_t* const stage1 = smem + a.stage_bytes;
  uint16_t* const ccols = reinterpret_cast<uint16_t*>(smem + 2 * (size_t)a.stage_bytes);
  uint16_t* const coffs = ccols + a.chunk_cols + kChunkSlack;
  const uint32_t col_stride = TS * 128 * VEC;  // bytes of one column in a stage

  auto issue = [&](int64_t item, int s) {
    const int64_t tile = item % n_tiles;
    uint8_t* dst = s ? stage1 : stage0;
    dev::mbar_arrive_expect_tx(&full_bar[s], a.stage_bytes);
    for (int b = 0; b < a.n_col_boxes; ++b)
      dev::tma_load_3d(dst + (size_t)b * a.col_box * col_stride, &tmap, &full_bar[s], 0,
                       (int32_t)(tile * TS), b * a.col_box);
  };

  if (tid == 0) {
    dev::prefetch_tensormap(&tmap);
    dev::mbar_init(&full_bar[0], 1);
    dev::mbar_init(&full_bar[1], 1);
    dev::fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    issue(i0, 0);
    if (i0 + 1 < i1) issue(i0 + 1, 1);
  }

  int64_t cur_chunk = -1;
  uint32_t lo = 0, nc = 0;
  int64_t it = i0;
  bool timed_out = false;
  for (; it < i1; ++it) {
    const int64_t k = it / n_tiles, tile = it % n_tiles;
    const int s = (int)((it - i0) & 1);
    const uint32_t parity = (uint32_t)(((it - i0) >> 1) & 1);
    if (k != cur_chunk) {
      // stage the column lists of the candidates whose first column lies in
      // [k*CC, (k+1)*CC): at most CC candidates and CC+63 columns
      __syncthreads();
      if (tid == 0) {
        const uint32_t l = lower_bound_u32(a.cand_offsets, a.n_cand, (uint64_t)k * a.chunk_cols);
        const uint32_t h =
            lower_bound_u32(a.cand_offsets, a.n_cand, (uint64_t)(k + 1) * a.chunk_cols);
        chunk_info[0] = l;
        chunk_info[1] = h;
        chunk_info[2] = a.cand_offsets[l];
      }
      __syncthreads();
      lo = chunk_info[0];
      const uint32_t hi = chunk_info[1], c0 = chunk_info[2];
      nc = hi - lo;
      const uint32_t span = a.cand_offsets[hi] - c0;
      for (uint32_t i = tid; i < span; i += THREADS) ccols[i] = a.cand_cols[c0 + i];
      for (uint32_t i = tid; i <= nc; i += THREADS)
        coffs[i] = (uint16_t)(a.cand_offsets[lo + i] - c0);
      __syncthreads();
      cur_chunk = k;
    }

    const bool ok = dev::mbar_wait_bounded(&full_bar[s], parity, a.timeout_ns);
    if (!__syncthreads_and(ok)) { timed_out = true; break; }

    const uint8_t* lane_base = (s ? stage1 : stage0) + lane * 4 * VEC;
    const int64_t word0 = tile * WPT;
    const int64_t g0 = tile * GT;
    for (uint32_t ci = warp; ci < nc; ci += WARPS) {
      const int o = coffs[ci];
      const int L = coffs[ci + 1] - o;
      uint32_t acc[GT];
      trend_masks<WIDTH, VEC, TS, NEG>(lane_base, col_stride, ccols + o, L, acc);
      const uint32_t cand = lo + ci;
      uint32_t cnt = 0;
      if constexpr (BITMAPS) {
        // lane j of transpose block b ends up with bitmap word (b*WIDTH + j%WIDTH)*WPG + j/WIDTH
        uint32_t* out = a.bitmaps + (size_t)cand * (size_t)a.bitmap_stride;
#pragma unroll
        for (int b = 0; b < (GT + WIDTH - 1) / WIDTH; ++b) {
          const uint32_t w = transpose32(pack_block<WIDTH, GT>(acc, b), trot, tsel);
          const int g = b * WIDTH + (lane % WIDTH);
          const int64_t widx = word0 + g * Swar<WIDTH>::WPG + lane / WIDTH;
          if (g < GT && widx < a.words) {
            out[widx] = w;
            cnt += __popc(w);
          }
        }
      } else {
#pragma unroll
        for (int g = 0; g < GT; ++g)
          if (g0 + g < a.groups) cnt += __popc(acc[g]);
      }
      cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
      if (lane == 0 && cnt) atomicAdd(&a.counts[cand], cnt);
    }
    __syncthreads();  // every warp is done with stage s
    if (tid == 0 && it + 2 < i1) issue(it + 2, s);
  }

  if (timed_out && tid == 0) {
    atomicOr(a.err_out, kErrTimeout);
    atomicOr(a.status, kErrTimeout);
    // wait, again bounded, for the copies still in flight into this CTA's shared memory
    const int s = (int)((it - i0) & 1);
    dev::mbar_wait_bounded(&full_bar[s], (uint32_t)(((it - i0) >> 1) & 1), a.timeout_ns);
    if (it + 1 < i1)
      dev::mbar_wait_bounded(&full_bar[s ^ 1], (uint32_t)(((it + 1 - i0) >> 1) & 1),
                             a.timeout_ns);
  }
}

// The dynamic shared-memory limit of one instantiation, raised on the current device. The
// attribute is a per-device property of the function, so it is set once per device (a bit per
// device index, set after the call succeeded; concurrent first calls may both set it, which is
// harmless). Setting it also loads the function's code on that device under lazy module loading.
template <int WIDTH, int VEC, int TS, bool NEG, bool BITMAPS>
cudaError_t ready_eval_variant() {
  static std::atomic<uint64_t> ready_devices{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
  if (bit && (ready_devices.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(eval_population_kernel<WIDTH, VEC, TS, NEG, BITMAPS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDynMax);
  if (e != cudaSuccess) return e;
  if (bit) ready_devices.fetch_or(bit, std::memory_order_acq_rel);
  return cudaSuccess;
}

template <int WIDTH, int VEC, int TS, bool NEG, bool BITMAPS>
cudaError_t launch_eval_variant(int grid, const CUtensorMap* tmap, const EvalArgs& a,
                                cudaStream_t s) {
  cudaError_t e = ready_eval_variant<WIDTH, VEC, TS, NEG, BITMAPS>();
  if (e != cudaSuccess) return e;
  count_launch();
  eval_population_kernel<WIDTH, VEC, TS, NEG, BITMAPS>
      <<<grid, eval_threads<TS * VEC, NEG>(), a.smem_bytes, s>>>(*tmap, a);
  return cudaGetLastError();
}

// Readies every (NEG, BITMAPS) instantiation of one tile shape on the current device.
template <int WIDTH, int VEC, int TS>
cudaError_t ready_eval_ts() {
  cudaError_t e = ready_eval_variant<WIDTH, VEC, TS, false, false>();
  if (e == cudaSuccess) e = ready_eval_variant<WIDTH, VEC, TS, false, true>();
  if (e == cudaSuccess) e = ready_eval_variant<WIDTH, VEC, TS, true, false>();
  if (e == cudaSuccess) e = ready_eval_variant<WIDTH, VEC, TS, true, true>();
  return e;
}

template <int WIDTH, int VEC, int TS>
cudaError_t launch_eval_ts(const EvalConfig& c, const CUtensorMap* t, const EvalArgs& a,
                           cudaStream_t s) {
  if (c.negative)
    return c.bitmaps ? launch_eval_variant<WIDTH, VEC, TS, true, true>(c.grid, t, a, s)
                     : launch_eval_variant<WIDTH, VEC, TS, true, false>(c.grid, t, a, s);
  return c.bitmaps ? launch_eval_variant<WIDTH, VEC, TS, false, true>(c.grid, t, a, s)
                   : launch_eval_variant<WIDTH, VEC, TS, false, false>(c.grid, t, a, s);
}

// 8-bit ranks (<= 127 columns) can stage 1, 2 or 4 slabs per stage; for 16-bit ranks VEC is
// already chosen so that one slab fills a stage, so only TS = 1 is instantiated.
template <int WIDTH, int VEC>
cudaError_t ready_eval_layout() {
  cudaError_t e = ready_eval_ts<WIDTH, VEC, 1>();
  if constexpr (WIDTH == 8) {
    if (e == cudaSuccess) e = ready_eval_ts<WIDTH, VEC, 2>();
    if (e == cudaSuccess) e = ready_eval_ts<WIDTH, VEC, 4>();
  }
  return e;
}

template <int WIDTH, int VEC>
cudaError_t launch_eval_layout(const EvalConfig& c, const CUtensorMap* t, const EvalArgs& a,
                               cudaStream_t s) {
  if constexpr (WIDTH == 8) {
    switch (c.ts) {
      case 1: return launch_eval_ts<WIDTH, VEC, 1>(c, t, a, s);
      case 2: return launch_eval_ts<WIDTH, VEC, 2>(c, t, a, s);
      case 4: return launch_eval_ts<WIDTH, VEC, 4>(c, t, a, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    if (c.ts != 1) return cudaErrorInvalidValue;
    return launch_eval_ts<WIDTH, VEC, 1>(c, t, a, s);
  }
}

}  // namespace ebic
