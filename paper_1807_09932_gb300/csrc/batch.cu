// Batched evaluation: many populations on many matrices in one persistent launch.
//
// EBIC runs that proceed side by side (many runs, many datasets) each submit one population per
// generation. Scoring each with its own launch leaves most of the GPU idle for small matrices and
// pays a launch per population. Here one persistent kernel scores all of them:
//   * work items are (request, candidate chunk, row tile) triples; a device-side plan kernel turns
//     each request's candidate count and column total into an item range (prefix sums), so the
//     sequence of launches needs no host round trip and can be captured in a CUDA graph;
//   * CTAs take items from one atomic counter (dynamic load balance across uneven candidate
//     lengths, 2-64, and uneven matrix sizes) and prefetch the next item's row tile with TMA into
//     the other of two shared-memory stages while they compute the current one;
//   * every request keeps its own rank layout (8- or 16-bit ranks, VEC, tile height) and
//     negative-trend option; a switch per item selects the matching instantiation of the same
//     inner loop as the single-population evaluator, so results are identical to it;
//   * tensor maps of all matrices sit in a device array.
// A check kernel first validates every request's candidate list on the device (CSR shape,
// column range, repeats) and zeroes its counts; a failed request gets no work items.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ebic.h"
#include "eval_kernel.cuh"
#include "pair_chain.cuh"
#include "prep_dev.cuh"

namespace ebic {
namespace {

// 32 warps per CTA: the cases the batch uses (8-bit ranks with tiles of at most 2 slabs, or 1
// with negative trends; 16-bit ranks with 1 slab) all fit in 64 registers per thread.
constexpr int kBatchThreads = 1024;
constexpr int kBatchWarps = kBatchThreads / 32;

// The largest tile height the batch uses for a request (results never depend on the tile).
int batch_tile_cap(const Layout& L, bool neg) { return L.width == 8 ? (neg ? 1 : 2) : 1; }

// layout cases: 0..2 = 8-bit ranks, VEC 4, TS 1/2/4; 3 = 16-bit VEC 4; 4 = VEC 2; 5 = VEC 1
int layout_case(const Layout& L, int ts) {
  if (L.width == 8) return ts == 1 ? 0 : ts == 2 ? 1 : 2;
  return L.vec == 4 ? 3 : L.vec == 2 ? 4 : 5;
}

struct BatchReq {
  const uint16_t* cand_cols;
  const uint32_t* cand_offsets;
  uint32_t* counts;
  uint32_t* bitmaps;  // may be null: counts only
  uint32_t* status;   // the matrix's deferred-status word
  int64_t slabs, groups, words;
  uint32_t n_cand;
  uint32_t cand_base;  // sum of n_cand of the requests before this one
  int32_t lcase;       // layout case
  int32_t vec;         // row groups per slab
  int32_t neg;
  int32_t ts;
  int32_t col_box, n_col_boxes;
  uint32_t stage_bytes;
  int32_t chunk_cols;
  uint32_t tmap;       // index into the tensor-map array
  const uint32_t* pairs;  // the matrix's pair table: the request runs on the batched pair pass
  uint32_t pair_stride;
  int32_t pair_cols;
  // fitness against an archive (pair-table requests only; fitness null: none)
  uint64_t* fitness;
  const uint16_t* arch_cols;
  const uint32_t* arch_offsets;
  const uint32_t* arch_src;         // the caller's [n_arch][words] archive
  uint32_t* arch_pad;               // scratch: [ov_stride][pair_stride], zero padding
  uint32_t* overlaps;               // scratch: [n_cand][ov_stride], zeroed by the check kernel
  uint32_t* arch_counts;            // scratch: [n_arch], zeroed by the check kernel
  unsigned long long* colmask;      // scratch: [pair_cols] members holding each column
  uint64_t* share;                  // scratch: [n_cand] members sharing a column with each
  uint32_t n_arch;
  uint32_t ov_stride;               // n_arch rounded up to even
  uint32_t* terms;                  // pair-table requests: [n_cand][term_slots(neg)] scratch
};

struct BatchHeader {
  uint32_t n_req;
  uint32_t total_cand;
  unsigned long long next_item;   // work counter, reset by the plan kernel
  unsigned long long total_items;
  unsigned long long grab;        // consecutive items taken per grab (set by the plan kernel)
  uint32_t* zero;                 // the fitness requests' counters, one block of n_zero words
  unsigned long long n_zero;
  uint32_t n_fit;                 // requests with a fitness output (set by the host)
};

constexpr int kCheckWarps = 8;     // warps per block of the check kernel
constexpr int kPlanThreads = 256;  // threads per block of the plan kernel

__device__ __forceinline__ uint32_t find_request(const BatchReq* reqs, uint32_t n, uint32_t cand) {
  uint32_t lo = 0, hi = n;  // last request with cand_base <= cand
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (reqs[mid].cand_base <= cand) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t find_item(const unsigned long long* start, uint32_t n,
                                              unsigned long long g) {
  uint32_t lo = 0, hi = n;  // last request with start <= g
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (start[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Check every candidate of every request (same rules and bounds as the single-population
// check) and zero the counts. Grid-stride, so the grid does not depend on the batch.
__global__ void __launch_bounds__(kCheckWarps * 32)
    batch_check_kernel(const BatchReq* __restrict__ reqs, const BatchHeader* __restrict__ hdr,
                       int32_t* ncols_of, uint32_t* __restrict__ req_err) {
  __shared__ uint32_t sets[kCheckWarps][prepdev::kSetWords];
  const uint32_t n_req = hdr->n_req, total = hdr->total_cand;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a warp per candidate: the single-population check (columns distinct through a bitset in
  // shared memory) and, on a matrix with a pair table, its term list for the pair pass. Each
  // warp takes a contiguous run of candidates. Its lanes load the offsets of up to 32 of them in
  // one round (lane k: candidate k of the chunk, with its request and counter); the columns of
  // two candidates at a time are then loaded into registers together, checked and turned into
  // term lists from there.
  const uint32_t nwarps = gridDim.x * kCheckWarps;
  const uint32_t per = (total + nwarps - 1) / nwarps;
  const uint32_t g0 = (blockIdx.x * kCheckWarps + warp) * per;
  const uint32_t g1 = min(g0 + per, total);
  uint32_t* const set = sets[warp];
  uint32_t r = g0 < g1 ? find_request(reqs, n_req, g0) : 0u;
  for (uint32_t c0 = g0; c0 < g1; c0 += 32) {
    const uint32_t cnt = min(32u, g1 - c0);
    // lane k: candidate c0 + k
    uint32_t rk = r, ik = 0, lok = 0, hik = 0, totk = 0;
    if ((uint32_t)lane < cnt) {
      const uint32_t g = c0 + lane;
      while (rk + 1 < n_req && reqs[rk + 1].cand_base <= g) ++rk;
      const BatchReq& q = reqs[rk];
      ik = g - q.cand_base;
      const uint32_t* offs = q.cand_offsets;
      lok = offs[ik];
      hik = offs[ik + 1];
      totk = offs[q.n_cand];
      q.counts[ik] = 0u;
    }
    r = __shfl_sync(0xFFFFFFFFu, rk, cnt - 1);  // the request of the chunk's last candidate
    for (uint32_t j = 0; j < cnt; j += 2) {
      // candidates j and j + 1 (when there is one): offsets from their lanes, columns loaded
      // for both before either is checked
      uint32_t ra[2], ia[2], lo[2], hi[2], ca_lo[2], ca_hi[2];
      bool sane[2], has[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint32_t src = min(j + t, cnt - 1);
        has[t] = j + t < cnt;
        ra[t] = __shfl_sync(0xFFFFFFFFu, rk, src);
        ia[t] = __shfl_sync(0xFFFFFFFFu, ik, src);
        lo[t] = __shfl_sync(0xFFFFFFFFu, lok, src);
        hi[t] = __shfl_sync(0xFFFFFFFFu, hik, src);
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, totk, src);
        sane[t] = has[t] && prepdev::offsets_sane(lo[t], hi[t], tot, ia[t] == 0);
        ca_lo[t] = ca_hi[t] = 0u;
        if (sane[t])
          prepdev::load_cols_regs(reqs[ra[t]].cand_cols, lo[t], hi[t], lane, ca_lo[t], ca_hi[t]);
      }
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (!has[t]) continue;  // warp-uniform
        const BatchReq& q = reqs[ra[t]];
        const int32_t nc = ncols_of[ra[t]];
        for (int w = lane; w < (nc + 31) / 32; w += 32) set[w] = 0u;
        __syncwarp();
        const uint32_t L = hi[t] - lo[t];
        const bool bad =
            !sane[t] || prepdev::cols_bad_regs(ca_lo[t], ca_hi[t], L, nc, set, lane);
        if (bad) {
          if (lane == 0) {
            atomicOr(&req_err[ra[t]], kErrInvalid);
            atomicOr(q.status, kErrInvalid);
          }
        } else if (q.terms) {
          prepdev::build_terms_regs(ca_lo[t], ca_hi[t], (int)L, (uint32_t)q.pair_cols,
                                    q.pair_stride, q.neg != 0,
                                    q.terms + (size_t)ia[t] * term_slots(q.neg != 0), lane);
        }
        __syncwarp();  // the bitset is rebuilt for the next candidate
      }
    }
  }
  // the fitness requests: counters zeroed, archives copied into rows of the table's stride, the
  // column -> member masks, and the archive lists checked like candidate lists
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nthreads = (size_t)gridDim.x * blockDim.x;
  for (size_t i = tid; i < hdr->n_zero; i += nthreads) hdr->zero[i] = 0u;
  // the requests with an archive, found 32 at a time (a lane per request, one ballot) rather
  // than by one dependent load per request; every warp finds the same ones
  // The archive copy of a request takes every thread; its column -> member masks and its list
  // check take one block (the request's ordinal among them, modulo the grid), which loads every
  // (member, position) of the list in one round and builds the masks in shared memory.
  __shared__ unsigned long long cmask[kMaxCols];
  uint32_t ordinal = 0;
  for (uint32_t r0 = 0; r0 < n_req; r0 += 32) {
    const uint32_t rl = r0 + lane;
    const bool has = rl < n_req && reqs[rl].fitness != nullptr && reqs[rl].n_arch != 0;
    for (uint32_t todo = __ballot_sync(0xFFFFFFFFu, has); todo; todo &= todo - 1u, ++ordinal) {
      const uint32_t r = r0 + (uint32_t)(__ffs(todo) - 1);
      const BatchReq& q = reqs[r];
      prepdev::copy_archive_padded(q.arch_src, q.arch_pad, q.n_arch, q.words, q.pair_stride, tid,
                                   nthreads);
      if (ordinal % gridDim.x != blockIdx.x) continue;  // block-uniform
      const uint32_t* ao = q.arch_offsets;
      const uint32_t na = q.n_arch, atot = ao[na];
      const int pc = q.pair_cols;
      for (int c = threadIdx.x; c < pc; c += blockDim.x) cmask[c] = 0ull;
      __syncthreads();
      bool bad = false;
      for (uint32_t t = threadIdx.x; t < na * (uint32_t)kMaxLen; t += blockDim.x) {
        const uint32_t m = t / kMaxLen, j = t % kMaxLen;
        const uint32_t lo = ao[m], hi = ao[m + 1];
        if (!prepdev::offsets_sane(lo, hi, atot, m == 0)) {
          bad |= j == 0;  // once per member
          continue;
        }
        if (j >= hi - lo) continue;
        const uint32_t c = q.arch_cols[lo + j];
        if (c >= (uint32_t)pc) {
          bad = true;
          continue;
        }
        const unsigned long long bit = 1ull << m;
        bad |= (atomicOr(&cmask[c], bit) & bit) != 0ull;  // the member holds c twice
      }
      if (__syncthreads_or(bad) && threadIdx.x == 0) {
        atomicOr(&req_err[r], kErrInvalid);
        atomicOr(q.status, kErrInvalid);
      }
      for (int c = threadIdx.x; c < pc; c += blockDim.x) q.colmask[c] = cmask[c];
      __syncthreads();  // the masks are rebuilt for the block's next request
    }
  }
}

// Item ranges: request r owns items [start[r], start[r+1]) = chunks x row tiles. One thread.
// Requests on matrices with a pair table get no items here: they own items of the batched pair
// pass instead, [pstart[k][r], pstart[k][r+1]) for k = their negative-trend flag + 2 when they
// have an archive to score against, one item per (range of pairdev::kItemWords words, group of
// pairdev::kPairWarps candidates).
__global__ void batch_plan_kernel(const BatchReq* __restrict__ reqs, BatchHeader* hdr,
                                  const uint32_t* __restrict__ req_err,
                                  unsigned long long* __restrict__ start,
                                  unsigned long long* __restrict__ pstart,
                                  uint32_t n_max, unsigned long long gridDim_eval) {
  // every thread: the share masks of the fitness requests' candidates (the check kernel has
  // built the column masks and rejected bad lists)
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < hdr->total_cand;
       g += gridDim.x * blockDim.x) {
    const uint32_t r = find_request(reqs, hdr->n_req, g);
    const BatchReq& q = reqs[r];
    if (!q.fitness || q.n_arch == 0 || req_err[r] != 0u) continue;
    const uint32_t i = g - q.cand_base;
    unsigned long long mask = 0ull;
    for (uint32_t j = q.cand_offsets[i]; j < q.cand_offsets[i + 1]; ++j)
      mask |= q.colmask[q.cand_cols[j]];
    q.share[i] = mask;
  }
  // block 0: the plan, an exclusive scan of the requests' item counts in five spaces (the four
  // pair passes, then the rank-code pass), each thread taking a contiguous run of requests
  if (blockIdx.x != 0) return;
  __shared__ unsigned long long part[kPlanThreads][5];
  const uint32_t n = hdr->n_req;
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t r0 = min(threadIdx.x * per, n), r1 = min(r0 + per, n);
  auto items_of = [&](uint32_t r, unsigned long long (&sz)[5]) {
    for (int k = 0; k < 5; ++k) sz[k] = 0ull;
    const BatchReq& q = reqs[r];
    if (q.n_cand == 0 || req_err[r] != 0u) return;
    if (q.pairs != nullptr) {
      const unsigned long long ranges = (q.words + pairdev::kItemWords - 1) / pairdev::kItemWords;
      const unsigned long long groups =
          (q.n_cand + pairdev::kPairWarps - 1) / pairdev::kPairWarps;
      sz[(q.neg ? 1 : 0) + (q.fitness && q.n_arch ? 2 : 0)] = ranges * groups;
    } else {
      const unsigned long long total = q.cand_offsets[q.n_cand];
      const unsigned long long chunks = (total + q.chunk_cols - 1) / q.chunk_cols;
      const unsigned long long tiles = (unsigned long long)((q.slabs + q.ts - 1) / q.ts);
      sz[4] = chunks * tiles;
    }
  };
  unsigned long long acc[5] = {0ull, 0ull, 0ull, 0ull, 0ull}, sz[5];
  for (uint32_t r = r0; r < r1; ++r) {
    items_of(r, sz);
    for (int k = 0; k < 5; ++k) acc[k] += sz[k];
  }
  for (int k = 0; k < 5; ++k) part[threadIdx.x][k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive offsets of the threads' runs, and the totals
    unsigned long long run[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
    for (uint32_t t = 0; t < blockDim.x; ++t)
      for (int k = 0; k < 5; ++k) {
        const unsigned long long v = part[t][k];
        part[t][k] = run[k];
        run[k] += v;
      }
    for (int k = 0; k < 4; ++k) pstart[k * (n_max + 1) + n] = run[k];
    start[n] = run[4];
    hdr->total_items = run[4];
    hdr->next_item = 0ull;
  }
  __syncthreads();
  for (int k = 0; k < 5; ++k) acc[k] = part[threadIdx.x][k];
  for (uint32_t r = r0; r < r1; ++r) {
    for (int k = 0; k < 4; ++k) pstart[k * (n_max + 1) + r] = acc[k];
    start[r] = acc[4];
    items_of(r, sz);
    for (int k = 0; k < 5; ++k) acc[k] += sz[k];
  }
  if (threadIdx.x != 0) return;
  const unsigned long long acc_total = start[n];
  // runs of consecutive items (same candidate chunk, neighbouring row tiles) keep chunk restaging
  // and item decoding rare; about 8 runs per CTA keep the dynamic balance
  const unsigned long long runs = 8ull * gridDim_eval;
  unsigned long long g = (acc_total + runs - 1) / runs;
  hdr->grab = g < 1 ? 1 : (g > 64 ? 64 : g);
}

// One row tile of one request for every candidate of the staged chunk.
template <int WIDTH, int VEC, int TS, bool NEG>
__device__ __forceinline__ void batch_tile(const uint8_t* stage, const BatchReq& q,
                                           const uint16_t* ccols, const uint16_t* coffs,
                                           uint32_t lo, uint32_t nc, int64_t tile, int lane,
                                           int warp, const uint32_t (&trot)[5],
                                           const uint32_t (&tsel)[5]) {
  constexpr int GT = TS * VEC;
  constexpr int WPT = GT * Swar<WIDTH>::WPG;
  const uint32_t col_stride = TS * 128 * VEC;
  const uint8_t* lane_base = stage + lane * 4 * VEC;
  const int64_t word0 = tile * WPT;
  const int64_t g0 = tile * GT;
  for (uint32_t ci = warp; ci < nc; ci += kBatchWarps) {
    const int o = coffs[ci];
    const int L = coffs[ci + 1] - o;
    uint32_t acc[GT];
    trend_masks<WIDTH, VEC, TS, NEG>(lane_base, col_stride, ccols + o, L, acc);
    const uint32_t cand = lo + ci;
    uint32_t cnt = 0;
    if (q.bitmaps) {
      uint32_t* out = q.bitmaps + (size_t)cand * (size_t)q.words;
#pragma unroll
      for (int b = 0; b < (GT + WIDTH - 1) / WIDTH; ++b) {
        const uint32_t w = transpose32(pack_block<WIDTH, GT>(acc, b), trot, tsel);
        const int g = b * WIDTH + (lane % WIDTH);
        const int64_t widx = word0 + g * Swar<WIDTH>::WPG + lane / WIDTH;
        if (g < GT && widx < q.words) {
          out[widx] = w;
          cnt += __popc(w);
        }
      }
    } else {
#pragma unroll
      for (int g = 0; g < GT; ++g)
        if (g0 + g < q.groups) cnt += __popc(acc[g]);
    }
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (lane == 0 && cnt) atomicAdd(&q.counts[cand], cnt);
  }
}

template <bool NEG>
__device__ __forceinline__ void batch_tile_case(int lcase, const uint8_t* stage,
                                                const BatchReq& q, const uint16_t* ccols,
                                                const uint16_t* coffs, uint32_t lo, uint32_t nc,
                                                int64_t tile, int lane, int warp,
                                                const uint32_t (&trot)[5],
                                                const uint32_t (&tsel)[5]) {
  switch (lcase) {
    case 0: batch_tile<8, 4, 1, NEG>(stage, q, ccols, coffs, lo, nc, tile, lane, warp, trot, tsel); break;
    case 1:
      if constexpr (!NEG)
        batch_tile<8, 4, 2, NEG>(stage, q, ccols, coffs, lo, nc, tile, lane, warp, trot, tsel);
      break;
    case 3: batch_tile<16, 4, 1, NEG>(stage, q, ccols, coffs, lo, nc, tile, lane, warp, trot, tsel); break;
    case 4: batch_tile<16, 2, 1, NEG>(stage, q, ccols, coffs, lo, nc, tile, lane, warp, trot, tsel); break;
    default: batch_tile<16, 1, 1, NEG>(stage, q, ccols, coffs, lo, nc, tile, lane, warp, trot, tsel); break;
  }
}

// Shared memory: [stage 0][stage 1][chunk columns (chunk_cap + slack)][chunk offsets]
__global__ void __launch_bounds__(kBatchThreads, 1)
    batch_eval_kernel(const BatchReq* __restrict__ reqs, const CUtensorMap* __restrict__ tmaps,
                      BatchHeader* hdr, const unsigned long long* __restrict__ start,
                      uint32_t stage_cap, int32_t chunk_cap, uint64_t timeout_ns,
                      uint32_t* err_out) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full_bar[2];
  __shared__ unsigned long long item_s[2];
  __shared__ BatchReq q;
  __shared__ uint32_t cur_r, cur_lo, cur_nc;
  __shared__ long long cur_k;
  __shared__ long long it_tile;
  __shared__ int it_stage;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t trot[5], tsel[5];
  transpose_consts(lane, trot, tsel);
  const uint32_t n_req = hdr->n_req;
  const unsigned long long total = hdr->total_items;
  uint8_t* const stage0 = smem;
  uint8_t* const stage1 = smem + stage_cap;
  uint16_t* const ccols = reinterpret_cast<uint16_t*>(smem + 2 * (size_t)stage_cap);
  uint16_t* const coffs = ccols + chunk_cap + kChunkSlack;

  // thread-0 state: the current run of grabbed items and the request whose range was decoded last
  unsigned long long run_next = 0, run_end = 0;
  uint32_t dec_r = 0;
  unsigned long long dec_lo = 1, dec_hi = 0;
  auto next_item = [&]() -> unsigned long long {  // thread 0 only
    if (run_next >= run_end) {
      const unsigned long long gsz = hdr->grab;
      run_next = atomicAdd(&hdr->next_item, gsz);
      run_end = run_next + gsz < total ? run_next + gsz : total;
      if (run_next >= total) return total;
    }
    return run_next++;
  };
  auto decode = [&](unsigned long long g) -> uint32_t {  // thread 0 only
    if (g < dec_lo || g >= dec_hi) {
      dec_r = find_item(start, n_req, g);
      dec_lo = start[dec_r];
      dec_hi = start[dec_r + 1];
    }
    return dec_r;
  };
  auto issue = [&](unsigned long long g, int s) {  // thread 0 only
    const uint32_t r = decode(g);
    const BatchReq& rq = reqs[r];
    const unsigned long long local = g - dec_lo;
    const long long n_tiles = (rq.slabs + rq.ts - 1) / rq.ts;
    const long long tile = (long long)(local % (unsigned long long)n_tiles);
    const uint32_t col_stride = (uint32_t)rq.ts * 128u * (uint32_t)rq.vec;
    uint8_t* dst = s ? stage1 : stage0;
    dev::acquire_tensormap(&tmaps[rq.tmap]);
    dev::mbar_arrive_expect_tx(&full_bar[s], rq.stage_bytes);
    for (int b = 0; b < rq.n_col_boxes; ++b)
      dev::tma_load_3d(dst + (size_t)b * rq.col_box * col_stride, &tmaps[rq.tmap], &full_bar[s],
                       0, (int32_t)(tile * rq.ts), b * rq.col_box);
  };

  if (tid == 0) {
    dev::mbar_init(&full_bar[0], 1);
    dev::mbar_init(&full_bar[1], 1);
    dev::fence_barrier_init();
    cur_r = 0xFFFFFFFFu;
    cur_k = -1;
    for (int s = 0; s < 2; ++s) {
      const unsigned long long g = next_item();
      item_s[s] = g;
      if (g < total) issue(g, s);
    }
  }
  __syncthreads();

  bool timed_out = false;
  int it = 0;
  for (;; ++it) {
    const int s = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const unsigned long long g = item_s[s];
    if (g >= total) break;
    // thread 0 decides, before the barrier, whether this item needs a new chunk staged, so that
    // every thread takes the same branch
    if (tid == 0) {
      const uint32_t r = decode(g);
      const unsigned long long local = g - dec_lo;
      const long long n_tiles = (reqs[r].slabs + reqs[r].ts - 1) / reqs[r].ts;
      const long long k = (long long)(local / (unsigned long long)n_tiles);
      it_tile = (long long)(local % (unsigned long long)n_tiles);
      it_stage = (r != cur_r || k != cur_k) ? 1 : 0;
      if (it_stage) {
        q = reqs[r];
        const uint32_t l = lower_bound_u32(q.cand_offsets, q.n_cand, (uint64_t)k * q.chunk_cols);
        const uint32_t h =
            lower_bound_u32(q.cand_offsets, q.n_cand, (uint64_t)(k + 1) * q.chunk_cols);
        cur_lo = l;
        cur_nc = h - l;
        cur_r = r;
        cur_k = k;
      }
    }
    __syncthreads();
    const long long tile = it_tile;
    if (it_stage) {  // stage the chunk's candidate lists
      const uint32_t c0 = q.cand_offsets[cur_lo];
      const uint32_t span = q.cand_offsets[cur_lo + cur_nc] - c0;
      for (uint32_t i = tid; i < span; i += kBatchThreads) ccols[i] = q.cand_cols[c0 + i];
      for (uint32_t i = tid; i <= cur_nc; i += kBatchThreads)
        coffs[i] = (uint16_t)(q.cand_offsets[cur_lo + i] - c0);
      __syncthreads();
    }
    const bool ok = dev::mbar_wait_bounded(&full_bar[s], parity, timeout_ns);
    if (!__syncthreads_and(ok)) { timed_out = true; break; }
    const uint8_t* stage = s ? stage1 : stage0;
    if (q.neg)
      batch_tile_case<true>(q.lcase, stage, q, ccols, coffs, cur_lo, cur_nc, tile, lane, warp,
                            trot, tsel);
    else
      batch_tile_case<false>(q.lcase, stage, q, ccols, coffs, cur_lo, cur_nc, tile, lane, warp,
                             trot, tsel);
    __syncthreads();  // every warp is done with stage s
    if (tid == 0) {  // item_s[s] is next read two iterations on, after further barriers
      const unsigned long long gn = next_item();
      item_s[s] = gn;
      if (gn < total) issue(gn, s);
    }
  }
  if (timed_out && tid == 0) {
    atomicOr(err_out, kErrTimeout);
    atomicOr(q.status, kErrTimeout);
    // wait, bounded, for the copies still in flight into this CTA's shared memory
    for (int d = 0; d < 2; ++d) {
      const int s = (it + d) & 1;
      if (item_s[s] < total)
        dev::mbar_wait_bounded(&full_bar[s], (uint32_t)(((it + d) >> 1) & 1), timeout_ns);
    }
  }
}

// The batched pair-table pass: every request whose matrix has a pair table and whose negative-
// trend flag is NEG, its items (range of kItemWords words, group of kPairWarps candidates) laid
// end to end in request order and taken round-robin by a persistent grid, so the CTAs walk each
// request's ranges in order and its table rows stay in L2 while its candidates read them. The
// chain and epilogue are the single-population pass's (pair_chain.cuh); the term list is
// computed in registers from the checked candidate list.
constexpr uint32_t kStartCache = 1024;  // item starts kept in shared memory (requests)

template <bool NEG, bool FIT>
__global__ void __launch_bounds__(pairdev::kPairThreads, 1)
    batch_pair_kernel(const BatchReq* __restrict__ reqs, const BatchHeader* __restrict__ hdr,
                      const unsigned long long* __restrict__ pstart) {
  __shared__ __align__(16) uint32_t stage[pairdev::kPairWarps][pairdev::kRangeWords];
  __shared__ unsigned long long starts[kStartCache + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n_req = hdr->n_req;
  // the item starts, searched once per item: from shared memory when they fit
  const bool cached = n_req <= kStartCache;
  if (cached)
    for (uint32_t i = threadIdx.x; i <= n_req; i += blockDim.x) starts[i] = pstart[i];
  __syncthreads();
  const unsigned long long* ps = cached ? starts : pstart;
  const unsigned long long total = ps[n_req];
  // an item's request, row range and this warp's candidate in it
  struct Item {
    uint32_t r = 0, cand = 0xFFFFFFFFu;
    uint64_t range = 0;
    bool first_group = false;
  };
  auto decode = [&](unsigned long long it) {
    Item m;
    m.r = find_item(ps, n_req, it);
    const BatchReq& q = reqs[m.r];
    const unsigned long long local = it - ps[m.r];
    const uint32_t n_groups = (q.n_cand + pairdev::kPairWarps - 1) / pairdev::kPairWarps;
    m.range = local / n_groups;
    const uint64_t grp = local - m.range * n_groups;
    m.first_group = grp == 0;
    m.cand = (uint32_t)grp * pairdev::kPairWarps + warp;
    return m;
  };
  // the term list (written by the check kernel) and share mask of the warp's next item are
  // loaded while the current one is walked
  auto fetch = [&](const Item& m, pairdev::Terms& t, uint64_t& sh) {
    const BatchReq& q = reqs[m.r];
    if (m.cand >= q.n_cand) return;
    const uint32_t* tp = q.terms + (uint64_t)m.cand * (NEG ? 2 * kTermSlots : kTermSlots);
    t.lo = __ldg(tp + lane);
    t.hi = __ldg(tp + 32 + lane);
    if (NEG) {
      t.blo = __ldg(tp + 64 + lane);
      t.bhi = __ldg(tp + 96 + lane);
    }
    if (FIT) sh = __ldg(q.share + m.cand);
  };
  unsigned long long it = blockIdx.x;
  Item nxt;
  pairdev::Terms t_next;
  uint64_t sh_next = 0;
  if (it < total) {
    nxt = decode(it);
    fetch(nxt, t_next, sh_next);
  }
  while (it < total) {
    const Item m = nxt;
    const pairdev::Terms t = t_next;
    const uint64_t sh = sh_next;
    it += gridDim.x;
    if (it < total) {
      nxt = decode(it);
      fetch(nxt, t_next, sh_next);
    }
    const BatchReq& q = reqs[m.r];
    const uint64_t rword = m.range * pairdev::kItemWords;
    if (FIT && m.first_group) {  // the archive members' own row counts, once per range
      for (uint32_t a = warp; a < q.n_arch; a += pairdev::kPairWarps) {
        const uint32_t* ar = q.arch_pad + (uint64_t)a * q.pair_stride + rword + 4 * lane;
        uint32_t pa4 = 0;
#pragma unroll
        for (int k = 0; k < pairdev::kParts; ++k)
          pa4 += pairdev::popc4(pairdev::ld_arch4(ar + k * pairdev::kRangeWords));
        const uint32_t n = __reduce_add_sync(0xFFFFFFFFu, pa4);
        if (lane == 0 && n) atomicAdd(&q.arch_counts[a], n);
      }
    }
    if (m.cand >= q.n_cand) continue;  // warp-uniform
    const uint32_t cand = m.cand;
    uint4 x[pairdev::kParts];
    pairdev::pair_chain<NEG>(t, q.pairs + rword + 4 * lane,
                             pair_ones(q.pairs, (uint64_t)q.pair_cols, q.pair_stride), lane,
                             x);
    uint32_t pc = 0;
#pragma unroll
    for (int k = 0; k < pairdev::kParts; ++k) pc += pairdev::popc4(x[k]);
    const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, pc);
    if (lane == 0 && c) atomicAdd(&q.counts[cand], c);
    PairArgs pa;
    pa.bitmaps = q.bitmaps;
    pa.W = q.words;
    if constexpr (FIT) {
      pa.arch = q.arch_pad;
      pa.stride = q.pair_stride;
      pa.n_arch = q.n_arch;
      pa.overlaps = q.overlaps;
      pa.ov_stride = q.ov_stride;
      const int n_pairs = (int)(q.n_arch + 1) >> 1;
      if (q.bitmaps)  // warp-uniform
        pairdev::item_epilogue<true, true>(pa, cand, rword, x, c, stage[warp], lane, q.n_arch,
                                           n_pairs, sh);
      else
        pairdev::item_epilogue<false, true>(pa, cand, rword, x, c, stage[warp], lane, q.n_arch,
                                            n_pairs, sh);
    } else if (q.bitmaps) {  // warp-uniform
      pairdev::item_epilogue<true, false>(pa, cand, rword, x, c, stage[warp], lane, 0u, 0, 0ull);
    }
  }
}

// F_c of every candidate of the fitness requests, a warp per candidate (as ebic_eval_fitness's
// finalize), after the batched pair pass. Requests that failed their check get no fitness.
__global__ void batch_fitness_kernel(const BatchReq* __restrict__ reqs,
                                     const BatchHeader* __restrict__ hdr,
                                     const uint32_t* __restrict__ req_err) {
  const int lane = threadIdx.x & 31;
  if (hdr->n_fit == 0) return;
  const uint32_t n_req = hdr->n_req;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (uint32_t r = 0; r < n_req; ++r) {
    const BatchReq& q = reqs[r];
    if (!q.fitness || req_err[r] != 0u) continue;  // the same for the whole grid
    for (uint32_t i = gw; i < q.n_cand; i += nw) {
      const uint32_t o = q.cand_offsets[i];
      const uint32_t L = q.cand_offsets[i + 1] - o;
      if (q.n_arch == 0) {
        if (lane == 0) q.fitness[i] = (uint64_t)q.counts[i] << ((L < 33u ? L : 33u) - 1u);
        continue;
      }
      const uint64_t sh = q.share[i];
      const uint32_t* ao = q.arch_offsets;
      const uint32_t al0 = lane < (int)q.n_arch ? ao[lane + 1] - ao[lane] : 0u;
      const uint32_t al1 = lane + 32 < (int)q.n_arch ? ao[lane + 33] - ao[lane + 32] : 0u;
      prepdev::fused_fitness_mask(i, L, al0, al1, q.n_arch, sh, q.counts, q.overlaps,
                                  q.ov_stride, q.arch_counts, q.fitness, lane);
    }
  }
}

}  // namespace
}  // namespace ebic

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
using namespace ebic;

namespace {

struct HostPlan {
  std::vector<BatchReq> reqs;
  std::vector<CUtensorMap> tmaps;
  std::vector<int32_t> ncols;
  uint32_t total_cand = 0;
  uint32_t stage_cap = 0;
  int32_t chunk_cap = 0;
  int device = -1;
  int num_sms = 0;
  size_t fit_bytes = 0;  // device scratch of the fitness requests (see place_fitness)
};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The batch's scratch, in one block: first the fitness requests' counters, contiguous so that
// one loop zeroes them (per request: overlaps [n_cand][ov_stride], then archive counts
// [ov_stride], so every overlap row starts on 8 bytes), then their padded archives, column
// masks and share masks, then the term lists of every pair-table request. With base null only
// the size is computed (hp->fit_bytes); else the pointers are set, and the counter block is
// reported in *zero / *n_zero.
void place_fitness(HostPlan* hp, uint8_t* base, uint32_t** zero, unsigned long long* n_zero) {
  size_t words = 0;
  for (BatchReq& q : hp->reqs) {
    if (!q.fitness || q.n_arch == 0) continue;
    if (base) {
      q.overlaps = reinterpret_cast<uint32_t*>(base) + words;
      q.arch_counts = q.overlaps + (size_t)q.n_cand * q.ov_stride;
    }
    words += ((size_t)q.n_cand + 1) * q.ov_stride;
  }
  if (base) {
    *zero = reinterpret_cast<uint32_t*>(base);
    *n_zero = words;
  }
  size_t off = round_up(words * 4, 256);
  for (BatchReq& q : hp->reqs) {
    if (!q.fitness || q.n_arch == 0) continue;
    if (base) q.arch_pad = reinterpret_cast<uint32_t*>(base + off);
    off += round_up((size_t)q.ov_stride * q.pair_stride * 4, 256);
  }
  for (BatchReq& q : hp->reqs) {
    if (!q.fitness || q.n_arch == 0) continue;
    if (base) q.colmask = reinterpret_cast<unsigned long long*>(base + off);
    off += round_up((size_t)q.pair_cols * 8, 256);
    if (base) q.share = reinterpret_cast<uint64_t*>(base + off);
    off += round_up((size_t)q.n_cand * 8, 256);
  }
  for (BatchReq& q : hp->reqs) {
    if (!q.pairs || q.n_cand == 0) continue;
    if (base) q.terms = reinterpret_cast<uint32_t*>(base + off);
    off += round_up((size_t)q.n_cand * term_slots(q.neg != 0) * 4, 256);
  }
  hp->fit_bytes = off;
}

bool is_dev(const void* p, int dev) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

// Host-side checks and per-request plans. fixed_stage_cap > 0 fixes the stage size (graphs).
int build_plan(const ebic_eval_request* reqs, uint32_t n, uint32_t fixed_stage_cap,
               HostPlan* hp) {
  hp->reqs.clear();
  hp->tmaps.clear();
  hp->ncols.clear();
  hp->total_cand = 0;
  uint64_t total = 0;
  uint32_t cap = fixed_stage_cap;
  std::vector<EvalArgs> args(n);
  std::vector<EvalConfig> cfgs(n);
  std::vector<const CUtensorMap*> maps(n);
  for (uint32_t i = 0; i < n; ++i) {
    const ebic_eval_request& r = reqs[i];
    if (!r.m) return set_last_error(EBIC_ERR_INVALID_ARG, "request has a NULL matrix");
    MatrixView v;
    matrix_view(r.m, &v);
    if (hp->device < 0) {
      hp->device = v.device;
      hp->num_sms = v.num_sms;
    }
    if (v.device != hp->device)
      return set_last_error(EBIC_ERR_INVALID_ARG, "all requests must use matrices of one device");
    if (r.flags & ~EBIC_NEGATIVE_TRENDS) return set_last_error(EBIC_ERR_INVALID_ARG, "unknown flag");
    if (r.n_cand > 0) {
      if (!is_dev(r.cols, v.device) || !is_dev(r.offsets, v.device) ||
          !is_dev(r.counts, v.device) || (r.bitmaps && !is_dev(r.bitmaps, v.device)))
        return set_last_error(EBIC_ERR_INVALID_ARG,
                              ("request " + std::to_string(i) +
                               ": batched requests take device buffers only").c_str());
    }
    if (r.fitness) {
      const std::string who = "request " + std::to_string(i) + ": ";
      if (!v.pairs)
        return set_last_error(EBIC_ERR_UNSUPPORTED,
                              (who + "fitness in a batch needs the matrix's pair table").c_str());
      if (r.n_arch > (uint32_t)kPairMaxArch)
        return set_last_error(EBIC_ERR_INVALID_ARG, (who + "more than 64 archive members").c_str());
      if ((r.n_cand > 0 && !is_dev(r.fitness, v.device)) ||
          (r.n_arch > 0 && (!is_dev(r.arch_cols, v.device) || !is_dev(r.arch_offsets, v.device) ||
                            !is_dev(r.arch_bitmaps, v.device))))
        return set_last_error(EBIC_ERR_INVALID_ARG,
                              (who + "the archive and fitness must be device buffers").c_str());
    }
    int rc = matrix_eval_plan(r.m, r.n_cand > 0 ? r.n_cand : 1, 0, &args[i], &cfgs[i], &maps[i],
                              batch_tile_cap(v.L, (r.flags & EBIC_NEGATIVE_TRENDS) != 0));
    if (rc != EBIC_OK) return rc;
    if (!fixed_stage_cap && args[i].stage_bytes > cap) cap = args[i].stage_bytes;
    if (args[i].stage_bytes > cap)
      return set_last_error(EBIC_ERR_UNSUPPORTED, "a request's tile exceeds the batch's stage");
    total += r.n_cand;
  }
  if (total > 0xFFFFFFFFull) return set_last_error(EBIC_ERR_UNSUPPORTED, "too many candidates");
  int64_t cc_cap = (kSmemDynMax - 2 * (int64_t)cap - 2 * (kChunkSlack + 1) - 256) / 4;
  cc_cap = std::min<int64_t>(cc_cap, kMaxChunkCols) / 64 * 64;
  if (cc_cap < 64) return set_last_error(EBIC_ERR_UNSUPPORTED, "no shared-memory plan");
  hp->stage_cap = cap;
  hp->chunk_cap = (int32_t)cc_cap;
  uint32_t base = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const ebic_eval_request& r = reqs[i];
    const EvalArgs& a = args[i];
    BatchReq q;
    std::memset(&q, 0, sizeof(q));
    q.cand_cols = r.cols;
    q.cand_offsets = r.offsets;
    q.counts = r.counts;
    q.bitmaps = r.bitmaps;
    MatrixView v;
    matrix_view(r.m, &v);
    q.status = v.status;
    q.slabs = a.slabs;
    q.groups = a.groups;
    q.words = a.words;
    q.n_cand = r.n_cand;
    q.cand_base = base;
    q.lcase = layout_case(v.L, cfgs[i].ts);
    q.vec = v.L.vec;
    q.neg = (r.flags & EBIC_NEGATIVE_TRENDS) ? 1 : 0;
    q.ts = cfgs[i].ts;
    q.col_box = a.col_box;
    q.n_col_boxes = a.n_col_boxes;
    q.stage_bytes = a.stage_bytes;
    // chunks: about 2 items per SM over the whole batch is enough with dynamic scheduling
    q.chunk_cols = std::min<int32_t>(hp->chunk_cap, std::max<int32_t>(64, a.chunk_cols));
    q.tmap = i;
    q.pairs = v.pairs;
    q.pair_stride = v.pair_stride;
    q.pair_cols = v.L.cols;
    if (r.fitness) {
      q.fitness = r.fitness;
      q.n_arch = r.n_arch;
      q.ov_stride = (r.n_arch + 1u) & ~1u;
      q.arch_cols = r.arch_cols;
      q.arch_offsets = r.arch_offsets;
      q.arch_src = r.arch_bitmaps;
    }
    hp->tmaps.push_back(*maps[i]);
    hp->ncols.push_back(v.L.cols);
    hp->reqs.push_back(q);
    base += r.n_cand;
  }
  hp->total_cand = base;
  place_fitness(hp, nullptr, nullptr, nullptr);
  return EBIC_OK;
}

int cerr(cudaError_t e, const char* what) {
  (void)cudaGetLastError();
  return set_last_error(e == cudaErrorMemoryAllocation ? EBIC_ERR_OOM : EBIC_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

#define B_CUDA(expr)                               \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cerr(e_, #expr); \
  } while (0)

// Device-side buffers of one batch (capacity n_max requests).
struct DeviceBatch {
  BatchReq* reqs = nullptr;
  CUtensorMap* tmaps = nullptr;
  int32_t* ncols = nullptr;
  uint32_t* req_err = nullptr;
  unsigned long long* start = nullptr;
  unsigned long long* pstart = nullptr;  // [4][n_max + 1]: the pair passes' item starts
  BatchHeader* hdr = nullptr;
  uint32_t* err = nullptr;
  uint32_t n_max = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t batch_bytes(uint32_t n_max) {
  return align256(sizeof(BatchReq) * n_max) + align256(sizeof(CUtensorMap) * n_max) +
         align256(4 * (size_t)n_max) + align256(4 * (size_t)n_max) +
         align256(8 * ((size_t)n_max + 1)) + align256(32 * ((size_t)n_max + 1)) +
         align256(sizeof(BatchHeader)) + 256;
}

void carve(uint8_t* base, uint32_t n_max, DeviceBatch* d) {
  size_t o = 0;
  d->reqs = reinterpret_cast<BatchReq*>(base + o);
  o += align256(sizeof(BatchReq) * n_max);
  d->tmaps = reinterpret_cast<CUtensorMap*>(base + o);
  o += align256(sizeof(CUtensorMap) * n_max);
  d->ncols = reinterpret_cast<int32_t*>(base + o);
  o += align256(4 * (size_t)n_max);
  d->req_err = reinterpret_cast<uint32_t*>(base + o);
  o += align256(4 * (size_t)n_max);
  d->start = reinterpret_cast<unsigned long long*>(base + o);
  o += align256(8 * ((size_t)n_max + 1));
  d->pstart = reinterpret_cast<unsigned long long*>(base + o);
  o += align256(32 * ((size_t)n_max + 1));
  d->hdr = reinterpret_cast<BatchHeader*>(base + o);
  o += align256(sizeof(BatchHeader));
  d->err = reinterpret_cast<uint32_t*>(base + o);
  d->n_max = n_max;
}

int ensure_batch_attr() {
  static std::once_flag once;
  static cudaError_t e = cudaSuccess;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(batch_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemDynMax);
  });
  if (e != cudaSuccess) return cerr(e, "cudaFuncSetAttribute(batch_eval_kernel)");
  return EBIC_OK;
}

// The launches of a batch (check, plan, the rank-code pass, the two pair-table passes, the
// fitness), stream-ordered.
int launch_batch(const DeviceBatch& d, uint32_t stage_cap, int32_t chunk_cap, int num_sms,
                 cudaStream_t s) {
  const size_t smem = 2 * (size_t)stage_cap + 2 * ((size_t)chunk_cap + kChunkSlack) +
                      2 * ((size_t)chunk_cap + 1) + 16;
  int rc = ensure_batch_attr();
  if (rc != EBIC_OK) return rc;
  count_launch();
  batch_check_kernel<<<8 * num_sms, kCheckWarps * 32, 0, s>>>(d.reqs, d.hdr, d.ncols, d.req_err);
  B_CUDA(cudaGetLastError());
  count_launch();
  batch_plan_kernel<<<4 * num_sms, kPlanThreads, 0, s>>>(d.reqs, d.hdr, d.req_err, d.start,
                                                         d.pstart, d.n_max,
                                                         (unsigned long long)num_sms);
  B_CUDA(cudaGetLastError());
  count_launch();
  batch_eval_kernel<<<num_sms, kBatchThreads, smem, s>>>(d.reqs, d.tmaps, d.hdr, d.start,
                                                          stage_cap, chunk_cap, 1000000000ull,
                                                          d.err);
  B_CUDA(cudaGetLastError());
  // the requests on matrices with a pair table, by trend option and archive (an item space
  // without requests: its grid exits at once)
  const size_t ps = (size_t)d.n_max + 1;
  count_launch();
  batch_pair_kernel<false, false><<<num_sms, pairdev::kPairThreads, 0, s>>>(d.reqs, d.hdr,
                                                                           d.pstart);
  B_CUDA(cudaGetLastError());
  count_launch();
  batch_pair_kernel<true, false><<<num_sms, pairdev::kPairThreads, 0, s>>>(d.reqs, d.hdr,
                                                                          d.pstart + ps);
  B_CUDA(cudaGetLastError());
  count_launch();
  batch_pair_kernel<false, true><<<num_sms, pairdev::kPairThreads, 0, s>>>(d.reqs, d.hdr,
                                                                          d.pstart + 2 * ps);
  B_CUDA(cudaGetLastError());
  count_launch();
  batch_pair_kernel<true, true><<<num_sms, pairdev::kPairThreads, 0, s>>>(d.reqs, d.hdr,
                                                                         d.pstart + 3 * ps);
  B_CUDA(cudaGetLastError());
  // the fitness of the requests that asked for it (none: the grid finds no such request)
  count_launch();
  batch_fitness_kernel<<<4 * num_sms, 256, 0, s>>>(d.reqs, d.hdr, d.req_err);
  B_CUDA(cudaGetLastError());
  return EBIC_OK;
}

void fill_header(const HostPlan& hp, uint32_t n, BatchHeader* h) {
  std::memset(h, 0, sizeof(*h));
  h->n_req = n;
  h->total_cand = hp.total_cand;
  for (const BatchReq& q : hp.reqs) h->n_fit += q.fitness != nullptr;
}

}  // namespace

struct ebic_batch {
  uint32_t n_max = 0;
  int device = 0;
  int num_sms = 0;
  uint8_t* dmem = nullptr;   // device buffers
  uint8_t* hmem = nullptr;   // pinned mirror of the request/tensor-map/ncols/header part
  DeviceBatch d, h;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool pending = false;
  uint32_t last_n = 0;
  uint8_t* fmem = nullptr;   // the fitness requests' scratch, grown when a run needs more
  size_t fbytes = 0;
  std::mutex mu;
};

extern "C" {

int ebic_eval_batch(const ebic_eval_request* reqs, uint32_t n_req, void* stream) {
  if (n_req == 0) return EBIC_OK;
  if (!reqs) return set_last_error(EBIC_ERR_INVALID_ARG, "reqs is NULL");
  HostPlan hp;
  int rc = build_plan(reqs, n_req, 0, &hp);
  if (rc != EBIC_OK) return rc;
  if (hp.total_cand == 0) return EBIC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { (void)cudaGetLastError(); prev = -1; }
  if (prev != hp.device) B_CUDA(cudaSetDevice(hp.device));
  void* mem = nullptr;
  const size_t bb = round_up(batch_bytes(n_req), 256);
  B_CUDA(cudaMallocAsync(&mem, bb + hp.fit_bytes, s));
  DeviceBatch d;
  carve(static_cast<uint8_t*>(mem), n_req, &d);
  BatchHeader h;
  fill_header(hp, n_req, &h);
  place_fitness(&hp, static_cast<uint8_t*>(mem) + bb, &h.zero, &h.n_zero);
  cudaError_t e = cudaMemcpyAsync(d.reqs, hp.reqs.data(), sizeof(BatchReq) * n_req,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.tmaps, hp.tmaps.data(), sizeof(CUtensorMap) * n_req,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.ncols, hp.ncols.data(), 4 * (size_t)n_req, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.req_err, 0, 4 * (size_t)n_req, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, 4, s);
  if (e != cudaSuccess) {
    (void)cudaFreeAsync(mem, s);
    return cerr(e, "batch set-up");
  }
  rc = launch_batch(d, hp.stage_cap, hp.chunk_cap, hp.num_sms, s);
  cudaError_t f = cudaFreeAsync(mem, s);
  if (prev >= 0 && prev != hp.device) (void)cudaSetDevice(prev);
  if (rc != EBIC_OK) return rc;
  if (f != cudaSuccess) return cerr(f, "cudaFreeAsync");
  return EBIC_OK;
}

int ebic_batch_create(uint32_t max_requests, ebic_batch** out) {
  if (!out || max_requests == 0 || max_requests > 65536)
    return set_last_error(EBIC_ERR_INVALID_ARG, "max_requests must be in [1, 65536]");
  *out = nullptr;
  ebic_batch* b = new ebic_batch();
  b->n_max = max_requests;
  auto fail_free = [&](int code) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->done) cudaEventDestroy(b->done);
    if (b->dmem) cudaFree(b->dmem);
    if (b->hmem) cudaFreeHost(b->hmem);
    delete b;
    return code;
  };
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  const size_t bytes = batch_bytes(max_requests);
  if (e == cudaSuccess) e = cudaMalloc(&b->dmem, bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&b->hmem, bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail_free(cerr(e, "ebic_batch_create"));
  std::memset(b->hmem, 0, bytes);
  carve(b->dmem, max_requests, &b->d);
  carve(b->hmem, max_requests, &b->h);
  int arc = ensure_batch_attr();  // before the capture: not a stream operation
  if (arc != EBIC_OK) return fail_free(arc);
  // capture: copy the descriptor block (pinned -> device), clear the error words, then the
  // three kernels; the stage size is fixed at the largest tile so any batch composition fits
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail_free(cerr(e, "capture stream"));
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  const size_t desc_bytes = reinterpret_cast<uint8_t*>(b->d.req_err) - b->dmem;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->dmem, b->hmem, desc_bytes, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d.hdr, b->h.hdr, sizeof(BatchHeader), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d.req_err, 0, 4 * (size_t)max_requests, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d.err, 0, 4, cs);
  int rc = EBIC_OK;
  if (e == cudaSuccess) {
    const int64_t cc = std::min<int64_t>(
        kMaxChunkCols, (kSmemDynMax - 2 * (int64_t)kStageMax - 2 * (kChunkSlack + 1) - 256) / 4);
    rc = launch_batch(b->d, kStageMax, (int32_t)(cc / 64 * 64), b->num_sms, cs);
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && rc == EBIC_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc != EBIC_OK) return fail_free(rc);
  if (e != cudaSuccess) return fail_free(cerr(e, "batch graph capture"));
  *out = b;
  return EBIC_OK;
}

int ebic_batch_run(ebic_batch* b, const ebic_eval_request* reqs, uint32_t n_req, void* stream) {
  if (!b) return set_last_error(EBIC_ERR_INVALID_ARG, "batch is NULL");
  if (n_req > b->n_max) return set_last_error(EBIC_ERR_INVALID_ARG, "more requests than capacity");
  if (n_req > 0 && !reqs) return set_last_error(EBIC_ERR_INVALID_ARG, "reqs is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  HostPlan hp;
  if (n_req > 0) {
    int rc = build_plan(reqs, n_req, kStageMax, &hp);
    if (rc != EBIC_OK) return rc;
    if (hp.device != b->device)
      return set_last_error(EBIC_ERR_INVALID_ARG, "requests on another device than the batch");
    const int64_t cc = std::min<int64_t>(
        kMaxChunkCols, (kSmemDynMax - 2 * (int64_t)kStageMax - 2 * (kChunkSlack + 1) - 256) / 4);
    for (auto& q : hp.reqs) q.chunk_cols = std::min<int32_t>(q.chunk_cols, (int32_t)(cc / 64 * 64));
  }
  // the pinned block and the fitness scratch are used by the previous replay until it ends
  if (b->pending) B_CUDA(cudaEventSynchronize(b->done));
  b->pending = false;
  if (hp.fit_bytes > b->fbytes) {
    if (b->fmem) B_CUDA(cudaFree(b->fmem));
    b->fmem = nullptr;
    b->fbytes = 0;
    B_CUDA(cudaMalloc(&b->fmem, hp.fit_bytes));
    b->fbytes = hp.fit_bytes;
  }
  fill_header(hp, n_req, b->h.hdr);
  if (hp.fit_bytes) place_fitness(&hp, b->fmem, &b->h.hdr->zero, &b->h.hdr->n_zero);
  if (n_req > 0) {
    std::memcpy(b->h.reqs, hp.reqs.data(), sizeof(BatchReq) * n_req);
    std::memcpy(b->h.tmaps, hp.tmaps.data(), sizeof(CUtensorMap) * n_req);
    std::memcpy(b->h.ncols, hp.ncols.data(), 4 * (size_t)n_req);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  B_CUDA(cudaGraphLaunch(b->exec, s));
  B_CUDA(cudaEventRecord(b->done, s));
  b->pending = true;
  b->last_n = n_req;
  return EBIC_OK;
}

int ebic_batch_status(ebic_batch* b, uint32_t* req_status, uint32_t n, void* stream) {
  if (!b || (n > 0 && !req_status)) return set_last_error(EBIC_ERR_INVALID_ARG, "NULL argument");
  if (n > b->n_max) return set_last_error(EBIC_ERR_INVALID_ARG, "n exceeds capacity");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  B_CUDA(cudaStreamSynchronize(s));
  uint32_t err = 0;
  B_CUDA(cudaMemcpy(&err, b->d.err, 4, cudaMemcpyDeviceToHost));
  if (n) B_CUDA(cudaMemcpy(req_status, b->d.req_err, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  if (err & kErrTimeout)
    return set_last_error(EBIC_ERR_DEVICE_TIMEOUT, "a bounded device wait expired");
  for (uint32_t i = 0; i < n; ++i)
    if (req_status[i]) return set_last_error(EBIC_ERR_INVALID_ARG, "a request failed its check");
  return EBIC_OK;
}

int ebic_batch_free(ebic_batch* b) {
  if (!b) return EBIC_OK;
  if (b->pending) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fmem) cudaFree(b->fmem);
  cudaFree(b->dmem);
  cudaFreeHost(b->hmem);
  delete b;
  return EBIC_OK;
}

}  // extern "C"
