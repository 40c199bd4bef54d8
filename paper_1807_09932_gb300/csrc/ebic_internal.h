// Internal declarations of the EBIC GB300 library (not part of the public ABI).
//
// Rank-matrix layout in HBM (built once per matrix by the rank transform):
//   Ranks are dense per-row ranks, stored in WIDTH = 8 bits (cols <= 127) or 16 bits. A 32-bit
//   "lane word" packs 32/WIDTH rows of one column: byte/half k of the word of lane l in row
//   group g holds row g*RPG + 32*k + l, where RPG = 32 * (32/WIDTH) rows per group (128 or 64).
//   VEC consecutive groups form a slab. The matrix is stored column-major over slabs:
//       word(c, q, l, j) = ((c * Q + q) * 32 + l) * VEC + j,   group g = q * VEC + j
//   so that one 16-byte load per lane (VEC = 4) fetches four groups of one column, and a 3-D
//   TMA box {32*VEC words, TS slabs, columns} lands in shared memory column-major with the TS
//   slabs of one column contiguous.
//   Stored codes: 0 marks a missing value (and every padding row past the end); a real value is
//   stored as its dense rank + 1, in 1..cols. Since cols <= 127 (8-bit) or <= 32767 (16-bit), the
//   top bit of every field is always 0, which the SWAR compare in the evaluator relies on.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace ebic {

constexpr int kMaxCols = 832;
constexpr int kMaxLen = 64;
// The host and the device generation loops draw at most this many random columns when looking
// for one not in a candidate, then take the smallest unused one (the same bound on both sides).
constexpr uint32_t kUnusedDraws = 1u << 16;
constexpr int kSmemLimit = 232448;            // 227 KB shared memory per CTA (static + dynamic)
constexpr int kSmemDynMax = kSmemLimit - 2048;  // dynamic part: room for the kernels' static smem
constexpr int kStageMax = 104 * 1024;         // per pipeline stage (two stages)
constexpr int kMaxChunkCols = 16384;
constexpr int kChunkSlack = 72;  // spare column slots past a chunk (candidate tail + prefetch)

// error bits written by kernels into the per-call error word and the matrix status word
constexpr uint32_t kErrInvalid = 1u;
constexpr uint32_t kErrTimeout = 2u;

struct Layout {
  int32_t width = 8;         // bits per stored rank: 8 or 16
  int32_t vec = 4;           // groups per slab: 4, 2 or 1
  int32_t rows_per_group = 128;
  int32_t words_per_group = 4;  // bitmap words produced by one group
  int64_t rows = 0;
  int32_t cols = 0;
  int64_t groups = 0;        // ceil(rows / rows_per_group), padded up to a whole slab
  int64_t slabs = 0;         // Q
  int64_t words = 0;         // W = ceil(rows / 32)
  size_t rank_words() const { return (size_t)cols * (size_t)slabs * 32u * (size_t)vec; }
  int64_t rows_per_slab() const { return (int64_t)rows_per_group * vec; }
  int64_t words_per_slab() const { return (int64_t)words_per_group * vec; }
  size_t slab_col_bytes() const { return 128u * (size_t)vec; }  // one column of one slab
};

// Diagnostics: every kernel launch of the library is counted (defined in capi.cpp).
void count_launch();
void count_launches(int64_t n);  // n kernels at once (a negative n takes back counted ones)

// Choose width and VEC for a column count (host).
Layout make_layout(int64_t rows, int32_t cols);

// ---- rank transform ------------------------------------------------------------------------
// `num_sms`: the device's SM count (the ranking grid of rows up to 64 columns); `status`: a
// device word that receives kErrTimeout if a bounded wait of the transform expired.
cudaError_t launch_rank_transform(const Layout& L, const float* dX, int64_t ld, int exclude,
                                  float fill, uint32_t* ranks, uint32_t* status, int num_sms,
                                  cudaStream_t s);

// ---- population preparation (device-side argument checks, zeroing) ----------------------------
// One launch checks up to two CSR candidate lists (n[l] == 0 skips list l) against ncols and
// zeroes zero[0 .. n_zero). A failed check ORs kErrInvalid into *err and *status.
struct PrepareArgs {
  const uint16_t* cols[2] = {nullptr, nullptr};
  const uint32_t* offsets[2] = {nullptr, nullptr};
  uint32_t n[2] = {0, 0};
  int32_t ncols = 0;
  uint32_t* zero = nullptr;
  size_t n_zero = 0;
  uint32_t* zero2 = nullptr;
  size_t n_zero2 = 0;
  uint32_t* err = nullptr;
  uint32_t* status = nullptr;
  // pair-table term lists of list 0 (see kTermSlots), built when terms is not null
  uint32_t* terms = nullptr;
  uint32_t n_terms_cand = 0;  // candidates of list 0 to build them for
  int32_t pair_cols = 0;      // C of the pair table
  uint32_t pair_stride = 0;   // its row stride (words)
  bool negative = false;
};
cudaError_t launch_prepare(const PrepareArgs& a, cudaStream_t s);

// ---- population evaluator ------------------------------------------------------------------
struct EvalArgs {
  int32_t cols = 0;          // matrix columns
  int64_t slabs = 0;         // Q
  int64_t groups = 0;        // groups incl. slab padding (Q * VEC)
  int64_t words = 0;         // W
  uint32_t n_cand = 0;
  const uint16_t* cand_cols = nullptr;     // device CSR
  const uint32_t* cand_offsets = nullptr;  // device CSR
  uint32_t* counts = nullptr;              // device, zeroed before the launch
  uint32_t* bitmaps = nullptr;             // device [n_cand][bitmap_stride] or null
  int64_t bitmap_stride = 0;               // words between candidates' bitmaps (>= W)
  int32_t chunk_cols = 0;    // CC: candidate columns staged per chunk
  int32_t col_box = 0;       // columns per TMA box
  int32_t n_col_boxes = 0;
  uint32_t stage_bytes = 0;  // bytes of one pipeline stage
  uint32_t smem_bytes = 0;   // dynamic shared memory of the launch
  const uint32_t* err = nullptr;  // per-call error word: non-zero -> do nothing
  uint32_t* err_out = nullptr;    // where a timeout is reported (per call)
  uint32_t* status = nullptr;     // matrix status word
  uint64_t timeout_ns = 1000000000ull;
};

struct EvalConfig {
  int width = 8, vec = 4, ts = 1;
  bool negative = false, bitmaps = true;
  int grid = 0;
};

// Tile choice and shared-memory plan for a matrix layout (host).
int default_tile_slabs(const Layout& L);
bool plan_eval(const Layout& L, int ts, uint32_t n_cand, int64_t total_cols_hint, int grid,
               EvalArgs* a, int32_t chunk_override = 0);

cudaError_t launch_eval(const EvalConfig& cfg, const CUtensorMap* tmap, const EvalArgs& a,
                        cudaStream_t s);
// one translation unit per rank layout (width, VEC)
cudaError_t launch_eval_w8v4(const EvalConfig&, const CUtensorMap*, const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_w16v4(const EvalConfig&, const CUtensorMap*, const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_w16v2(const EvalConfig&, const CUtensorMap*, const EvalArgs&, cudaStream_t);
cudaError_t launch_eval_w16v1(const EvalConfig&, const CUtensorMap*, const EvalArgs&, cudaStream_t);
// Ready every evaluator instantiation of a layout on the current device (shared-memory limit
// raised, code loaded).
cudaError_t ready_eval_w8v4();
cudaError_t ready_eval_w16v4();
cudaError_t ready_eval_w16v2();
cudaError_t ready_eval_w16v1();
// Load the list-check kernel's code on the current device.
cudaError_t ready_prepare();

// ---- pair-table evaluation (optionally with the archive overlaps fused in) -----------------
constexpr int kPairRangeWords = 512;  // table and padded archive row strides are multiples
constexpr int kPairMaxArch = 64;      // archive members the fused overlap pass takes
// Row stride (words) of the pair table and of padded archive bitmaps for W-word bitmaps.
// A pair table allocation ends with one row of kOnesWords all-ones words (after the C*C
// table rows): a lane of a chain step reads its first 16 bytes in place of a segment whose
// words it has already zeroed.
constexpr int kOnesWords = 128;
__host__ __device__ inline const uint32_t* pair_ones(const uint32_t* table, uint64_t cols,
                                                    uint64_t stride) {
  return table + cols * cols * stride;
}
inline int64_t pair_stride(int64_t words) {
  return (words + kPairRangeWords - 1) / kPairRangeWords * kPairRangeWords;
}
// A candidate's term list, written by the preparation kernels: [kTermSlots] uint32 words per
// candidate, slot t < L-1 the table-row offset (words) of its consecutive pair t (the diagonal
// row for L = 1), slot 63 the length L; with negative trends slots 64 + t hold the reversed
// pairs' rows. Unused slots are 0.
constexpr int kTermSlots = 64;
__host__ __device__ inline int term_slots(bool negative) {
  return negative ? 2 * kTermSlots : kTermSlots;
}
struct PairArgs {
  const uint32_t* table = nullptr;   // [C*C][stride], padding words zero
  uint32_t stride = 0;               // row stride of table and arch (words)
  int32_t C = 0;                     // matrix columns
  int64_t W = 0;                     // words per bitmap
  const uint32_t* terms = nullptr;   // [n_cand][term_slots(negative)] term lists
  uint32_t n_cand = 0;
  uint32_t* counts = nullptr;        // [n_cand], zeroed before the launch
  uint32_t* bitmaps = nullptr;       // [n_cand][W] or null
  // fused overlaps: null arch = evaluation only
  const uint32_t* arch = nullptr;    // [n_arch rounded up to even][stride], padding words zero
  uint32_t n_arch = 0;               // <= kPairMaxArch
  const uint64_t* score = nullptr;   // per candidate: members whose overlap is needed; null: all
  uint32_t* overlaps = nullptr;      // [n_cand][ov_stride], zeroed before the launch
  uint32_t ov_stride = 0;            // n_arch rounded up to even (pairs of counters, 8-byte aligned)
  uint32_t* arch_counts = nullptr;   // [n_arch], zeroed before the launch
  const uint32_t* err = nullptr;     // non-zero: do nothing (when flags is null)
  const uint32_t* flags = nullptr;   // else: the preparation's block flags; any non-zero: do
  uint32_t n_flags = 0;              // nothing, and CTA 0 stores their OR in *err_out
  uint32_t* err_out = nullptr;       // the call's error word
  uint32_t* status = nullptr;        // matrix status word
  uint64_t timeout_ns = 1000000000ull;  // limit of each wait for staged table rows
};
// pdl: launch with programmatic stream serialization (the kernel waits for the previous one in
// the stream itself, so its launch overlaps that kernel's tail).
cudaError_t launch_pair_eval(const PairArgs& p, bool negative, int grid, bool pdl,
                             cudaStream_t s);

// Preparation of the fused pass, one launch: checks the candidate list and (check_arch) the
// archive list, zeroes counts, overlaps and archive counts, writes for every candidate the mask
// of archive members sharing a column with it, and copies the archive bitmaps (row stride W)
// into rows of `stride` words with zero padding. A failed check ORs kErrInvalid into *err and
// *status.
struct FusedPrepareArgs {
  const uint16_t* cols = nullptr;
  const uint32_t* offsets = nullptr;
  uint32_t n_cand = 0;
  const uint16_t* acols = nullptr;
  const uint32_t* aoffsets = nullptr;
  uint32_t n_arch = 0;               // <= kPairMaxArch
  bool check_arch = true;
  int32_t ncols = 0;
  int64_t W = 0;
  uint32_t stride = 0;
  const uint32_t* arch_src = nullptr;  // [n_arch][W]
  uint32_t* arch_pad = nullptr;        // [n_arch rounded up to even][stride]
  uint32_t* counts = nullptr;
  uint32_t* overlaps = nullptr;        // [n_cand][ov_stride]
  uint32_t ov_stride = 0;
  uint32_t* arch_counts = nullptr;
  uint64_t* share = nullptr;
  uint32_t* terms = nullptr;           // [n_cand][term_slots(negative)]
  bool negative = false;
  uint32_t* flags = nullptr;           // [blocks]: each block stores kErrInvalid or 0
  uint32_t* status_cand = nullptr;     // ORed with kErrInvalid when the candidate list fails
  uint32_t* status_arch = nullptr;     // ... when the archive list fails (null: not reported)
  // the pair table (or null): each candidate's first chain step in the first two row ranges is
  // prefetched into L2 for the pass's first wave
  const uint32_t* table = nullptr;
};
// Blocks of the fused preparation launch (and so the number of its flags).
uint32_t fused_prepare_blocks(uint32_t n_cand, uint32_t n_arch, uint32_t stride, int num_sms);
cudaError_t launch_fused_prepare(const FusedPrepareArgs& a, uint32_t blocks, cudaStream_t s);
// F_c from counts, overlaps and the share masks of the fused preparation. counts_out (or null)
// receives a copy of the counts and err_out (or null) of the call's error word: both may be
// pinned host memory, written by the kernel directly.
cudaError_t launch_fused_finalize(const uint32_t* offsets, uint32_t n_cand, const uint32_t* counts,
                                  const uint32_t* arch_offsets, uint32_t n_arch,
                                  const uint32_t* overlaps, uint32_t ov_stride,
                                  const uint32_t* arch_counts, const uint64_t* share,
                                  uint64_t* fitness, const uint32_t* err, uint32_t* counts_out,
                                  uint32_t* err_out, bool pdl, cudaStream_t s);

// Launch `kernel` with or without programmatic stream serialization.
template <typename... Params, typename... Args>
cudaError_t launch_maybe_pdl(bool pdl, void (*kernel)(Params...), dim3 grid, dim3 block,
                             size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- fitness -------------------------------------------------------------------------------
cudaError_t launch_overlap(const uint32_t* bitmaps, uint32_t n_cand, const uint32_t* arch_bitmaps,
                           uint32_t n_arch, int64_t words, uint32_t* overlaps,
                           uint32_t* arch_counts, const uint32_t* err, int num_sms,
                           cudaStream_t s);
cudaError_t launch_fitness_finalize(const uint16_t* cols, const uint32_t* offsets, uint32_t n_cand,
                                    const uint32_t* counts, const uint16_t* arch_cols,
                                    const uint32_t* arch_offsets, uint32_t n_arch,
                                    const uint32_t* overlaps, const uint32_t* arch_counts,
                                    uint64_t* fitness, const uint32_t* err, cudaStream_t s);

// Row gather for the host GA: dst row k = a's row idx[k] when idx[k] >= 0, else b's row
// -idx[k]-1 (rows of W words; idx in device memory). One launch instead of a copy per row.
cudaError_t launch_gather_rows(const uint32_t* a, const uint32_t* b, const int32_t* idx,
                               uint32_t n, int64_t W, uint32_t* dst, cudaStream_t s);

// ---- host helpers shared by the C-ABI translation units ------------------------------------
}  // namespace ebic

struct ebic_matrix;
struct ebic_params;
struct ebic_result;

namespace ebic {

struct MatrixView {
  int device = 0;
  Layout L;
  uint32_t* status = nullptr;
  int num_sms = 0;
  const uint32_t* pairs = nullptr;  // the matrix's pair table, or null
  uint32_t pair_stride = 0;
  int64_t row_offset = 0;           // a row shard's first row in the whole matrix
  int64_t total_rows = 0;           // the whole matrix's rows (L.rows when not a shard)
};
// Read-only view of a matrix handle's shape and device words.
void matrix_view(const ebic_matrix* m, MatrixView* v);
// Tile choice, launch plan and tensor map for evaluating n_cand candidates on m (the same choice
// ebic_eval_population makes). Returns EBIC_OK or an error code with the last-error message set.
int matrix_eval_plan(const ebic_matrix* m, uint32_t n_cand, int64_t total_cols_hint,
                     EvalArgs* a, EvalConfig* cfg, const CUtensorMap** tmap, int ts_cap = 0);
// Record the calling thread's last-error message and return `code`.
int set_last_error(int code, const char* msg);

// The generation loop on the device (ga_device.cu), from the host loop's initial population:
// init_cols [population][kMaxLen] (a candidate's columns first), init_n its lengths, init_h its
// hashes. The archive is at most 32 members.
int run_ga_on_device(const ebic_matrix* m, int64_t rows, int32_t ncols, int64_t W,
                     const ebic_params& p, cudaStream_t s, const uint16_t* init_cols,
                     const uint32_t* init_n, const uint64_t* init_h, ebic_result** out);
// Host-side check of a CSR candidate list; empty string when valid.
const char* check_candidates_host_c(const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                                    int32_t ncols);

}  // namespace ebic
