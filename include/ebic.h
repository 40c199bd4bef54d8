/*
 * ebic.h -- C ABI of the GB300 EBIC population evaluator.
 *
 * EBIC (arXiv 1807.09932) is an evolutionary biclustering method. Each generation it scores a
 * population of candidate biclusters against every row of a float32 matrix. A candidate is an
 * ordered list of distinct column indices. A row joins the candidate when its values obey the
 * "greater or equal" relation along that column order, and a candidate's score counts its rows
 * (Methods, "Handling missing values"). This library evaluates that rule on one GPU
 * (sm_103a).
 *
 * Conventions that hold for every call:
 *  - Pointer placement is detected per pointer (cudaPointerGetAttributes). Any input or output
 *    may be host memory (pageable or pinned) or device memory of the current device. Host
 *    inputs are copied to device scratch that the library allocates stream-ordered and frees on
 *    the same stream.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). A call whose outputs are
 *    all in device memory is asynchronous on that stream. A call with any host output
 *    synchronizes the stream before it returns.
 *  - The caller owns every buffer it passes. The library owns only ebic_matrix handles and its
 *    internal scratch.
 *  - Return values are EBIC_OK (0) or a negative EBIC_ERR_* code. No exception crosses the ABI.
 *    ebic_last_error() returns a message for the calling thread's last failure.
 *  - Arguments are checked before any launch. Candidate lists in host memory are checked on
 *    the host. Candidate lists already in device memory are checked by a device kernel, which
 *    makes every later kernel of the call do nothing. The failure is then reported by the
 *    call's return code when the call synchronizes (host outputs), else by
 *    ebic_matrix_status().
 *  - Calls on distinct streams may run concurrently, including on the same matrix.
 *
 * Bitmap layout: one bitmap per candidate of W = ceil(rows/32) little-endian uint32 words. Bit b
 * of word w is row 32w+b. Padding bits of the last word are 0. A population's bitmaps are
 * row-major [n_cand][W].
 *
 * Candidate lists are in CSR form. cols holds uint16 column indices. offsets[n_cand+1] holds
 * uint32 offsets with offsets[0] == 0. Candidate i is cols[offsets[i] .. offsets[i+1]). Its
 * length L is in [1, 64] and its columns are distinct and < the matrix's column count.
 */
#ifndef EBIC_GB300_H
#define EBIC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define EBIC_OK                  0
#define EBIC_ERR_INVALID_ARG    -1  /* a size, pointer, flag or candidate list is invalid      */
#define EBIC_ERR_OOM            -2  /* device or host allocation failed                        */
#define EBIC_ERR_CUDA           -3  /* a CUDA runtime call failed (message has the CUDA error)   */
#define EBIC_ERR_DEVICE_TIMEOUT -4  /* a bounded device wait expired; the kernel returned early  */
#define EBIC_ERR_UNSUPPORTED    -5  /* valid but outside this build's limits (e.g. too many cols)*/
#define EBIC_ERR_NO_DEVICE      -6  /* no CUDA device is visible                                 */

/* ---- ebic_load_matrix flags ------------------------------------------------------------- */
/* Missing-value exclusion (Methods, "Handling missing values"). NaN marks a missing value. With
 * the flag, a row with NaN in any column of a candidate does not match that candidate. Without
 * it, NaN is replaced by fill_value and compared as a number (the old behaviour). */
#define EBIC_EXCLUDE_MISSING 0x1u

/* ---- ebic_eval_population / ebic_fitness flags ------------------------------------------- */
/* Negative trends: a row that is non-increasing along the candidate's order also matches. A row
 * that is both non-decreasing and non-increasing (constant) is counted once. */
#define EBIC_NEGATIVE_TRENDS 0x1u
/* Evaluate with the rank-code evaluator even when the matrix has a pair table (speed only). */
#define EBIC_EVAL_DIRECT 0x2u

/* Largest supported column count of this build. Rows are limited to 2^31 - 1, the paper's
 * per-GPU row limit (Methods, "Support for Big Data"). */
#define EBIC_MAX_COLS 832
#define EBIC_MAX_CANDIDATE_LEN 64

typedef struct ebic_matrix ebic_matrix;

/*
 * Load a float32 matrix and build its device-resident rank matrix (one pass).
 *   x          row-major float32 values, rows x cols, leading dimension ld >= cols (elements);
 *              host or device memory. The library does not keep x.
 *   rows       1 .. 2^31-1 (Methods, "Support for Big Data": up to 2^31-1 rows on one GPU)
 *   cols       1 .. EBIC_MAX_COLS
 *   flags      EBIC_EXCLUDE_MISSING or 0
 *   fill_value the number that replaces NaN when exclusion is off. It must not be NaN.
 *   out        receives the handle; free it with ebic_free_matrix.
 * The rank transform replaces each value by its dense rank within its row (the number of
 * distinct non-missing values of the row strictly below it). So x <= y exactly when
 * rank(x) <= rank(y), which keeps the "greater or equal" relation of Methods, "Handling missing
 * values" intact. IEEE semantics: -0 == +0, infinities ordered, subnormals exact.
 * The call returns after the rank matrix is built (the stream is synchronized).
 */
int ebic_load_matrix(const float* x, int64_t rows, int32_t cols, int64_t ld, uint32_t flags,
                     float fill_value, void* stream, ebic_matrix** out);

/* Free a matrix handle and its device memory. Synchronizes the device. NULL is a no-op. */
int ebic_free_matrix(ebic_matrix* m);

/*
 * Shape of a loaded matrix. Any output pointer may be NULL.
 *   words      W = ceil(rows/32), the bitmap length per candidate
 *   rank_bits  8 (cols <= 127) or 16: the width of the stored ranks
 */
int ebic_matrix_info(const ebic_matrix* m, int64_t* rows, int32_t* cols, int64_t* words,
                     int32_t* rank_bits);

/*
 * Copy the dense ranks out, row-major uint16 [rows][cols], 0xFFFF for a missing value
 * (exclusion on). out is host memory of rows*cols uint16. Synchronous. This call exists to check
 * the transform; the evaluator never needs it.
 */
int ebic_matrix_ranks(const ebic_matrix* m, uint16_t* out, void* stream);

/*
 * Score a population against every row (the hot path of each EBIC generation; "search is
 * driven by counting of rows", Methods, "Handling missing values").
 *   cols, offsets  the population in CSR form (see above); n_cand >= 0 (0 is a no-op)
 *   flags          EBIC_NEGATIVE_TRENDS or 0
 *   counts         out: uint32[n_cand], the matched-row count of each candidate
 *   bitmaps        out: uint32[n_cand][W] row bitmaps, or NULL for counts only
 * Results are exact integers. They do not depend on the launch configuration.
 */
int ebic_eval_population(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                         uint32_t n_cand, uint32_t flags, uint32_t* counts, uint32_t* bitmaps,
                         void* stream);

/*
 * Allocation-free variant of ebic_eval_population, for callers that cannot allocate device
 * memory while they evaluate: a serving loop that must not take the allocator's lock or meet an
 * out-of-memory error mid-request, or a process whose device memory is already owned by another
 * framework's caching allocator. It has no counterpart in the paper; it computes exactly what
 * ebic_eval_population computes, with the same kernels.
 *   counts, bitmaps   must be device memory of the matrix's device (no staging buffer exists).
 *   cols, offsets     device memory (used in place, checked by a device kernel), or host memory
 *                     (checked on the host and copied into the library's fixed scratch; the
 *                     offsets rounded up to 256 bytes plus the columns must fit in 1 MiB minus
 *                     256 bytes, otherwise EBIC_ERR_UNSUPPORTED). Both in the same placement.
 *   Memory of another device, for any of the four, returns EBIC_ERR_INVALID_ARG.
 * Scratch: a fixed 1 MiB device array inside the library (held by every GPU that loads the
 * library until exit). The library calls no allocation or free routine on this path. The first
 * call on each device looks up that array's device address and loads the code of every kernel
 * variant this call can launch on that device (under CUDA's lazy module loading, loading code is
 * the one step in which the CUDA runtime itself reserves device memory); later calls load
 * nothing. Make that first call before any stream capture. All calls share the array and its
 * previous contents: the call clears its status word itself, and calls that overlap on the GPU
 * race on the array, so issue one at a time.
 * With device-resident lists the call is asynchronous on `stream`. Host-resident lists are
 * copied with cudaMemcpyAsync: from pageable memory that copy has consumed the host buffer when
 * the call returns; from pinned memory it is asynchronous, and the buffer must stay unchanged
 * until the stream has run the call. Device-side check failures are reported by
 * ebic_matrix_status().
 */
int ebic_eval_population_noalloc(const ebic_matrix* m, const uint16_t* cols,
                                 const uint32_t* offsets, uint32_t n_cand, uint32_t flags,
                                 uint32_t* counts, uint32_t* bitmaps, void* stream);

/*
 * Overlap-penalised fitness of a population against an elite archive. This is the project's
 * reading of the paper's "driven by counting of rows" (Methods, "Handling missing values").
 *   cols, offsets, n_cand  the population (CSR), as given to ebic_eval_population
 *   counts, bitmaps        its evaluation: uint32[n_cand] and uint32[n_cand][W]
 *   arch_cols, arch_offsets, arch_bitmaps, n_arch   the archive: CSR column lists and
 *                          uint32[n_arch][W] row bitmaps. n_arch may be 0 (pointers then unused).
 *   fitness                out: uint64[n_cand]
 *   overlaps               out: uint32[n_cand][n_arch] = popcount(M_c & M_a), or NULL
 * Definition: q(x) = (uint64)n_x << (min(L_x, 33) - 1) is the raw quality (n_a of an archive
 * member is the popcount of its bitmap) and o(c,a) = popcount(M_c & M_a). Let p_c = counts[c]
 * minus the largest o(c,a) over archive members a whose column SET meets c's and with
 * q(a) >= q(c) (0 if there is none). Then fitness[c] = (uint64)p_c << (min(L_c, 33) - 1).
 * Only members at least as good as the candidate penalise it, so improving on an archived
 * bicluster is not penalised.
 * flags is reserved (pass 0).
 */
int ebic_fitness(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                 uint32_t n_cand, const uint32_t* counts, const uint32_t* bitmaps,
                 const uint16_t* arch_cols, const uint32_t* arch_offsets,
                 const uint32_t* arch_bitmaps, uint32_t n_arch, uint32_t flags,
                 uint64_t* fitness, uint32_t* overlaps, void* stream);

/*
 * One generation's scoring in one call: ebic_eval_population followed by ebic_fitness, with
 * the same results (arXiv 1807.09932, Methods: the population is evaluated by counting rows,
 * "Handling missing values"; the fitness as defined for ebic_fitness above).
 *   cols, offsets, n_cand, flags   the population and flags, as for ebic_eval_population
 *   arch_cols, arch_offsets, arch_bitmaps, n_arch   the archive, as for ebic_fitness
 *   counts     out: uint32[n_cand] matched rows
 *   bitmaps    out: uint32[n_cand][W] row bitmaps, or NULL when the caller needs none
 *   fitness    out: uint64[n_cand]
 *   overlaps   out: uint32[n_cand][n_arch], or NULL. When NULL, the overlap of a candidate with
 *              a member that shares no column with it is not computed (it cannot change F_c).
 * When the matrix has a pair table, EBIC_EVAL_DIRECT is not given and n_arch <= 64, the call
 * runs as one preparation launch, one pass that evaluates the population and ANDs its words
 * with the archive's while they are in registers (the bitmaps never round-trip through device
 * memory), and one finalize launch. Otherwise it makes the two calls in sequence (with the
 * bitmaps in stream-ordered scratch when `bitmaps` is NULL). Buffers may be host or device memory
 * as for the two calls; a candidate list keeps its columns and offsets in the same memory.
 * Errors as for the two calls.
 */
int ebic_eval_fitness(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                      uint32_t n_cand, uint32_t flags, const uint16_t* arch_cols,
                      const uint32_t* arch_offsets, const uint32_t* arch_bitmaps,
                      uint32_t n_arch, uint32_t* counts, uint32_t* bitmaps, uint64_t* fitness,
                      uint32_t* overlaps, void* stream);

/*
 * Synchronize `stream` and return the deferred device status of `m`, then clear it. That
 * status is EBIC_OK, EBIC_ERR_INVALID_ARG (a device-resident candidate list failed the device
 * check) or EBIC_ERR_DEVICE_TIMEOUT (a bounded wait in a kernel expired). The status is shared by
 * all streams that use `m`.
 */
int ebic_matrix_status(ebic_matrix* m, void* stream);

/*
 * ---- Row shards: one matrix spread over several GPUs by rows ----
 * The paper's multi-GPU support (Abstract; Methods, "Support for Big Data"; Results, Fig. 1
 * and Table 1: rows of one matrix spread over up to 8 GPUs) rests on rows being independent:
 * a candidate's row count and its overlaps with archive members are sums over row ranges, and
 * its bitmap is the concatenation of the ranges' bitmaps. Only the fitness needs the whole sums.
 * So a sharded generation is: on every shard ebic_eval_partials; one sum over the shards of
 * counts [n_cand], overlaps [n_cand][n_arch] and arch_counts [n_arch] (an all-reduce, all uint32:
 * a sum is at most the total row count); then ebic_fitness_reduced on the sums. The fitness
 * equals ebic_eval_fitness's on the whole matrix.
 */

/*
 * Load rows [row_offset, row_offset + rows) of a matrix of total_rows rows; x points to the
 * shard's first row (other arguments as for ebic_load_matrix). row_offset must be a multiple of
 * 32 and every shard but the last must hold a multiple of 32 rows, so that a shard's bitmap word
 * w is word row_offset / 32 + w of the whole matrix's bitmap. The shard is an ordinary matrix of
 * `rows` rows for every call (bitmaps, archive bitmaps and counts are the shard's own), except
 * ebic_run, which returns EBIC_ERR_UNSUPPORTED on a shard that is not the whole matrix.
 * Errors: EBIC_ERR_INVALID_ARG for an offset or size outside those rules.
 */
int ebic_load_matrix_shard(const float* x, int64_t rows, int32_t cols, int64_t ld,
                           int64_t row_offset, int64_t total_rows, uint32_t flags,
                           float fill_value, void* stream, ebic_matrix** out);

/* A matrix's place in the whole matrix: its first row, the whole matrix's rows and its first
 * bitmap word (0, rows, 0 for a matrix loaded by ebic_load_matrix). Any pointer may be NULL. */
int ebic_matrix_shard(const ebic_matrix* m, int64_t* row_offset, int64_t* total_rows,
                      int64_t* word_offset);

/*
 * One shard's share of a generation's scoring (Methods, "Handling missing values": the search
 * counts rows; the sums make the whole matrix's counts and overlaps).
 *   cols, offsets, n_cand, flags  the population and flags, as for ebic_eval_population
 *   arch_cols, arch_offsets, n_arch  the archive's column lists (the whole archive, every shard)
 *   arch_bitmaps    uint32[n_arch][W]: the archive members' bitmaps over THIS shard's rows
 *   counts          out: uint32[n_cand], the shard's matched rows per candidate
 *   overlaps        out: uint32[n_cand][n_arch], the shard's popcount(M_c & M_a) for every
 *                   member a that shares a column with c; entries of members sharing no column
 *                   are 0 or that popcount (ebic_fitness_reduced never reads them). Needed, and
 *                   arch_counts too, when n_arch > 0; otherwise unused.
 *   arch_counts     out: uint32[n_arch], the shard's popcount of each member's bitmap
 *   bitmaps         out: uint32[n_cand][W] over the shard's rows, or NULL
 * Buffers may be host or device memory, as for ebic_eval_fitness; with all outputs on the device
 * the call is asynchronous on `stream`.
 */
int ebic_eval_partials(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                       uint32_t n_cand, uint32_t flags, const uint16_t* arch_cols,
                       const uint32_t* arch_offsets, const uint32_t* arch_bitmaps,
                       uint32_t n_arch, uint32_t* counts, uint32_t* overlaps,
                       uint32_t* arch_counts, uint32_t* bitmaps, void* stream);

/*
 * The fitness of ebic_fitness from whole-matrix counts, overlaps and archive counts (the sums
 * of every shard's ebic_eval_partials outputs), with no bitmap: q(x) = n_x << (min(L_x,33)-1),
 * p_c = counts[c] - the largest overlaps[c][a] over members a that share a column with c and
 * have q(a) >= q(c) (0 if none), fitness[c] = p_c << (min(L_c,33)-1).
 *   m               any shard of the matrix (it gives the device and the column count)
 *   counts          uint32[n_cand]; overlaps uint32[n_cand][n_arch]; arch_counts uint32[n_arch]
 *   fitness         out: uint64[n_cand]
 * flags is reserved (pass 0). Host or device buffers; asynchronous when fitness is on the device.
 */
int ebic_fitness_reduced(const ebic_matrix* m, const uint16_t* cols, const uint32_t* offsets,
                         uint32_t n_cand, const uint32_t* counts, const uint32_t* overlaps,
                         const uint16_t* arch_cols, const uint32_t* arch_offsets,
                         const uint32_t* arch_counts, uint32_t n_arch, uint32_t flags,
                         uint64_t* fitness, void* stream);

/*
 * Row-tile height of the evaluator for this matrix, in slabs (1, 2 or 4), or 0 for the
 * built-in choice. A slab is 512 rows for 8-bit ranks and 256, 128 or 64 rows for 16-bit ranks
 * (ebic_matrix_get_tile reports it). The tile changes speed only, never results. The autotuner
 * sets it from timed sweeps. A tile whose shared-memory stage would not fit returns
 * EBIC_ERR_UNSUPPORTED. Not thread-safe with concurrent evaluations of the same matrix.
 */
int ebic_matrix_set_tile(ebic_matrix* m, int32_t tile_slabs);
/*
 * Pair table: an exact alternative encoding of the same rule, for populations scored many times
 * on one matrix. For every ordered column pair (a, b) the table holds the bitmap of rows where a
 * is not missing and b's value is >= a's; the diagonal holds "a not missing". A candidate's
 * bitmap is then the AND of its consecutive pairs' rows (the reversed pairs for decreasing
 * trends), one 32-bit AND per 32 rows per column, instead of a compare per row per column.
 * The table takes cols * cols * W' * 4 + 512 bytes of device memory, W' = W rounded up to a
 * multiple of 512 (its rows are padded with zero words; one all-ones row of 128 words follows
 * them), and is built once, by the evaluator itself (on the population of all pairs), so results
 * never change.
 *   ebic_matrix_build_pairs: build it if it needs at most max_bytes (else EBIC_ERR_UNSUPPORTED);
 *                            *bytes (may be NULL) receives the size. Synchronous.
 *   ebic_matrix_drop_pairs:  free it.
 * While a matrix has a table, ebic_eval_population and ebic_eval_fitness use it unless
 * EBIC_EVAL_DIRECT is given.
 * ebic_eval_population_noalloc always uses the rank-code evaluator; the batched calls use the
 * table for the requests on a matrix that has one.
 */
int ebic_matrix_build_pairs(ebic_matrix* m, uint64_t max_bytes, void* stream, uint64_t* bytes);
int ebic_matrix_drop_pairs(ebic_matrix* m);

/* Candidate columns staged per chunk (the candidate tile: each chunk of the population is
 * checked against each row tile), or 0 for the built-in choice. Rounded up to a multiple of 64
 * and capped by the shared memory left after the row-tile stages. Speed only, never results.
 * Values outside [0, 16384] return EBIC_ERR_INVALID_ARG. */
int ebic_matrix_set_chunk_cols(ebic_matrix* m, int32_t chunk_cols);
/* The tile height in slabs that the next evaluation will use, and the rows per slab. */
int ebic_matrix_get_tile(const ebic_matrix* m, int32_t* tile_slabs, int32_t* rows_per_slab);

/* ---- batched evaluation: many populations on many matrices in one launch ------------------ */
/*
 * One request = one population to score on one loaded matrix, as for ebic_eval_population,
 * except that every buffer must be device memory of the matrices' (common) device. Candidate lists
 * are checked on the device; a failed request produces zero counts and no bitmaps, its matrix's
 * status records EBIC_ERR_INVALID_ARG, and the others are unaffected.
 * Results are identical to scoring each request alone with ebic_eval_population.
 */
typedef struct ebic_eval_request {
  const ebic_matrix* m;
  const uint16_t* cols;      /* device CSR columns                                            */
  const uint32_t* offsets;   /* device CSR offsets [n_cand+1]                                 */
  uint32_t n_cand;
  uint32_t flags;            /* EBIC_NEGATIVE_TRENDS or 0                                     */
  uint32_t* counts;          /* device [n_cand]                                               */
  uint32_t* bitmaps;         /* device [n_cand][W], or NULL for counts only                   */
  /* Optional, for a matrix with a pair table (ebic_matrix_build_pairs): the overlap-penalised
   * fitness of ebic_fitness against an archive, with the overlaps computed inside the batched
   * pass (as ebic_eval_fitness does for one population). fitness NULL: none. */
  const uint16_t* arch_cols;     /* device CSR columns of the archive (n_arch > 0)           */
  const uint32_t* arch_offsets;  /* device [n_arch+1]                                         */
  const uint32_t* arch_bitmaps;  /* device [n_arch][W]                                        */
  uint32_t n_arch;               /* 0 .. 64                                                   */
  uint64_t* fitness;             /* device [n_cand], or NULL                                  */
} ebic_eval_request;

/* Score all requests in one persistent launch (plus a check and a plan kernel), asynchronously on
 * `stream`. Row tiles and candidate chunks of all requests share one dynamic work queue; requests
 * on matrices with a pair table run on the batched pair pass instead, and those with `fitness`
 * also get their archive overlaps there and their fitness from one more kernel. A request asking
 * for fitness on a matrix without a pair table is rejected (EBIC_ERR_UNSUPPORTED). Archive lists
 * are checked on the device like candidate lists. */
int ebic_eval_batch(const ebic_eval_request* reqs, uint32_t n_req, void* stream);

/* The same batched launch, captured once in a CUDA graph and replayed. A batch holds device and
 * pinned host buffers for up to max_requests requests; ebic_batch_run writes the requests into its
 * pinned block (waiting for the previous replay to finish reading it) and launches the graph on
 * `stream`. Any composition of up to max_requests requests replays the same graph. */
typedef struct ebic_batch ebic_batch;
int ebic_batch_create(uint32_t max_requests, ebic_batch** out);
int ebic_batch_run(ebic_batch* b, const ebic_eval_request* reqs, uint32_t n_req, void* stream);
/* Synchronize `stream`; req_status[i] (i < n) receives request i's check bits of the last run. */
int ebic_batch_status(ebic_batch* b, uint32_t* req_status, uint32_t n, void* stream);
int ebic_batch_free(ebic_batch* b);

/* ---- the EBIC generation loop (host genetic algorithm over the device evaluator) --------- */
/*
 * The paper says EBIC uses evolutionary computation over a population of up to 65,535
 * candidates, with 1,600 or fewer usually enough to converge (Methods, "Support for Big Data").
 * It does not define the operators. The ones here are the project's definition: deterministic
 * given `seed` (splitmix64 counter generators: one for the initial population, one per child
 * slot and generation), tournament selection, an order-preserving
 * crossover, four mutations (swap, substitute, insert, delete), a tabu list of evaluated column
 * sequences, and an elite archive of `archive_size` biclusters ranked by raw quality
 * n << (min(L,33)-1). A candidate enters the archive unless a member sharing a column overlaps
 * it by more than overlap_threshold x its row count without being strictly worse; strictly worse
 * members it overlaps that much are replaced by it.
 * Each generation the population is scored with ebic_eval_fitness against the current archive
 * (device-resident rank matrix, bitmaps and archive); when the matrix has a pair table
 * (ebic_matrix_build_pairs) that is one fused pass. Results do not depend on the table.
 * The children of a generation are bred by host threads (the environment variable
 * EBIC_HOST_THREADS, 1..64, sets their number; by default the cores, at most 16, with at least
 * 128 children each); results do not depend on their number either.
 */
typedef struct ebic_params {
  uint32_t population;       /* candidates per generation (default 1600)                      */
  uint32_t generations;      /* generations to run (default 100)                              */
  uint32_t archive_size;     /* elite archive size K (default 20)                             */
  uint32_t elite;            /* best candidates copied unchanged to the next generation (16)  */
  uint32_t tournament;       /* tournament size (default 4)                                   */
  uint32_t min_len;          /* shortest candidate (default 2)                                */
  uint32_t max_init_len;     /* longest initial candidate (default 6)                         */
  uint32_t max_len;          /* longest candidate (default 64, at most cols)                  */
  float p_crossover;         /* crossover probability (default 0.5)                           */
  float p_mutation;          /* mutation probability (default 0.7)                            */
  float overlap_threshold;   /* archive admission threshold (default 0.5)                     */
  uint32_t tabu_retries;     /* re-mutations of a tabu child before a random one (default 8)  */
  uint32_t flags;            /* EBIC_NEGATIVE_TRENDS, EBIC_RUN_ON_DEVICE, or 0               */
  uint32_t reserved;
  uint64_t seed;             /* default 1807099320                                            */
} ebic_params;
/* ebic_params.flags: the whole generation loop runs on the device (breeding, tabu list,
 * duplicate handling, archive update), with no host round trip per generation; the archive is
 * the same, bit for bit, as the host loop's. Takes archive_size <= 32 (else
 * EBIC_ERR_UNSUPPORTED); ebic_run only. */
#define EBIC_RUN_ON_DEVICE 0x2u

typedef struct ebic_result {
  uint32_t n;                /* archive members, best first                                   */
  uint16_t* cols;            /* CSR columns of the members                                    */
  uint32_t* offsets;         /* [n+1]                                                         */
  uint32_t* counts;          /* [n] matched rows                                              */
  uint64_t* quality;         /* [n] counts << (min(L,33)-1): the archive's order key          */
  uint32_t* bitmaps;         /* [n][W] row bitmaps (NULL from ebic_run_custom)               */
  int64_t words;             /* W                                                             */
  uint32_t generations_run;
  uint64_t candidates_evaluated;
} ebic_result;

/* Fill *p with the defaults listed above. */
int ebic_params_default(ebic_params* p);

/* Run EBIC on a loaded matrix; *out receives the archive (free it with ebic_free_result).
 * stream: the CUDA stream the generations run on. Synchronous. */
int ebic_run(const ebic_matrix* m, const ebic_params* p, void* stream, ebic_result** out);

/* The same generation loop over caller-supplied evaluation (host buffers throughout). It exists
 * so the loop can be driven by another implementation of the scoring (a CPU reference) and is
 * pure host code. Callbacks return 0 on success.
 *   evaluate:       counts[n], fitness[n] and overlaps[n][n_arch] of the population against the
 *                   current archive (as last set by set_archive; empty at first)
 *   pair_overlaps:  out[t][t] = popcount(M_i & M_j) for population indices idx[0..t)
 *   set_archive:    the new archive, member i = population candidate src[i] if src[i] >= 0,
 *                   else old archive member -(src[i]+1)
 */
typedef struct ebic_evaluator {
  void* user;
  int (*evaluate)(void* user, const uint16_t* cols, const uint32_t* offsets, uint32_t n,
                  uint32_t* counts, uint64_t* fitness, uint32_t* overlaps);
  int (*pair_overlaps)(void* user, const uint32_t* idx, uint32_t t, uint32_t* out);
  int (*set_archive)(void* user, const int32_t* src, uint32_t k);
} ebic_evaluator;
int ebic_run_custom(int64_t rows, int32_t cols, const ebic_params* p, const ebic_evaluator* ev,
                    ebic_result** out);

int ebic_free_result(ebic_result* r);

/* ---- text input and bicluster output ---------------------------------------------------- */
/*
 * A matrix read from a delimited text file (arXiv 1807.09932, Methods, "Different input file
 * formats support"): values separated by commas, tabs or semicolons; a header row of column
 * names and a first column of row names are optional; with both, the upper-left (corner) field
 * may be absent (R's write.table layout). Quotes around names are dropped.
 *   values      [rows][cols] row-major float32; missing values are NaN
 *   row_names   [rows] NUL-terminated strings, or NULL when the file has no row names
 *   col_names   [cols], or NULL when the file has no header row
 */
typedef struct ebic_text_matrix {
  float* values;
  int64_t rows;
  int32_t cols;
  char** row_names;
  char** col_names;
} ebic_text_matrix;

/*
 * Read `path`. delimiter: ',', '\t', ';' or 0 to take the one most frequent in the first line.
 * missing: a marker of missing values (Methods, "Handling missing values": "replaced with a
 * predefined value (e.g. 0 or 999)"), compared as a number when it parses as one, else as text;
 * or NULL. Empty fields and NA / NaN are missing too. Missing cells are NaN, so the evaluator's
 * EBIC_EXCLUDE_MISSING applies to them. A header row is recognised by a field that is neither a
 * number nor missing; a row-name column likewise in the first data row. Returns
 * EBIC_ERR_INVALID_ARG (message with the line and column) for a row with another number of
 * fields or a cell that is not a number. *out is freed with ebic_free_text_matrix.
 */
int ebic_read_matrix_text(const char* path, char delimiter, const char* missing,
                          ebic_text_matrix** out);
int ebic_free_text_matrix(ebic_text_matrix* m);

/*
 * Write the archive of an ebic_run result (Methods, "Compatibility with R and Bioconductor")
 * in the layout of the biclust package's bicluster result files: a title line, then for each
 * member a line "rows cols", a line of its row names and a line of its column names (in the
 * member's column order), separated by spaces. Names come from `names` (the matrix the run was
 * on, as read by ebic_read_matrix_text) or, where it has none or names is NULL, are 1-based
 * indices. The result must carry bitmaps (ebic_run's does).
 */
int ebic_write_biclusters(const char* path, const char* title, const ebic_result* r,
                          const ebic_text_matrix* names);

/* ---- staging ---------------------------------------------------------------------------- */
/* A copy of `bytes` bytes from src to dst, ordered on `stream` (cudaMemcpyDefault: either side
 * may be device memory, pinned host memory or pageable host memory). The paper has no
 * counterpart. A caller that packs many requests' lists into one buffer uses it to move them, or
 * the requests' outputs, in one copy without a framework's tensor calls. Pinned and device
 * buffers: asynchronous on `stream`, and both must stay valid until the stream reaches the
 * copy. Pageable host memory: the call returns once the host side has been read or written.
 * bytes == 0 does nothing. Returns EBIC_ERR_INVALID_ARG for a NULL buffer and EBIC_ERR_CUDA
 * when the runtime rejects the copy. */
int ebic_copy_async(void* dst, const void* src, size_t bytes, void* stream);

/* ---- diagnostics ----------------------------------------------------------------------- */
/* Kernels launched by this library in this process so far (every launch is counted). */
int64_t ebic_launch_count(void);

/* Per-kernel timing with CUDA events recorded on the stream of each launch, around the
 * library's own kernel launches. Kinds: */
#define EBIC_TIMING_RANK_TRANSFORM 0
#define EBIC_TIMING_PREPARE        1  /* device-side argument checks and output zeroing */
#define EBIC_TIMING_EVALUATE       2  /* the population evaluator */
#define EBIC_TIMING_OVERLAP        3  /* bitmap overlaps against the archive */
#define EBIC_TIMING_FITNESS        4  /* penalised fitness */
#define EBIC_TIMING_PAIR_EVALUATE  5  /* the pair-table evaluator */
#define EBIC_TIMING_KINDS          6
/* Enable (1) or disable (0) recording. Either way, the events recorded so far are dropped. */
int ebic_timing_enable(int on);
/* Wait for the recorded events of `kind` and return their summed duration and count. */
int ebic_timing_read(int kind, double* total_ms, int64_t* launches);

/* Self-test of the failure path of every bounded device wait: launch a kernel whose wait on an
 * mbarrier can never complete; after timeout_ns (<= 0.1 s) it records the expiry and returns.
 * Returns EBIC_ERR_DEVICE_TIMEOUT when the path works; the context stays usable. */
int ebic_selftest_wait_timeout(uint64_t timeout_ns, void* stream);

/* Message for the calling thread's last failed call ("" if none). Valid until the next call. */
const char* ebic_last_error(void);

/* ABI version: (major << 16) | minor. */
int ebic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EBIC_GB300_H */
