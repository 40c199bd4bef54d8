/*
 * EBIC population-evaluation ORACLE -- test infrastructure only.
 *
 * A plain, slow, obviously correct CPU restatement of what the EBIC hot path computes
 * (arXiv 1807.09932). Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library; the product (the CUDA library and its Python binding) never
 * does, and shares no code, header or table with it.
 *
 * It works on the raw float32 matrix with IEEE comparisons. It never builds ranks for the
 * evaluation; the dense-rank routine at the end exists only to check the GPU's rank transform.
 *
 * Rules followed (the paper states the first three; the rest are the project's readings):
 *  - a row follows a candidate (an ordered list of distinct columns c_1..c_L) when its values
 *    satisfy the "greater or equal" relation along that order: X[c_1] <= X[c_2] <= ... <= X[c_L]
 *    (Methods, "Handling missing values"); equal values follow;
 *  - the search counts rows (same passage): the score of a candidate is its matched-row count;
 *  - with missing-value exclusion on, a missing value (NaN) no longer counts towards the score:
 *    a row with NaN in any of the candidate's columns does not match (same passage);
 *    with exclusion off, NaN is replaced by the fill value and compared as a number;
 *  - negative-trend option: a row that is non-increasing along the order also matches, counted
 *    once;
 *  - bitmaps are LSB-first uint32 words, bit b of word w = row 32w+b, padding bits 0;
 *  - fitness: quality q(x) = n_x << (min(L_x,33) - 1); overlap o(c,a) = |rows(c) & rows(a)|;
 *    penalty = max o(c,a) over archive members a that share a column with c and are at least
 *    as good (q(a) >= q(c)), 0 if none; F = (n - penalty) << (min(L,33) - 1).
 *
 * Parity status: every function here is pinned by the CPU tests (brute force with sorted(),
 * closed-form match probabilities, invariants, planted recovery, scipy's dense rankdata,
 * set-based overlap counting). No function is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Returns 1 when row r (pointer to its first value) follows the candidate, else 0. */
static int row_matches(const float* row, const uint16_t* cand, uint32_t L, int exclude_missing,
                       float fill_value, int negative)
{
    float v[64];
    for (uint32_t i = 0; i < L; ++i) {
        float x = row[cand[i]];
        if (isnan(x)) {
            if (exclude_missing) return 0; /* a missing value removes the row from this candidate */
            x = fill_value;                /* old behaviour: the marker is compared as a number */
        }
        v[i] = x;
    }
    int asc = 1, desc = 1;
    for (uint32_t i = 0; i + 1 < L; ++i) {
        if (!(v[i] <= v[i + 1])) asc = 0;  /* "greater or equal" between consecutive columns */
        if (!(v[i] >= v[i + 1])) desc = 0; /* the reverse relation, for negative trends */
    }
    return asc || (negative && desc);
}

/*
 * Scores every candidate of a population against every row.
 *   X          row-major float32, R rows, C columns, leading dimension ld (>= C)
 *   cols       concatenated candidate columns (CSR), offsets[P+1] (offsets[0] = 0)
 *   counts     out, P uint32
 *   bitmaps    out, P*W uint32 (may be NULL)
 * Returns 0, or -1 for an invalid candidate (length 0 or > 64, column out of range, repeat).
 */
int oracle_eval(const float* X, int64_t R, int32_t C, int64_t ld, int exclude_missing,
                float fill_value, const uint16_t* cols, const uint32_t* offsets, uint32_t P,
                int negative, uint32_t* counts, uint32_t* bitmaps, int nthreads)
{
    const int64_t W = (R + 31) / 32;
    for (uint32_t p = 0; p < P; ++p) {
        uint32_t L = offsets[p + 1] - offsets[p];
        if (offsets[p + 1] < offsets[p] || L == 0 || L > 64) return -1;
        for (uint32_t i = 0; i < L; ++i) {
            if (cols[offsets[p] + i] >= (uint32_t)C) return -1;
            for (uint32_t j = 0; j < i; ++j)
                if (cols[offsets[p] + i] == cols[offsets[p] + j]) return -1;
        }
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < (int64_t)P; ++p) {
        const uint16_t* cand = cols + offsets[p];
        uint32_t L = offsets[p + 1] - offsets[p];
        uint32_t n = 0;
        uint32_t* bm = bitmaps ? bitmaps + p * W : NULL;
        if (bm) memset(bm, 0, (size_t)W * sizeof(uint32_t));
        for (int64_t r = 0; r < R; ++r) {
            int m = row_matches(X + r * ld, cand, L, exclude_missing, fill_value, negative);
            n += (uint32_t)m;
            if (m && bm) bm[r >> 5] |= 1u << (r & 31);
        }
        counts[p] = n;
    }
    return 0;
}

/* Number of columns two candidates have in common, as sets. */
static int share_columns(const uint16_t* a, uint32_t la, const uint16_t* b, uint32_t lb)
{
    for (uint32_t i = 0; i < la; ++i)
        for (uint32_t j = 0; j < lb; ++j)
            if (a[i] == b[j]) return 1;
    return 0;
}

static uint32_t popcount32(uint32_t x)
{
    uint32_t n = 0;
    while (x) { n += x & 1u; x >>= 1; }
    return n;
}

static uint64_t quality(uint32_t n, uint32_t L)
{
    uint32_t shift = (L < 33 ? L : 33) - 1;
    return (uint64_t)n << shift;
}

/*
 * Overlap-penalised fitness against an elite archive of K biclusters.
 *   counts[P], bitmaps[P*W]        the population's evaluation
 *   acols/aoffsets, abitmaps[K*W]   the archive's columns (CSR) and row bitmaps
 *   fitness   out, P uint64
 *   overlaps  out, P*K uint32 (may be NULL)
 */
int oracle_fitness(int64_t R, const uint16_t* cols, const uint32_t* offsets, uint32_t P,
                   const uint32_t* counts, const uint32_t* bitmaps, const uint16_t* acols,
                   const uint32_t* aoffsets, const uint32_t* abitmaps, uint32_t K,
                   uint64_t* fitness, uint32_t* overlaps, int nthreads)
{
    const int64_t W = (R + 31) / 32;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < (int64_t)P; ++p) {
        uint32_t L = offsets[p + 1] - offsets[p];
        uint64_t qc = quality(counts[p], L);
        uint32_t penalty = 0;
        for (uint32_t a = 0; a < K; ++a) {
            uint32_t o = 0, na = 0;
            for (int64_t w = 0; w < W; ++w) {
                o += popcount32(bitmaps[p * W + w] & abitmaps[(int64_t)a * W + w]);
                na += popcount32(abitmaps[(int64_t)a * W + w]);
            }
            if (overlaps) overlaps[p * K + a] = o;
            uint32_t La = aoffsets[a + 1] - aoffsets[a];
            int s = share_columns(cols + offsets[p], L, acols + aoffsets[a], La);
            int at_least_as_good = quality(na, La) >= qc;
            if (s && at_least_as_good && o > penalty) penalty = o;
        }
        fitness[p] = quality(counts[p] - penalty, L);
    }
    return 0;
}

/*
 * Dense per-row ranks, written out by definition: rank(x) = number of DISTINCT non-missing values
 * of the row that are strictly less than x. Missing (NaN with exclusion on) -> 0xFFFF. With
 * exclusion off, NaN is first replaced by fill_value. Output row-major R*C uint16.
 * Used only to check the GPU's rank transform; the evaluation above never uses ranks.
 */
void oracle_dense_ranks(const float* X, int64_t R, int32_t C, int64_t ld, int exclude_missing,
                        float fill_value, uint16_t* ranks)
{
    float* v = (float*)malloc(sizeof(float) * (size_t)C);
    int* miss = (int*)malloc(sizeof(int) * (size_t)C);
    for (int64_t r = 0; r < R; ++r) {
        for (int32_t j = 0; j < C; ++j) {
            float x = X[r * ld + j];
            miss[j] = 0;
            if (isnan(x)) {
                if (exclude_missing) miss[j] = 1;
                else x = fill_value;
            }
            v[j] = x;
        }
        for (int32_t j = 0; j < C; ++j) {
            if (miss[j]) { ranks[r * C + j] = 0xFFFF; continue; }
            uint32_t rank = 0;
            for (int32_t i = 0; i < C; ++i) {
                if (miss[i] || !(v[i] < v[j])) continue;
                /* count v[i] only at its first occurrence, so equal values count once */
                int first = 1;
                for (int32_t k = 0; k < i; ++k)
                    if (!miss[k] && v[k] == v[i]) { first = 0; break; }
                rank += (uint32_t)first;
            }
            ranks[r * C + j] = (uint16_t)rank;
        }
    }
    free(v);
    free(miss);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
