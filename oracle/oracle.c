/*
 * oracle.c -- plain, serial, obviously-correct CPU reference for the assembly
 * of element matrices into a global sparse matrix (Sky et al., arXiv
 * 2012.00585).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA library, and it is slow on purpose:
 * every function is the plain definition, or the paper's algorithm in the
 * paper's order, with nothing blocked, fused or reordered.
 *
 * Conventions (0-based throughout; the paper's figures are 1-based):
 *   elem_dofs  int32 [n_e * n_loc]          DOFs of element e in local order
 *   K          double [n_e * n_loc * n_loc] element matrices, row-major
 *   row_ptr    int64 [n_rows + 1]           CSR row pointers
 *   col_idx    int32 [nnz]                  CSR column indices, sorted per row
 *   crac_ptr   int64 [n_rows + 1]           CRAC row pointers, in int units of
 *                                           the column-alignments array
 *   col_align  int32 [n_ca]                 (first column, value position) pairs,
 *                                           then the final pair (n_cols, nnz)
 *
 * Build with -O2 -ffp-contract=off so that every "a = a + b" is one IEEE
 * double add.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_DOF_RANGE (-2)
#define OR_ERR_DUP_DOF (-3)
#define OR_ERR_NOT_IN_PATTERN (-4)
#define OR_ERR_OOM (-5)

void or_free(void *p) { free(p); }

/* The problem statement of §2.1: each element lists its DOFs once, and every
 * DOF is a row of the global matrix.  Rejects out-of-range and repeated DOFs
 * (the paper is silent on both). */
int or_check_elements(int64_t n_e, int32_t n_loc, int64_t n_dofs, const int32_t *elem_dofs)
{
    if (n_e < 0 || n_loc <= 0 || n_dofs < 0) return OR_ERR_ARG;
    for (int64_t e = 0; e < n_e; ++e) {
        const int32_t *D = elem_dofs + e * n_loc;
        for (int32_t r = 0; r < n_loc; ++r) {
            if (D[r] < 0 || (int64_t)D[r] >= n_dofs) return OR_ERR_DOF_RANGE;
            for (int32_t c = 0; c < r; ++c)
                if (D[c] == D[r]) return OR_ERR_DUP_DOF;
        }
    }
    return OR_OK;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sort the candidates of one row and drop repeats; returns the new length. */
static int64_t sort_unique(int32_t *buf, int64_t n)
{
    if (n == 0) return 0;
    qsort(buf, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t w = 1;
    for (int64_t k = 1; k < n; ++k)
        if (buf[k] != buf[w - 1]) buf[w++] = buf[k];
    return w;
}

/*
 * CSR sparsity pattern (§2.2, Fig. 1b/1c).  Row i holds column j exactly when
 * some element lists both i and j, i.e. when the sequential assembly of
 * Listing 2 would ever touch G(i, j).  Each row is collected from the
 * elements that contain DOF i, sorted ascending and made unique.
 *
 * row_ptr [n_dofs+1] is written by the caller-provided array; col_idx is
 * allocated here (free with or_free).  Returns nnz (>= 0) or an OR_ERR_*.
 */
int64_t or_csr_pattern(int64_t n_e, int32_t n_loc, int64_t n_dofs, const int32_t *elem_dofs,
                       int64_t *row_ptr, int32_t **col_idx_out)
{
    *col_idx_out = NULL;
    int rc = or_check_elements(n_e, n_loc, n_dofs, elem_dofs);
    if (rc != OR_OK) return rc;

    /* elements containing each DOF, in ascending element order */
    int64_t *inc_ptr = calloc((size_t)n_dofs + 1, sizeof(int64_t));
    int64_t *inc_el = malloc(sizeof(int64_t) * (size_t)(n_e * n_loc + 1));
    int64_t *fill = calloc((size_t)n_dofs + 1, sizeof(int64_t));
    if (!inc_ptr || !inc_el || !fill) { free(inc_ptr); free(inc_el); free(fill); return OR_ERR_OOM; }
    for (int64_t e = 0; e < n_e; ++e)
        for (int32_t r = 0; r < n_loc; ++r) inc_ptr[elem_dofs[e * n_loc + r] + 1] += 1;
    for (int64_t i = 0; i < n_dofs; ++i) inc_ptr[i + 1] += inc_ptr[i];
    for (int64_t e = 0; e < n_e; ++e)
        for (int32_t r = 0; r < n_loc; ++r) {
            int64_t i = elem_dofs[e * n_loc + r];
            inc_el[inc_ptr[i] + fill[i]++] = e;
        }
    free(fill);

    int64_t max_deg = 0;
    for (int64_t i = 0; i < n_dofs; ++i)
        if (inc_ptr[i + 1] - inc_ptr[i] > max_deg) max_deg = inc_ptr[i + 1] - inc_ptr[i];
    int32_t *buf = malloc(sizeof(int32_t) * (size_t)(max_deg * n_loc + 1));
    if (!buf) { free(inc_ptr); free(inc_el); return OR_ERR_OOM; }

    /* pass 1: row lengths */
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n_dofs; ++i) {
        int64_t n = 0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t)
            for (int32_t c = 0; c < n_loc; ++c) buf[n++] = elem_dofs[inc_el[t] * n_loc + c];
        row_ptr[i + 1] = row_ptr[i] + sort_unique(buf, n);
    }
    int64_t nnz = row_ptr[n_dofs];
    int32_t *col_idx = malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    if (!col_idx) { free(buf); free(inc_ptr); free(inc_el); return OR_ERR_OOM; }

    /* pass 2: the columns themselves */
    for (int64_t i = 0; i < n_dofs; ++i) {
        int64_t n = 0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t)
            for (int32_t c = 0; c < n_loc; ++c) buf[n++] = elem_dofs[inc_el[t] * n_loc + c];
        int64_t len = sort_unique(buf, n);
        memcpy(col_idx + row_ptr[i], buf, sizeof(int32_t) * (size_t)len);
    }
    free(buf);
    free(inc_ptr);
    free(inc_el);
    *col_idx_out = col_idx;
    return nnz;
}

/* CSR coefficient search (§2.2, the text after Listing 1): the position of
 * column j inside row i, by binary search over the sorted columns of the row.
 * Returns the position in the values array, or -1 when (i, j) is not in the
 * pattern. */
int64_t or_csr_lookup(const int64_t *row_ptr, const int32_t *col_idx, int64_t i, int32_t j)
{
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col_idx[mid] < j) lo = mid + 1; else hi = mid;
    }
    if (lo < row_ptr[i + 1] && col_idx[lo] == j) return lo;
    return -1;
}

/*
 * Sequential assembly, Listing 2: for every element e (in the given order, or
 * ascending), every row r and every column c of K_e, G(D(r), D(c)) is
 * replaced by G(D(r), D(c)) + K(r, c).  G is the values array of the CSR
 * pattern; the caller resets it (to zero, §3) or leaves it to accumulate.
 * ``order`` may be NULL (elements 0..n_e-1) or a permutation of them.
 */
int or_assemble_csr(int64_t n_e, int32_t n_loc, const int32_t *elem_dofs, const double *K,
                    const int64_t *row_ptr, const int32_t *col_idx, double *values,
                    const int64_t *order)
{
    for (int64_t t = 0; t < n_e; ++t) {
        int64_t e = order ? order[t] : t;
        const int32_t *D = elem_dofs + e * n_loc;
        const double *Ke = K + e * (int64_t)n_loc * n_loc;
        for (int32_t r = 0; r < n_loc; ++r)
            for (int32_t c = 0; c < n_loc; ++c) {
                int64_t slot = or_csr_lookup(row_ptr, col_idx, D[r], D[c]);
                if (slot < 0) return OR_ERR_NOT_IN_PATTERN;
                values[slot] = values[slot] + Ke[(int64_t)r * n_loc + c];
            }
    }
    return OR_OK;
}

/*
 * CRAC from CSR (§2.2, Fig. 1d).  The column-alignments array stores, for
 * every maximal block of consecutive column indices in a row, the pair
 * (first column of the block, its position in the values array); after the
 * last row comes a final pair whose value position is nnz.  The final pair's
 * column, drawn as "-" in Fig. 1d, is written as n_cols.  The CRAC row
 * pointers address the pairs array in int units (Fig. 1d: 1, 3, 5, 9, ...).
 *
 * crac_ptr [n_rows+1] is caller-provided; col_align is allocated here.
 * Returns n_ca = 2 * (number of blocks + 1).
 */
int64_t or_crac_from_csr(int64_t n_rows, int64_t n_cols, const int64_t *row_ptr,
                         const int32_t *col_idx, int64_t *crac_ptr, int32_t **col_align_out)
{
    *col_align_out = NULL;
    int64_t n_blocks = 0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (k == row_ptr[i] || col_idx[k] != col_idx[k - 1] + 1) ++n_blocks;
    int64_t n_ca = 2 * (n_blocks + 1);
    int32_t *ca = malloc(sizeof(int32_t) * (size_t)n_ca);
    if (!ca) return OR_ERR_OOM;
    int64_t w = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        crac_ptr[i] = w;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            if (k == row_ptr[i] || col_idx[k] != col_idx[k - 1] + 1) {
                ca[w++] = col_idx[k];
                ca[w++] = (int32_t)k;
            }
    }
    crac_ptr[n_rows] = w;
    ca[w++] = (int32_t)n_cols;
    ca[w++] = (int32_t)row_ptr[n_rows];
    *col_align_out = ca;
    return n_ca;
}

/*
 * Value position of column c in row `row` of a CRAC matrix, from the
 * format's definition (§2.2, Fig. 1d).  The row's pairs (first column f_k,
 * value position p_k) describe its runs of consecutive columns: run k covers
 * the columns f_k .. f_k + (p_{k+1} - p_k) - 1, p_{k+1} being the value
 * position of the pair that follows (for the row's last run, the next row's
 * first pair or the final pair).  Column c sits at p_k + (c - f_k) in the run
 * that covers it; -1 when no run of the row covers c.  Runs are sorted and
 * disjoint, so this is the run the paper's block search stops at (the last
 * run of the row that starts at or before c).
 */
int64_t or_crac_lookup(const int64_t *crac_ptr, const int32_t *col_align, int64_t row, int32_t c)
{
    for (int64_t k = crac_ptr[row]; k < crac_ptr[row + 1]; k += 2) {
        int64_t first = col_align[k];
        int64_t len = (int64_t)col_align[k + 3] - col_align[k + 1];
        if (c >= first && c < first + len) return col_align[k + 1] + (c - first);
    }
    return -1;
}

/*
 * The compressed element_dofs_array of §2.1: for every maximal run of
 * consecutive DOF indices, in local order, the pair (first index, run
 * length).  Example of §2.1: 52..55, 96..103, 48..51  ->  52 4 96 8 48 4.
 * ``out`` needs room for 2*n ints.  Returns the number of ints written.
 */
int32_t or_compress_dofs(int32_t n, const int32_t *dofs, int32_t *out)
{
    int32_t w = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (k > 0 && dofs[k] == dofs[k - 1] + 1) {
            out[w - 1] += 1;
        } else {
            out[w++] = dofs[k];
            out[w++] = 1;
        }
    }
    return w;
}

/*
 * Assembly through the CRAC format with the compressed DOF array, the
 * arithmetic of Listing 5 run serially (no threads, so no row lock): for each
 * element, each row r of K, and each run (first, len) of the compressed DOF
 * array, find the value position of column ``first`` in row D(r) by the
 * block search of Listing 1, then add the slice K(r, c .. c+len-1) to the
 * len consecutive values there.  Per value, the additions happen in the same
 * element order as in Listing 2.
 */
int or_assemble_crac(int64_t n_e, int32_t n_loc, const int32_t *elem_dofs, const double *K,
                     const int64_t *crac_ptr, const int32_t *col_align, double *values,
                     const int64_t *order)
{
    int32_t *runs = malloc(sizeof(int32_t) * 2 * (size_t)n_loc);
    if (!runs) return OR_ERR_OOM;
    for (int64_t t = 0; t < n_e; ++t) {
        int64_t e = order ? order[t] : t;
        const int32_t *D = elem_dofs + e * n_loc;
        const double *Ke = K + e * (int64_t)n_loc * n_loc;
        int32_t n_runs2 = or_compress_dofs(n_loc, D, runs);
        for (int32_t r = 0; r < n_loc; ++r) {
            int32_t c = 0;
            for (int32_t a = 0; a < n_runs2; a += 2) {
                int64_t pos = or_crac_lookup(crac_ptr, col_align, D[r], runs[a]);
                if (pos < 0) { free(runs); return OR_ERR_NOT_IN_PATTERN; }
                for (int32_t s = 0; s < runs[a + 1]; ++s)
                    values[pos + s] = values[pos + s] + Ke[(int64_t)r * n_loc + c + s];
                c += runs[a + 1];
            }
        }
    }
    free(runs);
    return OR_OK;
}

/*
 * Greedy colouring of the elements (the colouring used by Listing 6): two
 * elements conflict when they share a DOF.  Elements are visited in
 * ascending order and each takes the smallest colour not used by an
 * already-coloured element that shares a DOF with it.  Returns the number
 * of colours; colour[e] receives the colour of element e.
 */
int32_t or_greedy_colouring(int64_t n_e, int32_t n_loc, int64_t n_dofs, const int32_t *elem_dofs,
                            int32_t *colour)
{
    int64_t *inc_ptr = calloc((size_t)n_dofs + 1, sizeof(int64_t));
    int64_t *inc_el = malloc(sizeof(int64_t) * (size_t)(n_e * n_loc + 1));
    int64_t *fill = calloc((size_t)n_dofs + 1, sizeof(int64_t));
    if (!inc_ptr || !inc_el || !fill) { free(inc_ptr); free(inc_el); free(fill); return OR_ERR_OOM; }
    for (int64_t e = 0; e < n_e; ++e)
        for (int32_t r = 0; r < n_loc; ++r) inc_ptr[elem_dofs[e * n_loc + r] + 1] += 1;
    for (int64_t i = 0; i < n_dofs; ++i) inc_ptr[i + 1] += inc_ptr[i];
    for (int64_t e = 0; e < n_e; ++e)
        for (int32_t r = 0; r < n_loc; ++r) {
            int64_t i = elem_dofs[e * n_loc + r];
            inc_el[inc_ptr[i] + fill[i]++] = e;
        }
    free(fill);
    int64_t cap = 64;
    uint8_t *used = malloc((size_t)cap);
    int32_t n_colours = 0;
    for (int64_t e = 0; e < n_e; ++e) colour[e] = -1;
    for (int64_t e = 0; e < n_e; ++e) {
        memset(used, 0, (size_t)cap);
        for (int32_t r = 0; r < n_loc; ++r) {
            int64_t i = elem_dofs[e * n_loc + r];
            for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
                int32_t k = colour[inc_el[t]];
                if (k < 0) continue;
                if (k >= cap) {
                    int64_t ncap = cap;
                    while (k >= ncap) ncap *= 2;
                    used = realloc(used, (size_t)ncap);
                    memset(used + cap, 0, (size_t)(ncap - cap));
                    cap = ncap;
                }
                used[k] = 1;
            }
        }
        int32_t k = 0;
        while (k < cap && used[k]) ++k;
        colour[e] = k;
        if (k + 1 > n_colours) n_colours = k + 1;
    }
    free(used);
    free(inc_ptr);
    free(inc_el);
    return n_colours;
}

/* Sparse matrix-vector product y = G x over the CSR arrays (the operation the
 * paper's outlook names as the consumer of the assembled matrix), each row
 * summed left to right from +0.0. */
void or_spmv_csr(int64_t n_rows, const int64_t *row_ptr, const int32_t *col_idx,
                 const double *values, const double *x, double *y)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + values[k] * x[col_idx[k]];
        y[i] = s;
    }
}

/* The same product read through the CRAC arrays: every block contributes
 * values[pos .. pos+len-1] times x[first .. first+len-1], blocks in order. */
void or_spmv_crac(int64_t n_rows, const int64_t *crac_ptr, const int32_t *col_align,
                  const double *values, const double *x, double *y)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double s = 0.0;
        for (int64_t p = crac_ptr[i]; p < crac_ptr[i + 1]; p += 2) {
            int64_t first = col_align[p], pos = col_align[p + 1];
            int64_t len = (int64_t)col_align[p + 3] - pos;
            for (int64_t t = 0; t < len; ++t) s = s + values[pos + t] * x[first + t];
        }
        y[i] = s;
    }
}
