/*
 * Plain CPU oracle for the 2-domination transfer-matrix method of
 * "HPC acceleration of large (min,+) matrix products to compute
 * domination-type parameters in graphs" (arXiv 2409.17688).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  The CUDA library never
 * links, includes or calls it, and it shares no source with the CUDA library.
 *
 * Everything here is the plain definition written out, slow on purpose:
 *   - words are arrays of letters, enumerated by counting in base 3;
 *   - the arc rule is tested letter by letter, exactly as the three bullets
 *     of Section 2.2 state it;
 *   - the (min,+) product is the triple loop of its definition (Section 1),
 *     accumulated in 32-bit integers and clamped at the INF code.
 *
 * Notation: the paper writes the cylinder as P_m x C_n (m = path order);
 * here n is the path order and m the cycle length, so a "correct n-word" is
 * a column labelling of P_n.
 *
 * INF encoding (the paper only says 16-bit integers, Section 3): 0x7FFF for
 * int16 and 255 for uint8, with saturating semantics min(INF, x + y).
 * Inputs must lie in [0, INF].
 *
 * Parity pins: every function below is pinned by tests that do not reuse it
 * (Table 1 counts, Tables 3/4/5, the C_5 and m = 0 mod 3 formulas of
 * Section 4, exhaustive subset search on small cylinders, walk enumeration
 * for Theorem 1, and tropical identities).  Nothing here is parity-unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_INF16 32767
#define OR_INF8 255

/* ------------------------------------------------------------------ */
/* Correct words (Section 2.2, definition of correct m-words).          */
/* ------------------------------------------------------------------ */

/* A word is correct when it contains none of 020, 111, 211, 112, 212 at any
 * position, does not start with 11 or 12 (letters 1-2), and does not end
 * with 11 or 21 (letters n-1, n). */
static int word_is_correct(const uint8_t *w, int n)
{
    for (int i = 0; i + 2 < n; ++i) {
        int a = w[i], b = w[i + 1], c = w[i + 2];
        if (a == 0 && b == 2 && c == 0) return 0;
        if (a == 1 && b == 1 && c == 1) return 0;
        if (a == 2 && b == 1 && c == 1) return 0;
        if (a == 1 && b == 1 && c == 2) return 0;
        if (a == 2 && b == 1 && c == 2) return 0;
    }
    if (n >= 2) {
        if (w[0] == 1 && w[1] == 1) return 0;
        if (w[0] == 1 && w[1] == 2) return 0;
        if (w[n - 2] == 1 && w[n - 1] == 1) return 0;
        if (w[n - 2] == 2 && w[n - 1] == 1) return 0;
    }
    return 1;
}

/* Enumerate {0,1,2}^n in lexicographic order (letter 1 most significant,
 * 0 < 1 < 2: Algorithm 1 starts from all n-element variations of 0,1,2)
 * and keep the correct words.  If letters != NULL, word t occupies
 * letters[t*n .. t*n+n-1] (at most cap words are written).  Returns the
 * number of correct words, or -1 on bad n. */
int64_t or_enumerate_words(int n, uint8_t *letters, int64_t cap)
{
    if (n < 1 || n > 20) return -1;
    int64_t total = 1;
    for (int i = 0; i < n; ++i) total *= 3;
    uint8_t w[20];
    int64_t count = 0;
    for (int64_t v = 0; v < total; ++v) {
        int64_t x = v;
        for (int i = n - 1; i >= 0; --i) { w[i] = (uint8_t)(x % 3); x /= 3; }
        if (!word_is_correct(w, n)) continue;
        if (letters && count < cap) memcpy(letters + count * n, w, (size_t)n);
        ++count;
    }
    return count;
}

/* ------------------------------------------------------------------ */
/* Arc rule "p can follow q" (Section 2.2, three bullets).              */
/* ------------------------------------------------------------------ */

int or_can_follow(const uint8_t *q, const uint8_t *p, int n)
{
    for (int i = 0; i < n; ++i) {
        /* first bullet: q_i = 2 forces p_i = 0 */
        if (q[i] == 2 && p[i] != 0) return 0;
        /* zeros among the neighbours p_{i-1}, p_{i+1} (missing ones at the
         * ends do not count) and the previous column's q_i */
        int zeros = 0;
        if (i > 0 && p[i - 1] == 0) ++zeros;
        if (i + 1 < n && p[i + 1] == 0) ++zeros;
        if (q[i] == 0) ++zeros;
        /* second bullet: p_i = 2 needs exactly one zero */
        if (p[i] == 2 && zeros != 1) return 0;
        /* third bullet: p_i = 1 needs at least two zeros */
        if (p[i] == 1 && zeros < 2) return 0;
    }
    return 1;
}

static int count_zeros(const uint8_t *p, int n)
{
    int z = 0;
    for (int i = 0; i < n; ++i) z += (p[i] == 0);
    return z;
}

/* Algorithm 1: A[i][j] = number of zeros of p_j if p_j can follow q_i,
 * else INF.  Rows are the source word q_i, columns the target word p_j
 * (Theorem 2 indexes A by (q, p) for the arc q -> p).  A is N x N row-major
 * with leading dimension N.  Returns N, or -1 on error. */
int64_t or_build_transfer(int n, int16_t *A, int64_t cap_N)
{
    int64_t N = or_enumerate_words(n, NULL, 0);
    if (N < 0 || N > cap_N) return -1;
    uint8_t *L = (uint8_t *)malloc((size_t)(N * n));
    if (!L) return -1;
    or_enumerate_words(n, L, N);
    for (int64_t i = 0; i < N; ++i) {
        const uint8_t *q = L + i * n;
        for (int64_t j = 0; j < N; ++j) {
            const uint8_t *p = L + j * n;
            A[i * N + j] = or_can_follow(q, p, n) ? (int16_t)count_zeros(p, n)
                                                  : (int16_t)OR_INF16;
        }
    }
    free(L);
    return N;
}

/* ------------------------------------------------------------------ */
/* (min,+) product (Section 1): Z_ij = min(INF, min_l X_il + Y_lj).      */
/* ------------------------------------------------------------------ */

/* The loops run i, l, j so the innermost loop walks rows of Y; for exact
 * integers the order in which the minimum is taken does not change it.
 * A term whose X_il is INF is skipped: with Y_lj >= 0 it is >= INF and the
 * final clamp at INF makes it irrelevant.  threads > 1 splits the rows of
 * X among OpenMP threads, the paper's CPU strategy (Section 3). */
void or_minplus_mul_i16(const int16_t *X, const int16_t *Y, int16_t *Z,
                        int64_t M, int64_t N, int64_t K,
                        int64_t ldx, int64_t ldy, int64_t ldz, int threads)
{
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
#endif
    for (int64_t i = 0; i < M; ++i) {
        int32_t *acc = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
        for (int64_t j = 0; j < N; ++j) acc[j] = OR_INF16;
        for (int64_t l = 0; l < K; ++l) {
            int32_t x = X[i * ldx + l];
            if (x >= OR_INF16) continue;
            const int16_t *yrow = Y + l * ldy;
            for (int64_t j = 0; j < N; ++j) {
                int32_t s = x + (int32_t)yrow[j];
                if (s < acc[j]) acc[j] = s;
            }
        }
        for (int64_t j = 0; j < N; ++j)
            Z[i * ldz + j] = (int16_t)(acc[j] < OR_INF16 ? acc[j] : OR_INF16);
        free(acc);
    }
}

void or_minplus_mul_u8(const uint8_t *X, const uint8_t *Y, uint8_t *Z,
                       int64_t M, int64_t N, int64_t K,
                       int64_t ldx, int64_t ldy, int64_t ldz, int threads)
{
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
#endif
    for (int64_t i = 0; i < M; ++i) {
        int32_t *acc = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
        for (int64_t j = 0; j < N; ++j) acc[j] = OR_INF8;
        for (int64_t l = 0; l < K; ++l) {
            int32_t x = X[i * ldx + l];
            if (x >= OR_INF8) continue;
            const uint8_t *yrow = Y + l * ldy;
            for (int64_t j = 0; j < N; ++j) {
                int32_t s = x + (int32_t)yrow[j];
                if (s < acc[j]) acc[j] = s;
            }
        }
        for (int64_t j = 0; j < N; ++j)
            Z[i * ldz + j] = (uint8_t)(acc[j] < OR_INF8 ? acc[j] : OR_INF8);
        free(acc);
    }
}

/* min over the main diagonal of an N x N int16 matrix (Theorem 2 /
 * Algorithm 5), returned as int32 (INF if every diagonal entry is INF). */
int32_t or_diag_min(const int16_t *P, int64_t N, int64_t ld)
{
    int32_t g = OR_INF16;
    for (int64_t i = 0; i < N; ++i)
        if (P[i * ld + i] < g) g = P[i * ld + i];
    return g;
}

/* Algorithm 2: powers P_1 = A, P_k = A (x) P_{k-1} (the paper's operand
 * order, Algorithm 2) when left_mul != 0, or P_k = P_{k-1} (x) A otherwise.
 * Both orders give the same matrix by associativity.  powers, when not NULL,
 * receives kmax matrices N x N (slot k-1 = P_k); gdiag, when not NULL,
 * receives min diag P_k in slot k-1.  Returns 0, or -1 on allocation
 * failure. */
int or_power_sequence(const int16_t *A, int64_t N, int kmax, int16_t *powers,
                      int32_t *gdiag, int left_mul, int threads)
{
    if (kmax < 1 || N < 1) return -1;
    size_t bytes = (size_t)(N * N) * sizeof(int16_t);
    int16_t *prev = (int16_t *)malloc(bytes), *cur = (int16_t *)malloc(bytes);
    if (!prev || !cur) { free(prev); free(cur); return -1; }
    memcpy(prev, A, bytes);
    if (powers) memcpy(powers, A, bytes);
    if (gdiag) gdiag[0] = or_diag_min(A, N, N);
    for (int k = 2; k <= kmax; ++k) {
        if (left_mul)
            or_minplus_mul_i16(A, prev, cur, N, N, N, N, N, N, threads);
        else
            or_minplus_mul_i16(prev, A, cur, N, N, N, N, N, N, threads);
        if (powers) memcpy(powers + (size_t)(k - 1) * (size_t)(N * N), cur, bytes);
        if (gdiag) gdiag[k - 1] = or_diag_min(cur, N, N);
        int16_t *t = prev; prev = cur; cur = t;
    }
    free(prev); free(cur);
    return 0;
}

/* Rows of the power chain, one row at a time: with right multiplication,
 * row i of P_k = (row i of P_{k-1}) (x) A, so row i of every power follows
 * from row i of A alone.  The product r (x) A is the same triple loop
 * (one row of X), with the INF entries of A skipped by listing, per row l
 * of A, the columns whose entry is finite (start/col/val, row l in
 * [start[l], start[l+1])).  out receives nrows x kmax x N values:
 * out[(t*kmax + k-1)*N + p] = P_k[rows[t]][p]. */
static int chain_rows(int64_t N, const int64_t *start, const int32_t *col, const int32_t *val,
                      const int64_t *rows, int64_t nrows, int kmax, int16_t *out, int threads)
{
    int failed = 0;
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
#endif
    for (int64_t t = 0; t < nrows; ++t) {
        int16_t *o = out + (size_t)t * (size_t)kmax * (size_t)N;
        int32_t *acc = (int32_t *)malloc((size_t)N * sizeof(int32_t));
        if (!acc) { failed = 1; continue; }
        for (int64_t p = 0; p < N; ++p) o[p] = OR_INF16;
        for (int64_t e = start[rows[t]]; e < start[rows[t] + 1]; ++e) o[col[e]] = (int16_t)val[e];
        for (int k = 2; k <= kmax; ++k) {
            const int16_t *r = o + (size_t)(k - 2) * (size_t)N;
            for (int64_t p = 0; p < N; ++p) acc[p] = OR_INF16;
            for (int64_t l = 0; l < N; ++l) {
                int32_t x = r[l];
                if (x >= OR_INF16) continue;
                for (int64_t e = start[l]; e < start[l + 1]; ++e) {
                    int32_t s2 = x + val[e];
                    if (s2 < acc[col[e]]) acc[col[e]] = s2;
                }
            }
            int16_t *w = o + (size_t)(k - 1) * (size_t)N;
            for (int64_t p = 0; p < N; ++p) w[p] = (int16_t)(acc[p] < OR_INF16 ? acc[p] : OR_INF16);
        }
        free(acc);
    }
    return failed ? -1 : 0;
}

int or_power_rows(const int16_t *A, int64_t N, const int64_t *rows, int64_t nrows,
                  int kmax, int16_t *out, int threads)
{
    int64_t *start = (int64_t *)malloc((size_t)(N + 1) * sizeof(int64_t));
    if (!start) return -1;
    int64_t nnz = 0;
    for (int64_t l = 0; l < N; ++l) {
        start[l] = nnz;
        for (int64_t p = 0; p < N; ++p) nnz += (A[l * N + p] < OR_INF16);
    }
    start[N] = nnz;
    int32_t *col = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int32_t *val = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!col || !val) { free(start); free(col); free(val); return -1; }
    for (int64_t l = 0, e = 0; l < N; ++l)
        for (int64_t p = 0; p < N; ++p)
            if (A[l * N + p] < OR_INF16) { col[e] = (int32_t)p; val[e] = A[l * N + p]; ++e; }
    int r = chain_rows(N, start, col, val, rows, nrows, kmax, out, threads);
    free(start); free(col); free(val);
    return r;
}

/* The same rows for A(D_n) without forming the N x N matrix (path orders
 * whose A does not fit the host): the finite entries of every row of A are
 * listed straight from the rule -- word p can follow word q (Section 2.2),
 * label the zeros of p (Algorithm 1) -- then the rows follow as above.
 * Returns N, or -1 on error. */
int64_t or_transfer_power_rows(int n, const int64_t *rows, int64_t nrows, int kmax,
                               int16_t *out, int threads)
{
    int64_t N = or_enumerate_words(n, NULL, 0);
    if (N <= 0) return -1;
    uint8_t *L = (uint8_t *)malloc((size_t)(N * n));
    int64_t *deg = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    int32_t **lists = (int32_t **)calloc((size_t)N, sizeof(int32_t *));
    if (!L || !deg || !lists) { free(L); free(deg); free(lists); return -1; }
    or_enumerate_words(n, L, N);
    int failed = 0;
    (void)threads;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads > 0 ? threads : 1)
#endif
    {
        int32_t *tmp = (int32_t *)malloc((size_t)N * sizeof(int32_t));
        if (!tmp) failed = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t q = 0; q < N; ++q) {
            if (!tmp) continue;
            int64_t c = 0;
            for (int64_t p = 0; p < N; ++p)
                if (or_can_follow(L + q * n, L + p * n, n)) tmp[c++] = (int32_t)p;
            lists[q] = (int32_t *)malloc((size_t)(c > 0 ? c : 1) * sizeof(int32_t));
            if (!lists[q]) { failed = 1; continue; }
            memcpy(lists[q], tmp, (size_t)c * sizeof(int32_t));
            deg[q] = c;
        }
        free(tmp);
    }
    int64_t *start = (int64_t *)malloc((size_t)(N + 1) * sizeof(int64_t));
    int64_t nnz = 0;
    if (start) {
        for (int64_t q = 0; q < N; ++q) { start[q] = nnz; nnz += deg[q]; }
        start[N] = nnz;
    }
    int32_t *col = start ? (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t)) : NULL;
    int32_t *val = start ? (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t)) : NULL;
    int64_t r = -1;
    if (!failed && start && col && val) {
        for (int64_t q = 0; q < N; ++q)
            for (int64_t e = 0; e < deg[q]; ++e) {
                int32_t p = lists[q][e];
                col[start[q] + e] = p;
                val[start[q] + e] = count_zeros(L + (int64_t)p * n, n);
            }
        r = chain_rows(N, start, col, val, rows, nrows, kmax, out, threads) == 0 ? N : -1;
    }
    for (int64_t q = 0; q < N; ++q) free(lists[q]);
    free(lists); free(deg); free(L); free(start); free(col); free(val);
    return r;
}

/* ------------------------------------------------------------------ */
/* Algorithms 3 and 4 (recurrence search), over stored powers.          */
/* ------------------------------------------------------------------ */

/* "P_i - P_j is a constant matrix" (Algorithm 3).  Reading for entries
 * that are INF: both matrices must have INF at the same places, and every
 * finite difference must be the same number.  Returns 1 and sets *b when
 * constant (an all-INF pair has no constant and returns 0). */
int or_diff_is_constant(const int16_t *Pi, const int16_t *Pj, int64_t N, int32_t *b)
{
    int have = 0;
    int32_t c = 0;
    for (int64_t e = 0; e < N * N; ++e) {
        int fi = Pi[e] < OR_INF16, fj = Pj[e] < OR_INF16;
        if (fi != fj) return 0;
        if (!fi) continue;
        int32_t d = (int32_t)Pi[e] - (int32_t)Pj[e];
        if (!have) { c = d; have = 1; }
        else if (d != c) return 0;
    }
    if (!have) return 0;
    *b = c;
    return 1;
}

/* Algorithm 3 over powers[0..K-1] (slot k-1 = P_k): scan i = K down to 1,
 * and for each i, j = i-1 down to 1; the first pair with a constant
 * difference gives a = i - j, b = the constant, r0 = j.  Returns 1 when
 * found, 0 otherwise. */
int or_recurrence_search(const int16_t *powers, int64_t N, int K,
                         int *r0, int *a, int32_t *b)
{
    size_t sz = (size_t)(N * N);
    for (int i = K; i >= 1; --i)
        for (int j = i - 1; j >= 1; --j) {
            int32_t c;
            if (or_diff_is_constant(powers + (size_t)(i - 1) * sz,
                                    powers + (size_t)(j - 1) * sz, N, &c)) {
                *a = i - j; *b = c; *r0 = j;
                return 1;
            }
        }
    return 0;
}

/* Algorithm 4: walk i down from r0 + a while P_i - P_{i-a} equals b
 * everywhere; n0 is the last i - a for which it held.  The walk stops at
 * i = a + 1, the smallest i for which P_{i-a} exists.  Returns n0 (>= 1),
 * or -1 if not even i = r0 + a holds. */
int or_min_recurrence(const int16_t *powers, int64_t N, int r0, int a, int32_t b)
{
    size_t sz = (size_t)(N * N);
    int n0 = -1;
    for (int i = r0 + a; i >= a + 1; --i) {
        int32_t c;
        if (!or_diff_is_constant(powers + (size_t)(i - 1) * sz,
                                 powers + (size_t)(i - a - 1) * sz, N, &c) || c != b)
            break;
        n0 = i - a;
    }
    return n0;
}

int or_have_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
