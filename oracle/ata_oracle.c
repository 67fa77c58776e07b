/*
 * CPU oracle for the lower-triangle Gram product low(C) = low(A^T A).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library, and it is deliberately plain and slow so that a reader can check it
 * against the paper line by line.
 *
 * Arithmetic: IEEE binary64, round-to-nearest, and NO fused multiply-add (the
 * build passes -ffp-contract=off), so every result is reproducible bit for bit
 * on x86-64 and aarch64 hosts.
 *
 * Layout: A is m x n, row-major, leading dimension lda >= n (element (i,j) at
 * A[i*lda + j]).  C is n x n, row-major, leading dimension ldc >= n.
 *
 * Two independent oracles live here:
 *
 *  1. The plain definition (Section 3.1, Eq. "Cij": C = A^T A, C_jk =
 *     sum_i a_ij a_ik; the method stores only the lower triangle, k <= j).
 *     This is the reference VALUE every other path is judged against.  Beside
 *     it, D_jk = sum_i |a_ij| |a_ik| (the denominator of the componentwise
 *     error metric) is computed the same way.
 *
 *  2. The AtA recursion of Algorithm 1 (Section 3.1) with textbook Strassen
 *     (the paper's reference for Strassen's algorithm, 1969) for the A^T B
 *     products on the off-diagonal block.  It pins the STRUCTURE of the method
 *     (splits, Strassen wiring, multiplication counts; Section 3.2, Eq.
 *     "ATACC" and the count 2/3 n^log2(7) + 1/3 n^2 of the introduction), not
 *     the reference values.
 *
 * Readings of the paper used here (where it is silent or garbled):
 *  - Eq. "submatA" lists A_{2,1} twice; the fourth block is A_{2,2} =
 *    A[m1:m, n1:n].
 *  - AtA splits floor-first: m1 = floor(m/2), n1 = floor(n/2) (Eq. "submatA").
 *  - Strassen halves "rounding up" (Section 3.3): the first block takes
 *    ceil(d/2) and the smaller second block is treated as zero-padded to the
 *    size of the first (Section 3.1, handling of odd sizes).
 *  - The base case "m x n <= cache size" (Algorithm 1) becomes "n <= cutoff"
 *    (or m <= 1 or n <= 1).  The Strassen base case is a depth budget:
 *    depth == 0 (or any dimension <= 1) calls the classical leaf.
 *  - The scaling factor alpha of Algorithm 1 is 1 and C is accumulated into
 *    (C <- C + A^T A on the lower triangle), exactly as Algorithm 1 states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* 1. The plain definition                                                  */
/* ------------------------------------------------------------------------ */

/* Number of host threads the definition loops use (1 = serial).  The loops
 * below parallelise over output rows j only; every entry is still one
 * ascending-i sum, so the result does not depend on the thread count. */
static int g_threads = 1;

int oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t < 1) t = omp_get_max_threads();
    g_threads = t;
#else
    (void)t;
    g_threads = 1;
#endif
    return g_threads;
}

/* low(C) <- low(A^T A): C_jk = sum_{i=0}^{m-1} a_ij * a_ik for 0 <= k <= j < n,
 * summed in ascending i.  The strict upper triangle of C is not touched. */
void oracle_ata_lower(int64_t m, int64_t n, const double *A, int64_t lda,
                      double *C, int64_t ldc) {
    int64_t j;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
    for (j = 0; j < n; ++j) {
        for (int64_t k = 0; k <= j; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double p = A[i * lda + j] * A[i * lda + k];
                s = s + p;
            }
            C[j * ldc + k] = s;
        }
    }
}

/* low(D) <- low(|A|^T |A|): D_jk = sum_i |a_ij| * |a_ik|, same loop order. */
void oracle_abs_ata_lower(int64_t m, int64_t n, const double *A, int64_t lda,
                          double *D, int64_t ldd) {
    int64_t j;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
    for (j = 0; j < n; ++j) {
        for (int64_t k = 0; k <= j; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double p = fabs(A[i * lda + j]) * fabs(A[i * lda + k]);
                s = s + p;
            }
            D[j * ldd + k] = s;
        }
    }
}

/* Full square C = A^T A (both triangles, each entry its own ascending-i sum).
 * Used only to check the exact symmetry C_jk == C_kj. */
void oracle_ata_full(int64_t m, int64_t n, const double *A, int64_t lda,
                     double *C, int64_t ldc) {
    int64_t j;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
    for (j = 0; j < n; ++j) {
        for (int64_t k = 0; k < n; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double p = A[i * lda + j] * A[i * lda + k];
                s = s + p;
            }
            C[j * ldc + k] = s;
        }
    }
}

/* Sampled entries: for t < count, out[t] = C_{rows[t], cols[t]} and
 * dout[t] = D_{rows[t], cols[t]} (dout may be NULL).  Same arithmetic as
 * oracle_ata_lower, so a sampled value equals the full oracle's bit for bit.
 * Used where the full product is too large for the CPU. */
void oracle_ata_entries(int64_t m, int64_t n, const double *A, int64_t lda,
                        int64_t count, const int64_t *rows, const int64_t *cols,
                        double *out, double *dout) {
    (void)n;
    int64_t t;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
#endif
    for (t = 0; t < count; ++t) {
        int64_t j = rows[t], k = cols[t];
        double s = 0.0, d = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double p = A[i * lda + j] * A[i * lda + k];
            s = s + p;
            double q = fabs(A[i * lda + j]) * fabs(A[i * lda + k]);
            d = d + q;
        }
        out[t] = s;
        if (dout) dout[t] = d;
    }
}

/* Sampled entries from column panels: colj holds column j of A (length m,
 * contiguous) for every sampled pair, colk column k.  For t < count:
 * out[t] = sum_i colj[t*m+i] * colk[t*m+i], ascending i.  Lets a caller that
 * can only afford to materialise the sampled columns of a huge A still get
 * the plain-definition value. */
void oracle_dot_pairs(int64_t m, int64_t count, const double *colj,
                      const double *colk, double *out, double *dout) {
    int64_t t;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
#endif
    for (t = 0; t < count; ++t) {
        double s = 0.0, d = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double p = colj[t * m + i] * colk[t * m + i];
            s = s + p;
            double q = fabs(colj[t * m + i]) * fabs(colk[t * m + i]);
            d = d + q;
        }
        out[t] = s;
        if (dout) dout[t] = d;
    }
}

/* ------------------------------------------------------------------------ */
/* 2. The AtA recursion (Algorithm 1) with textbook Strassen                */
/* ------------------------------------------------------------------------ */

/* A matrix view: rows x cols, row-major with leading dimension ld.  A view
 * with rows == 0 or cols == 0 is empty. */
typedef struct {
    double *p;
    int64_t rows, cols, ld;
} view_t;

static view_t sub(view_t v, int64_t r0, int64_t c0, int64_t r, int64_t c) {
    view_t s;
    s.p = v.p + r0 * v.ld + c0;
    s.rows = r;
    s.cols = c;
    s.ld = v.ld;
    return s;
}

/* Counters the recursion reports (all counts of scalar multiplications or
 * calls; see Section 3.2). */
typedef struct {
    uint64_t mults;        /* scalar multiplications done by the leaves   */
    uint64_t syrk_leaves;  /* number of classical A^T A leaf calls        */
    uint64_t gemm_leaves;  /* number of classical A^T B leaf calls        */
    uint64_t ata_calls;    /* number of AtA invocations (incl. leaves)    */
    uint64_t strassen_levels; /* number of Strassen splits performed      */
    uint64_t block_adds;   /* number of matrix (block) additions (Sec 3.2) */
} oracle_counts_t;

/* Test-only mutations, used to show that the pins catch plausible mistakes.
 * 0 = the method as the paper states it. */
static int g_mutation = 0;
void oracle_set_mutation(int mu) { g_mutation = mu; }

/* The classical A^T A leaf (the '?syrk' of Algorithm 1):
 * low(C) += low(A^T A), C_jk += sum_i a_ij a_ik for k <= j. */
static void leaf_syrk(view_t A, view_t C, oracle_counts_t *cnt) {
    cnt->syrk_leaves++;
    for (int64_t j = 0; j < A.cols; ++j) {
        for (int64_t k = 0; k <= j; ++k) {
            double s = 0.0;
            int64_t rows = A.rows;
            if (g_mutation == 1 && rows > 0) rows -= 1; /* drop a term */
            for (int64_t i = 0; i < rows; ++i) {
                double p = A.p[i * A.ld + j] * A.p[i * A.ld + k];
                s = s + p;
            }
            C.p[j * C.ld + k] += s;
        }
    }
    cnt->mults += (uint64_t)A.rows * (uint64_t)A.cols * (uint64_t)(A.cols + 1) / 2;
}

/* The classical A^T B leaf (the '?gemm' of Algorithm 1):
 * C += A^T B with A r x p, B r x q, C p x q. */
static void leaf_gemm(view_t A, view_t B, view_t C, oracle_counts_t *cnt) {
    cnt->gemm_leaves++;
    for (int64_t j = 0; j < A.cols; ++j) {
        for (int64_t k = 0; k < B.cols; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < A.rows; ++i) {
                double p = A.p[i * A.ld + j] * B.p[i * B.ld + k];
                s = s + p;
            }
            C.p[j * C.ld + k] += s;
        }
    }
    cnt->mults += (uint64_t)A.rows * (uint64_t)A.cols * (uint64_t)B.cols;
}

/* A fresh zero matrix of the given size (caller frees .p). */
static view_t zeros(int64_t r, int64_t c) {
    view_t v;
    v.rows = r;
    v.cols = c;
    v.ld = c > 0 ? c : 1;
    v.p = (double *)calloc((size_t)(r > 0 ? r : 1) * (size_t)v.ld, sizeof(double));
    return v;
}

/* dst (r x c, zero-initialised) += sign * src, where src may be smaller than
 * dst: the missing rows/columns of src count as zeros (the paper's simulated
 * zero padding of odd-sized blocks, Section 3.1). */
static void add_into(view_t dst, view_t src, double sign) {
    for (int64_t i = 0; i < src.rows; ++i)
        for (int64_t j = 0; j < src.cols; ++j)
            dst.p[i * dst.ld + j] += sign * src.p[i * src.ld + j];
}

/* C (p x q view, possibly smaller than M) += sign * M clipped to C's size. */
static void add_clipped(view_t C, view_t M, double sign) {
    for (int64_t i = 0; i < C.rows; ++i)
        for (int64_t j = 0; j < C.cols; ++j)
            C.p[i * C.ld + j] += sign * M.p[i * M.ld + j];
}

/* Strassen for C += A^T B (A r x p, B r x q, C p x q), at most `depth` levels.
 *
 * With X = A^T (p x r) and Y = B (r x q), split every dimension ceil-first:
 * r1 = ceil(r/2), p1 = ceil(p/2), q1 = ceil(q/2).  The blocks of X are
 * X11 = A11^T, X12 = A21^T, X21 = A12^T, X22 = A22^T, where A11 = A[0:r1,0:p1],
 * A12 = A[0:r1,p1:p], A21 = A[r1:r,0:p1], A22 = A[r1:r,p1:p]; the blocks of Y
 * are the blocks of B.  Smaller blocks are zero-padded to r1 x p1 / r1 x q1.
 * Strassen's seven products (1969) in this A^T B form:
 *   M1 = (A11 + A22)^T (B11 + B22)     M5 = (A11 + A21)^T B22
 *   M2 = (A12 + A22)^T B11             M6 = (A12 - A11)^T (B11 + B12)
 *   M3 = A11^T (B12 - B22)             M7 = (A21 - A22)^T (B21 + B22)
 *   M4 = A22^T (B21 - B11)
 *   C11 += M1 + M4 - M5 + M7     C12 += M3 + M5
 *   C21 += M2 + M4               C22 += M1 - M2 + M3 + M6
 * i.e. 10 operand additions and 8 result additions: the 18 block additions of
 * Section 3.2. */
static void strassen(view_t A, view_t B, view_t C, int depth, oracle_counts_t *cnt) {
    int64_t r = A.rows, p = A.cols, q = B.cols;
    if (r == 0 || p == 0 || q == 0) return;
    if (depth <= 0 || r <= 1 || p <= 1 || q <= 1) {
        leaf_gemm(A, B, C, cnt);
        return;
    }
    cnt->strassen_levels++;
    int64_t r1 = (r + 1) / 2, r2 = r - r1;
    int64_t p1 = (p + 1) / 2, p2 = p - p1;
    int64_t q1 = (q + 1) / 2, q2 = q - q1;

    view_t A11 = sub(A, 0, 0, r1, p1), A12 = sub(A, 0, p1, r1, p2);
    view_t A21 = sub(A, r1, 0, r2, p1), A22 = sub(A, r1, p1, r2, p2);
    view_t B11 = sub(B, 0, 0, r1, q1), B12 = sub(B, 0, q1, r1, q2);
    view_t B21 = sub(B, r1, 0, r2, q1), B22 = sub(B, r1, q1, r2, q2);
    view_t C11 = sub(C, 0, 0, p1, q1), C12 = sub(C, 0, q1, p1, q2);
    view_t C21 = sub(C, p1, 0, p2, q1), C22 = sub(C, p1, q1, p2, q2);

    /* Operand sums, zero-padded to r1 x p1 (A side) and r1 x q1 (B side). */
    view_t S[5], T[5];
    for (int t = 0; t < 5; ++t) { S[t] = zeros(r1, p1); T[t] = zeros(r1, q1); }
    add_into(S[0], A11, 1.0); add_into(S[0], A22, 1.0);   /* A11 + A22 */
    add_into(S[1], A12, 1.0); add_into(S[1], A22, 1.0);   /* A12 + A22 */
    add_into(S[2], A11, 1.0); add_into(S[2], A21, 1.0);   /* A11 + A21 */
    add_into(S[3], A12, 1.0); add_into(S[3], A11, -1.0);  /* A12 - A11 */
    add_into(S[4], A21, 1.0); add_into(S[4], A22, -1.0);  /* A21 - A22 */
    add_into(T[0], B11, 1.0); add_into(T[0], B22, 1.0);   /* B11 + B22 */
    add_into(T[1], B12, 1.0); add_into(T[1], B22, -1.0);  /* B12 - B22 */
    add_into(T[2], B21, 1.0); add_into(T[2], B11, -1.0);  /* B21 - B11 */
    add_into(T[3], B11, 1.0); add_into(T[3], B12, 1.0);   /* B11 + B12 */
    add_into(T[4], B21, 1.0); add_into(T[4], B22, 1.0);   /* B21 + B22 */
    cnt->block_adds += 10;
    if (g_mutation == 2) add_into(T[2], B11, 2.0);        /* wrong sign in M4 */

    /* Plain (padded) quadrants used alone by M2..M5. */
    view_t PA11 = zeros(r1, p1), PA22 = zeros(r1, p1);
    view_t PB11 = zeros(r1, q1), PB22 = zeros(r1, q1);
    add_into(PA11, A11, 1.0); add_into(PA22, A22, 1.0);
    add_into(PB11, B11, 1.0); add_into(PB22, B22, 1.0);

    view_t M[7];
    for (int t = 0; t < 7; ++t) M[t] = zeros(p1, q1);
    strassen(S[0], T[0], M[0], depth - 1, cnt);           /* M1 */
    strassen(S[1], PB11, M[1], depth - 1, cnt);           /* M2 */
    if (g_mutation == 3)
        strassen(PA22, T[1], M[2], depth - 1, cnt);       /* wrong operand */
    else
        strassen(PA11, T[1], M[2], depth - 1, cnt);       /* M3 */
    strassen(PA22, T[2], M[3], depth - 1, cnt);           /* M4 */
    strassen(S[2], PB22, M[4], depth - 1, cnt);           /* M5 */
    strassen(S[3], T[3], M[5], depth - 1, cnt);           /* M6 */
    strassen(S[4], T[4], M[6], depth - 1, cnt);           /* M7 */

    /* Result sums, clipped to the true block sizes. */
    add_clipped(C11, M[0], 1.0); add_clipped(C11, M[3], 1.0);
    add_clipped(C11, M[4], -1.0); add_clipped(C11, M[6], 1.0);
    add_clipped(C12, M[2], 1.0); add_clipped(C12, M[4], 1.0);
    add_clipped(C21, M[1], 1.0); add_clipped(C21, M[3], 1.0);
    add_clipped(C22, M[0], 1.0); add_clipped(C22, M[1], -1.0);
    add_clipped(C22, M[2], 1.0); add_clipped(C22, M[5], 1.0);
    cnt->block_adds += 8;

    for (int t = 0; t < 5; ++t) { free(S[t].p); free(T[t].p); }
    free(PA11.p); free(PA22.p); free(PB11.p); free(PB22.p);
    for (int t = 0; t < 7; ++t) free(M[t].p);
}

/* AtA(A, C) of Algorithm 1: low(C) += low(A^T A) for A m x n, C n x n.
 * Split A floor-first into A11 (m1 x n1), A12 (m1 x n2), A21 (m2 x n1),
 * A22 (m2 x n2) (Eq. "submatA").  Then (Eq. "Cij"):
 *   C11 += A11^T A11 + A21^T A21   (two recursive AtA calls)
 *   C22 += A12^T A12 + A22^T A22   (two recursive AtA calls)
 *   C21 += A12^T A11 + A22^T A21   (two Strassen A^T B calls)
 * C12 = C21^T is never formed. */
static void ata(view_t A, view_t C, int64_t cutoff, int depth, oracle_counts_t *cnt) {
    int64_t m = A.rows, n = A.cols;
    if (m == 0 || n == 0) return;
    cnt->ata_calls++;
    if (n <= cutoff || m <= 1 || n <= 1) {
        leaf_syrk(A, C, cnt);
        return;
    }
    int64_t m1 = m / 2, m2 = m - m1;
    int64_t n1 = n / 2, n2 = n - n1;
    view_t A11 = sub(A, 0, 0, m1, n1), A12 = sub(A, 0, n1, m1, n2);
    view_t A21 = sub(A, m1, 0, m2, n1), A22 = sub(A, m1, n1, m2, n2);
    view_t C11 = sub(C, 0, 0, n1, n1), C22 = sub(C, n1, n1, n2, n2);
    view_t C21 = sub(C, n1, 0, n2, n1);
    ata(A11, C11, cutoff, depth, cnt);
    ata(A21, C11, cutoff, depth, cnt);
    ata(A12, C22, cutoff, depth, cnt);
    ata(A22, C22, cutoff, depth, cnt);
    strassen(A12, A11, C21, depth, cnt);
    strassen(A22, A21, C21, depth, cnt);
}

/* Public entry of the recursion oracle.  low(C) += low(A^T A).
 * cutoff >= 1: column count at or below which AtA calls the classical leaf.
 * depth >= 0: Strassen levels per A^T B call (a large value recurses until a
 * dimension reaches 1).  counts (6 uint64, may be NULL) receives
 * {mults, syrk_leaves, gemm_leaves, ata_calls, strassen_levels, block_adds}.
 * Returns 0, or -1 on invalid arguments. */
int oracle_ata_recursive(int64_t m, int64_t n, const double *A, int64_t lda,
                         double *C, int64_t ldc, int64_t cutoff, int depth,
                         uint64_t *counts) {
    if (m < 0 || n < 0 || lda < n || ldc < n || cutoff < 1 || depth < 0) return -1;
    oracle_counts_t cnt;
    memset(&cnt, 0, sizeof(cnt));
    view_t Av = {(double *)A, m, n, lda};
    view_t Cv = {C, n, n, ldc};
    ata(Av, Cv, cutoff, depth, &cnt);
    if (counts) {
        counts[0] = cnt.mults;
        counts[1] = cnt.syrk_leaves;
        counts[2] = cnt.gemm_leaves;
        counts[3] = cnt.ata_calls;
        counts[4] = cnt.strassen_levels;
        counts[5] = cnt.block_adds;
    }
    return 0;
}

/* Strassen alone, C += A^T B (A r x p, B r x q, C p x q), at most `depth`
 * levels; counts as above.  Exposed so the tests can pin the A^T B wiring by
 * itself. */
int oracle_strassen_atb(int64_t r, int64_t p, int64_t q, const double *A, int64_t lda,
                        const double *B, int64_t ldb, double *C, int64_t ldc,
                        int depth, uint64_t *counts) {
    if (r < 0 || p < 0 || q < 0 || lda < p || ldb < q || ldc < q || depth < 0) return -1;
    oracle_counts_t cnt;
    memset(&cnt, 0, sizeof(cnt));
    view_t Av = {(double *)A, r, p, lda};
    view_t Bv = {(double *)B, r, q, ldb};
    view_t Cv = {C, p, q, ldc};
    strassen(Av, Bv, Cv, depth, &cnt);
    if (counts) {
        counts[0] = cnt.mults;
        counts[1] = cnt.syrk_leaves;
        counts[2] = cnt.gemm_leaves;
        counts[3] = cnt.ata_calls;
        counts[4] = cnt.strassen_levels;
        counts[5] = cnt.block_adds;
    }
    return 0;
}
