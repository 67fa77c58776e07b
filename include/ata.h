/*
 * ata.h -- C ABI of the GB300 (sm_103a) lower-triangle Gram-product library.
 *
 * The library computes low(C) = low(A^T A) for a rectangular m x n matrix A,
 * the AtA method of Arrigoni, Maggioli, Massini & Rodola, "Efficiently
 * Parallelizable Strassen-Based Multiplication of a Matrix by its Transpose"
 * (arXiv:2110.13042):
 *   - Section 3.1, Eq. "submatA"/"Cij" and Algorithm 1: A is split 2 x 2;
 *     C11 and C22 are AtA sub-problems, C21 = A12^T A11 + A22^T A21 is an
 *     A^T B product done by Strassen's algorithm, and C12 = C21^T is never
 *     formed (only the lower triangle of C is produced).
 *   - Section 3.3: Strassen's workspace is allocated once up front
 *     (FastStrassen); here the handle owns a device workspace that grows on
 *     demand and is reused by every later call.
 *   - Algorithm 3 / Section 4.1: the recursion is "simulated" up front into a
 *     flat list of independent leaf tasks that write disjoint blocks of C; here
 *     the leaves are GPU tiles executed by persistent kernels.
 *
 * All matrices are ROW-MAJOR.  A is m x n with leading dimension lda >= n
 * (element (i, j) at A[i*lda + j]).  C is n x n with leading dimension
 * ldc >= n.  All pointers passed to ata_lower / ata_syrk / ata_batched are
 * DEVICE pointers on the current CUDA device; the caller owns them.  A is read only
 * and must not overlap C.  `stream` is a cudaStream_t (NULL = legacy default
 * stream); every call is asynchronous on it.
 *
 * Semantics: ata_lower overwrites, low(C) <- low(A^T A); ata_syrk takes the
 * BLAS scalars, low(C) <- alpha low(A^T A) + beta low(C).  Entries (j, k)
 * with k <= j are written; the strict upper triangle of C is never read or
 * written.  m == 0 writes zeros to low(C) (ata_syrk: scales it by beta);
 * n == 0 does nothing.
 *
 * Errors: every entry point returns an ata_status.  No exception crosses the
 * ABI and no call aborts the process.  A device-side wait that exceeds its
 * budget does not hang: the kernel records ATA_ERR_TIMEOUT in a status word
 * that ata_sync() returns.
 */
#ifndef ATA_H
#define ATA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ATA_OK = 0,
    ATA_ERR_INVALID = 1,   /* bad dimension, leading dimension, pointer or overlap */
    ATA_ERR_DTYPE = 2,     /* unknown or unsupported dtype                          */
    ATA_ERR_ALLOC = 3,     /* device or host allocation failed                      */
    ATA_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed           */
    ATA_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out (see ata_sync)     */
    ATA_ERR_UNSUPPORTED = 6/* no sm_103a device, or a size beyond a documented limit */
} ata_status;

/* Arithmetic modes.  The element type of A and C is double for the F64
 * modes and float for the F32 modes. */
typedef enum {
    /* double in/out; FP64 tensor-core (DMMA) leaves, FP64 Strassen sums. */
    ATA_F64 = 0,
    /* double in/out; FP64-accurate emulation: every column is scaled by a
     * power of two, converted to fixed point and split into `slices` BF16
     * digits (7 bits, then 8 bits per digit); the digit products run on the
     * tcgen05 tensor cores with FP32 accumulation that is exact by
     * construction, and are summed exactly in 64-bit integers.  Strassen
     * operand sums and result sums are exact integer arithmetic. */
    ATA_F64_EMU = 1,
    /* float in/out; the same engine with 3 digits (23 bits per column). */
    ATA_F32 = 2,
    /* float in/out; one BF16 digit (8 bits per column, power-of-two column
     * scaling), FP32 tensor-core accumulation. Low precision. */
    ATA_F32_BF16 = 4,
    /* float in/out; one FP8 E4M3 product (kind::f8f6f4 tensor cores).  Each
     * column is scaled by a power of two so that its largest entry is below
     * 2^8 (E4M3 saturates at 448), every entry (or exact Strassen operand
     * sum) is rounded to nearest-even E4M3, and the products are summed in
     * FP32: in the tensor core over 512 contraction rows, then in the
     * epilogue's FP32 registers.  Strassen result sums are formed in FP64.
     * Low precision: componentwise error <= (2u + u^2) (|A|^T|A|)_jk plus
     * subnormal and accumulation terms, u = 2^-4, at Strassen depth 0.
     * ata_batched answers ATA_ERR_UNSUPPORTED and ata_lower_noalloc
     * ATA_ERR_DTYPE for this mode. */
    ATA_F32_FP8 = 5
} ata_dtype;

/* Planning parameters.  Zero (or -1 for strassen_depth) selects the
 * automatic choice of the autotuner. */
typedef struct {
    int cutoff;          /* AtA recursion stops at panels of <= cutoff columns
                            (Algorithm 1 base case); 0 = auto                     */
    int strassen_depth;  /* Strassen levels on every off-diagonal block
                            (0 = classical tiles, i.e. plain tiled AtA);
                            -1 = auto (1 for n >= 4096 in ATA_F64, and in
                            ATA_F64_EMU when also m >= 4096; else 0).  At
                            most ATA_MAX_STRASSEN_DEPTH; a
                            level splits a block only while both its sides
                            are >= strassen_min, so ATA_MAX_STRASSEN_DEPTH
                            recurses Strassen down to that size cutoff, as
                            the paper's FastStrassen recurses to its base
                            case (Section 3.1, Algorithm 1)                       */
    int slices;          /* digits per column for ATA_F64_EMU (1..7); 0 = auto    */
    int strassen_min;    /* a Strassen level splits an off-diagonal (sub)block
                            only while both its sides are >= strassen_min
                            columns; 0 = auto                                      */
    int strassen_variant;/* ATA_STRASSEN (0, Strassen's products, the paper's
                            choice) or ATA_WINOGRAD (1, Winograd's variant of
                            the seven products); ATA_F32_FP8 always uses
                            Strassen's                                             */
    int streams;         /* 0 or 1: every leaf tile of the recursion in one
                            persistent launch (the default); 2..16: a static
                            partition of the recursion's units (diagonal
                            panels, classical blocks, Strassen products) over
                            that many leaf launches on their own streams,
                            forked from and joined back into the caller's
                            stream: the counterpart of the paper's static
                            task tree of AtA-S (Section 4.1-4.2, Algorithm
                            3).  Results are bit-identical either way.         */
    int split_k;         /* contraction chunks per plain leaf tile (not for
                            ATA_F64): 0 = automatic (a plan with fewer than 4
                            tiles per SM and m >= 8192 splits the contraction
                            into chunks of >= 4096 rows; otherwise, when the
                            whole-contraction tiles leave the last wave of
                            the persistent CTAs partly idle, the last
                            (tiles mod SMs) of them are split into chunks of
                            >= 1024 rows if that shortens the busiest CTA by
                            >= 0.5%), 1 = never, 2..16 = that many for every
                            plain tile.  The chunks' exact partial products
                            are summed in a fixed order by the combine pass:
                            results stay deterministic (run to run
                            bit-identical) and within the mode's tolerance    */
    int reserved[1];     /* must be zero                                          */
} ata_config;

#define ATA_MAX_STRASSEN_DEPTH 8
#define ATA_STRASSEN 0
#define ATA_WINOGRAD 1

typedef struct ata_handle_s *ata_handle;

/* Create a handle on the current CUDA device.  cfg may be NULL (all auto).
 * The handle owns: the device workspace (Strassen operands and products,
 * digit planes), the plan cache and the device status word.  Allocation is
 * lazy (first call that needs it).  Returns ATA_ERR_UNSUPPORTED if the
 * current device is not sm_103. */
int ata_create(ata_handle *out, const ata_config *cfg);

/* Replace the handle's planning parameters (same meaning as ata_create). */
int ata_set_config(ata_handle h, const ata_config *cfg);

/* low(C) <- low(A^T A) for one m x n matrix (see the header comment).
 * dtype: one of ata_dtype.  Asynchronous on `stream`.  The first call for a
 * new (m, n, dtype) may grow the workspace with cudaMalloc (synchronous);
 * make it once before capturing the call in a CUDA graph.  A captured call
 * expects the handle's workspace to hold its plan's tables when it is
 * replayed: between capture and replay, make no call of another shape,
 * dtype or configuration on the same handle (use a handle per graph). */
int ata_lower(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda,
              void *C, int64_t ldc, int dtype, void *stream);

/* low(C) <- alpha low(A^T A) + beta low(C): the BLAS ?syrk semantics of the
 * paper's Section 3.1 (Algorithm 1 takes alpha and accumulates into C; the
 * text applies beta by scaling C first).  Arguments, layout, ownership and
 * errors as ata_lower, which is the case alpha = 1, beta = 0 (bit-identical
 * results).  alpha and beta are applied where each entry of C is stored
 * (FP64 arithmetic for the F64 modes, FP32 for the F32 modes): c <- alpha*v
 * + beta*c, one extra rounding each.  beta == 0: C is not read (NaN or Inf
 * there do not propagate).  alpha == 0 or m == 0: low(C) <- beta low(C)
 * without touching A (beta == 1: nothing happens).  Non-finite alpha or
 * beta: ATA_ERR_INVALID.  The strict upper triangle is never read or
 * written. */
int ata_syrk(ata_handle h, int64_t m, int64_t n, double alpha, const void *A, int64_t lda,
             double beta, void *C, int64_t ldc, int dtype, void *stream);

/* Flags of ata_syrk_ex (bitwise or). */
#define ATA_TRANS 1   /* the product A A^T instead of A^T A                    */
#define ATA_PACKED 2  /* C is a packed lower triangle instead of a full array  */

/* ata_syrk with layout flags; flags == 0 is ata_syrk (bit-identical).
 *
 * ATA_TRANS: low(C) <- alpha low(A A^T) + beta low(C).  The paper's method
 *   covers this product too (Section 3 introduction: A A^T is the A^T A of
 *   the transposed matrix, and the same recursion of Section 3.1 /
 *   Algorithm 1 applies).  A is still m x n row-major with lda >= n (the
 *   caller's array, not transposed); C is m x m (ldc >= m).  The contraction
 *   runs over the n columns of A: the column exponents are taken over A's
 *   rows and the operand preparation reads A row by row.  Same modes,
 *   planning (cutoff, Strassen depth on the m x m recursion) and arithmetic
 *   as ata_syrk on an explicit copy of A^T: results are bit-identical to it.
 * ATA_PACKED: C holds only the lower triangle, packed by rows: entry (j, k),
 *   k <= j, at C[j (j + 1) / 2 + k]; ldc is ignored.  The row-major layout
 *   of ata_lower stores the same values.  Packed triangles are what the
 *   paper's distributed AtA sends up its task tree (Section 4.3).
 * Arguments and errors otherwise as ata_syrk; unknown flag bits:
 * ATA_ERR_INVALID.  A must not overlap C (C spans m (m + 1) / 2 or
 * n (n + 1) / 2 elements when packed). */
int ata_syrk_ex(ata_handle h, int flags, int64_t m, int64_t n, double alpha, const void *A, int64_t lda,
                double beta, void *C, int64_t ldc, int dtype, void *stream);

/* low(C) <- low(A A^T) for a row-major m x n A (C is m x m): ata_syrk_ex with
 * ATA_TRANS, alpha = 1, beta = 0. */
int ata_lower_aat(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc,
                  int dtype, void *stream);

/* low(C_i) <- low(A_i^T A_i) for `count` independent problems in one
 * persistent launch.  m, n, lda, ldc: HOST arrays of length count.  A, C:
 * HOST arrays of `count` DEVICE pointers.  Only ATA_F32, ATA_F32_BF16 and
 * ATA_F64_EMU are accepted (ATA_F64, ATA_F32_FP8: ATA_ERR_UNSUPPORTED); every problem is
 * done as plain lower-triangle tiles of its own digit planes (no Strassen),
 * with the same arithmetic and bits as an ata_lower call with
 * strassen_depth = 0 and split_k = 1 (whole tiles).  Three
 * launches serve the whole batch: column exponents, digit planes, and one
 * persistent leaf launch over all problems' tiles (longest first).  Problems
 * with n == 0 are skipped and m == 0 zero-fills low(C_i).  The plan and its
 * task table live in pinned host memory owned by the handle and are reused
 * while the same shapes (m, n, lda, ldc, dtype) come back; new pointers are
 * written into the pinned table (after its previous upload has completed).
 * The call can be captured in a CUDA graph after a first uncaptured call
 * with those shapes; a replay uses the pointers of the captured call, as
 * long as no later call rewrote them (use ata_batched_dev to replay on new
 * buffers).  Errors: as ata_lower, checked per problem before anything is
 * launched.  The recursion analogue is the paper's static task list
 * (Section 4.1, Algorithm 3): every tile of every problem is one task. */
int ata_batched(ata_handle h, int count, const int64_t *m, const int64_t *n,
                const void *const *A, const int64_t *lda, void *const *C,
                const int64_t *ldc, int dtype, void *stream);

/* ata_batched with DEVICE-resident pointer arrays: A_dev and C_dev are device
 * arrays of `count` device pointers (A_i, C_i); m, n, lda, ldc stay host
 * arrays (the plan is made on the host from the shapes alone).  The arrays
 * are read on the device every time the call runs, so a CUDA graph captured
 * from one call can be replayed after the caller rewrites the arrays with
 * other buffers of the same shapes.  Pointers are not checked on the host:
 * each A_i and C_i must be a valid device buffer of its shape, and A_i must
 * not overlap C_i.  Everything else as ata_batched (bit-identical results). */
int ata_batched_dev(ata_handle h, int count, const int64_t *m, const int64_t *n,
                    const void *const *A_dev, const int64_t *lda, void *const *C_dev,
                    const int64_t *ldc, int dtype, void *stream);

/* Wait for `stream`, then return (and clear) the device status word:
 * ATA_OK, or ATA_ERR_TIMEOUT if a device-side wait ran out since the last
 * ata_sync, or ATA_ERR_CUDA if the stream reported an error. */
int ata_sync(ata_handle h, void *stream);

/* Self-test of the bounded device-side waits (the failure detection of the
 * persistent kernels; no counterpart in the paper).  Launches one block on
 * `stream` whose thread waits, through the same bounded-wait routine the leaf
 * kernels use, on a barrier that nothing completes.  After budget_ns of GPU
 * time (1000 <= budget_ns <= 10^10) the wait gives up, records
 * ATA_ERR_TIMEOUT in the handle's status word and the kernel returns; the
 * next ata_sync reports it and clears it, and the handle and the CUDA context
 * stay usable.  For tests and health checks.  ATA_ERR_INVALID for a budget
 * outside the range. */
int ata_check_wait_timeout(ata_handle h, int64_t budget_ns, void *stream);

/* Release the handle and its workspace (synchronises the device first). */
int ata_destroy(ata_handle h);

/* Static English description of a status code. */
const char *ata_status_string(int status);

/* Description of the most recent failure on this handle ("" if none): the
 * step that failed and the CUDA error string.  Valid until the next call. */
const char *ata_last_error(ata_handle h);

/* Host-only plan description, for tests and tuning.  Fills `out` (host array
 * of ATA_PLAN_FIELDS int64) for the plan ata_lower would run for (m, n,
 * dtype) under the handle's configuration, without touching the GPU:
 *   [0] cutoff used            [1] Strassen depth used   [2] digits (slices)
 *   [3] diagonal panels        [4] off-diagonal blocks   [5] Strassen products
 *   [6] leaf tiles             [7] workspace bytes       [8] classical-equivalent
 *                                                           multiply-adds done by
 *                                                           the leaves (per digit
 *                                                           pair)
 *   [9] multiply-adds of plain tiled AtA on the same tile grid
 *   [10] contraction chunks per plain tile (split_k; 1 = not split)
 *   [11] fused operand-prep groups (Strassen operand sums of one side of a
 *        block written from one read of its blocks of A; any adds one prep
 *        kernel launch)
 *   [12] combine regions (Strassen result sums and tiles computed as
 *        contraction chunks; any adds one combine launch)
 * h may be NULL (default configuration). */
#define ATA_PLAN_FIELDS 13
int ata_plan_info(ata_handle h, int64_t m, int64_t n, int dtype, int64_t *out);

/* Host-only description of the off-diagonal blocks of the plan ata_lower
 * would run for (m, n, dtype) under the handle's configuration (the AtA
 * recursion of Section 3.1 / Algorithm 1: block C21 = A12^T A11 + A22^T A21 of
 * every split).  Writes up to max_blocks records of ATA_BLOCK_FIELDS int64
 * into `out` (host array):
 *   [0] r0  first row of the block in C (= first column of A12 / A22)
 *   [1] p   its rows
 *   [2] c0  first column of the block in C (= first column of A11 / A21)
 *   [3] q   its columns
 *   [4] Strassen levels applied to it (0: classical tiles)
 * in recursion order, and the total block count to *count (host).  Touches
 * no GPU; h may be NULL (default configuration).  Errors: ATA_ERR_INVALID
 * for bad sizes or a NULL count, ATA_ERR_DTYPE for an unknown dtype. */
#define ATA_BLOCK_FIELDS 5
int ata_plan_blocks(ata_handle h, int64_t m, int64_t n, int dtype, int64_t *out, int64_t max_blocks,
                    int64_t *count);

/* Phase timing.  When enabled, ata_lower records CUDA events on its stream
 * around each phase; ata_phase_times waits for the most recent call's events
 * and writes 4 durations in milliseconds: [0] column exponents, [1] operand
 * preparation (digit planes, Strassen operand sums), [2] leaf products (the
 * tensor-core kernel), [3] Strassen result sums.  Returns ATA_ERR_INVALID if
 * timing is off or no call has been timed since it was enabled. */
int ata_set_timing(ata_handle h, int enable);
int ata_phase_times(ata_handle h, double *out);

/* Autotuning of the planning parameters (the recursion cutoff, Strassen
 * depth and the smallest block Strassen splits) for one shape.  Candidate
 * configurations are planned on the host (identical plans are run once),
 * timed with CUDA events on `stream` using the caller's A and C (C ends up
 * holding low(A^T A)), and the fastest is stored in the handle's tuning
 * table under (m, n, dtype).  Later ata_lower / ata_plan_info calls with that
 * shape use it whenever the handle's configuration leaves cutoff, depth and
 * strassen_min on auto (0, -1, 0).  Synchronous; budget_ms bounds the total
 * time spent (candidates are tried cheapest-plan first, plain tiles always).
 * out (host, may be NULL) receives {cutoff, depth, strassen_min, candidates
 * timed} of the choice.  Errors: as ata_lower. */
#define ATA_TUNE_FIELDS 4
int ata_tune(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc, int dtype,
             void *stream, double budget_ms, int64_t *out);

/* Forget every tuned shape of the handle. */
int ata_tune_clear(ata_handle h);

/* Allocation-free variant of ata_lower, for callers that cannot allocate
 * device memory when they need the product (inside a CUDA-graph capture they
 * do not control, under a framework memory pool that forbids side
 * allocations, or in a service that must not call cudaMalloc after start-up).
 * The paper has no counterpart: this is a deployment convenience.
 *
 * Computes low(C) <- low(A^T A) exactly like ata_lower with
 * strassen_depth = 0 and split_k = 1 (plain whole tiles, same kernels and
 * digit count) for dtype
 * ATA_F64_EMU, ATA_F32 or ATA_F32_BF16 (others: ATA_ERR_DTYPE).  Arguments
 * are as for ata_lower; there is no handle.  It calls no cudaMalloc, cudaFree
 * or other allocating routine: its scratch is one fixed 32 MiB device array
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  Problems whose scratch (column exponents, task tables and
 * digit planes: about 2 * slices * roundup(m, 64) * (roundup(n, 128) + 128)
 * bytes) exceeds 32 MiB return ATA_ERR_UNSUPPORTED.
 *
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * Every call on a device shares the one array and leaves its contents behind
 * (the call clears what must start at zero): calls that overlap on the GPU
 * race, so serialise them (one stream, or events).  There is no handle and
 * no status word to read: a non-finite entry of A (ata_lower reports
 * ATA_ERR_INVALID at ata_sync) or a device-side wait that ran out leaves
 * every entry of low(C) NaN instead. */
int ata_lower_noalloc(int64_t m, int64_t n, const void *A, int64_t lda,
                      void *C, int64_t ldc, int dtype, void *stream);

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int ata_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ATA_H */
