// Launch wrappers for the device kernels (host side).  All launches are
// asynchronous on `stream` and return the launch's cudaError_t.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "plan.h"

namespace ata {

// Parameters shared by the leaf launches.
struct LeafParams {
    const uint8_t *fam_base[MAX_FAMILIES];  // digit families (1 KB images)
    int64_t fam_ncb[MAX_FAMILIES];          // column blocks per family
    const LeafTask *tasks;
    int ntasks;
    int pad0;
    void *C;            // output matrix (double or float)
    void *M;            // product workspace (int64 or double)
    const int *expo;    // column exponents of A
    int *status;        // device status word
    const double *A64;  // native FP64: A itself
    int64_t lda;
    const double *fam64[MAX_FAMILIES];  // native FP64: family arrays
    int64_t fam_ld[MAX_FAMILIES];
    const BatchProb *probs;             // batched calls: problem table (else null)
    const uint8_t *batch_planes;        // batched calls: base of all problems' planes
    double alpha = 1.0;                 // stores into C: alpha * product + beta * C
    double beta = 0.0;                  // (beta == 0: C is not read)
    int a_trans = 0;                    // native FP64 tiles reading A: element (i, j) at A[j * lda + i]
    int packed = 0;                     // C is a packed lower triangle (tasks: out_off = row, out_ld = col)
};

// Column exponents e_j (smallest e with max_i |a_ij| < 2^e); flags a
// non-finite column in *status.
// Batched calls: column exponents of every problem (one block per problem
// and 256-column chunk), and the digit planes of every problem (persistent
// grid over all prep tiles).  probs is the device copy of the plan's table.
cudaError_t launch_batched_expo(const BatchPlan &B, const BatchProb *probs, bool is_f32, int *expo, int *status,
                                cudaStream_t s);
cudaError_t launch_batched_prep(const BatchPlan &B, const BatchProb *probs, bool is_f32, const int *expo,
                                uint8_t *planes, cudaStream_t s);
// Batched calls with device-resident pointer arrays: copy A_i, C_i into the
// device problem table.  And low(C_i) <- 0 for every problem with m_i == 0.
cudaError_t launch_batched_ptrs(BatchProb *probs, int64_t count, const void *const *A, void *const *C,
                                cudaStream_t s);
cudaError_t launch_batched_zero(const BatchProb *probs, int64_t count, bool is_f32, cudaStream_t s);

// trans: the m x n operand is the transpose of the row-major n x m array A
// (element (i, j) at A[j * lda + i]); its column exponents are row maxima of A.
cudaError_t launch_colmax(const void *A, int64_t m, int64_t n, int64_t lda, bool is_f32, bool trans,
                          unsigned long long *colmax, int *expo, int *status, cudaStream_t s);
cudaError_t launch_prep(const Plan &P, const void *A, bool is_f32, const int *expo,
                        const uint8_t *tables, uint8_t *ws, cudaStream_t s);
cudaError_t launch_leaf_tc(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s);
cudaError_t launch_leaf_f64(const Plan &P, const LeafParams &lp, cudaStream_t s);
// One group of a static partition (Plan::groups): tasks [first, first + count).
cudaError_t launch_leaf_tc_group(const Plan &P, const LeafParams &lp, int64_t first, int64_t count, int ctas,
                                 cudaStream_t s);
cudaError_t launch_leaf_f64_group(const LeafParams &lp, int64_t first, int64_t count, cudaStream_t s);
cudaError_t launch_combine(const Plan &P, const uint8_t *tables, const void *M, void *C,
                           const int *expo, double alpha, double beta, cudaStream_t s);
// low(C) <- beta * low(C) (beta == 0: zeros, C not read); packed: C is a
// packed lower triangle (ldc unused).
cudaError_t launch_scale_lower(void *C, int64_t n, int64_t ldc, bool is_f32, double beta, cudaStream_t s,
                               bool packed = false);
// Launches from explicit tables (allocation-free entry point).
cudaError_t launch_prep_digits_raw(int slices, const void *A, bool is_f32, int64_t lda, const int *expo,
                                   const OpDesc *ops, int nops, const OpTerm *terms, const Family &fam0,
                                   int64_t prep_tiles, uint8_t *ws, cudaStream_t s);
cudaError_t launch_leaf_tc_raw(int slices, const LeafParams &lp, int ntasks, int num_sms, cudaStream_t s);
// Self-test of the bounded device wait (a barrier nothing completes).
cudaError_t launch_wait_check(int *status, unsigned long long budget_ns, cudaStream_t s);
// Shared-memory bytes the tcgen05 leaf kernel needs for `slices` digits.
int leaf_tc_smem_bytes(int slices);

}  // namespace ata
