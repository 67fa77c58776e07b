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

cudaError_t launch_colmax(const void *A, int64_t m, int64_t n, int64_t lda, bool is_f32,
                          unsigned long long *colmax, int *expo, int *status, cudaStream_t s);
cudaError_t launch_prep(const Plan &P, const void *A, bool is_f32, const int *expo,
                        const uint8_t *tables, uint8_t *ws, cudaStream_t s);
cudaError_t launch_leaf_tc(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s);
cudaError_t launch_leaf_f64(const Plan &P, const LeafParams &lp, cudaStream_t s);
cudaError_t launch_combine(const Plan &P, const uint8_t *tables, const void *M, void *C,
                           const int *expo, double alpha, double beta, cudaStream_t s);
// low(C) <- beta * low(C) (beta == 0: zeros, C not read).
cudaError_t launch_scale_lower(void *C, int64_t n, int64_t ldc, bool is_f32, double beta, cudaStream_t s);
// Launches from explicit tables (allocation-free entry point).
cudaError_t launch_prep_digits_raw(int slices, const void *A, bool is_f32, int64_t lda, const int *expo,
                                   const OpDesc *ops, int nops, const OpTerm *terms, const Family &fam0,
                                   int64_t prep_tiles, uint8_t *ws, cudaStream_t s);
cudaError_t launch_leaf_tc_raw(int slices, const LeafParams &lp, int ntasks, int num_sms, cudaStream_t s);
// Shared-memory bytes the tcgen05 leaf kernel needs for `slices` digits.
int leaf_tc_smem_bytes(int slices);

}  // namespace ata
