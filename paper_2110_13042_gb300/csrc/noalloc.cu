// ata_lower_noalloc: low(C) <- low(A^T A) without any memory allocation.
//
// Some callers cannot allocate device memory at the point they need the
// product: code running inside a CUDA-graph capture they do not control, a
// host framework with its own memory pool that forbids side allocations, or an
// embedded/real-time service that must not call cudaMalloc after start-up.
// This entry point serves them with a fixed, statically sized scratch array
// (a file-scope __device__ array; every GPU that loads the library holds it
// until the process exits).  It runs the plain tiled split-digit path (no
// Strassen, no recursion): column exponents, digit planes, tcgen05 leaf tiles.
// Its task tables are generated on the device, so it needs no host upload.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "ata.h"
#include "kernels.h"
#include "plan.h"

namespace ata {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB per device
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Scratch layout for one call (byte offsets, 1 KB aligned).
struct Layout {
    int64_t status, colmax, expo, ops, terms, tasks, planes, total;
    int64_t ntasks, prep_tiles;
    Family fam;
};

__host__ __device__ inline int64_t panel_tiles(int64_t J, int64_t n);

int64_t count_tiles(int64_t n) {
    int64_t t = 0;
    for (int64_t J = 0; J < ceil_div(n, TILE_M); ++J) t += panel_tiles(J, n);
    return t;
}

// Digit-plane bytes alone (the largest part of the scratch), in closed form.
int64_t plane_bytes(int64_t m, int64_t n, int slices) {
    return round_up(m, PREP_K) * (round_up(n, TILE) + TILE) * 2 * slices;
}

Layout layout_for(int64_t m, int64_t n, int slices) {
    Layout L{};
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        const int64_t o = off;
        off += round_up(bytes > 0 ? bytes : 0, 1024);
        return o;
    };
    L.ntasks = count_tiles(n);
    L.status = take(64);
    L.colmax = take(n * 8);
    L.expo = take(n * 4);
    L.ops = take(sizeof(OpDesc));
    L.terms = take(sizeof(OpTerm));
    L.tasks = take(L.ntasks * static_cast<int64_t>(sizeof(LeafTask)));
    L.fam.K_pitch = round_up(m, PREP_K);
    const int64_t p_pad = round_up(n, TILE);
    L.fam.cols = p_pad + TILE;
    L.fam.plane_elems = L.fam.cols * L.fam.K_pitch;
    L.planes = take(L.fam.plane_elems * 2 * slices);
    L.fam.offset = L.planes;
    L.prep_tiles = prep_tiles_for(true, L.fam.K_pitch, p_pad);
    L.total = off;
    return L;
}

// Lower-triangle tiles of row panel J (TILE_M rows starting at J * TILE_M) of
// an n x n product: columns blocks K with K * TILE_N < n that reach the
// diagonal, i.e. K * TILE_N <= J * TILE_M + rows - 1.
__host__ __device__ inline int64_t panel_tiles(int64_t J, int64_t n) {
    const int64_t rows = n - J * TILE_M < TILE_M ? n - J * TILE_M : TILE_M;
    const int64_t nk = (n + TILE_N - 1) / TILE_N;
    const int64_t reach = (J * TILE_M + rows - 1) / TILE_N + 1;
    return reach < nk ? reach : nk;
}

// The operand table and the lower-triangle tile list (the same tiles, in the
// same order, as the planner's single diagonal panel).  Block J writes the
// tiles of row panel J at the offset given by the tile counts of the panels
// before it (summed by the block's threads), one tile per thread; block 0
// also writes the operand descriptor.
__global__ void __launch_bounds__(128) noalloc_tables_kernel(int64_t m, int64_t n, int64_t ldc, int kind, int hbits,
                                                             int64_t K_pitch, OpDesc *op, OpTerm *term,
                                                             LeafTask *tasks) {
    __shared__ int64_t part[4];
    const int64_t J = blockIdx.x;
    if (J == 0 && threadIdx.x == 0) {
        OpTerm tm{};
        tm.row0 = 0;
        tm.col0 = 0;
        tm.rows = static_cast<int32_t>(m);
        tm.cols = static_cast<int32_t>(n);
        tm.coef = 1;
        *term = tm;
        OpDesc od{};
        od.family = 0;
        od.t_shift = 0;
        od.nterms = 1;
        od.first_term = 0;
        od.out_col = 0;
        od.K_pitch = static_cast<int32_t>(K_pitch);
        od.P_pad = static_cast<int32_t>(((n + TILE - 1) / TILE) * TILE);
        od.tile_base = 0;
        *op = od;
    }
    int64_t before = 0;
    for (int64_t j = threadIdx.x; j < J; j += blockDim.x) before += panel_tiles(j, n);
    for (int off = 16; off > 0; off >>= 1) before += __shfl_down_sync(0xffffffffu, before, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = before;
    __syncthreads();
    const int64_t base = part[0] + part[1] + part[2] + part[3];
    const int64_t r0 = J * TILE_M;
    const int64_t rows = n - r0 < TILE_M ? n - r0 : TILE_M;
    for (int64_t K = threadIdx.x; K < panel_tiles(J, n); K += blockDim.x) {
        const int64_t c0 = K * TILE_N;
        const int64_t cols = n - c0 < TILE_N ? n - c0 : TILE_N;
        LeafTask lt{};
        lt.fam_u = 0;
        lt.fam_v = 0;
        lt.col_u = static_cast<int32_t>(r0);
        lt.col_v = static_cast<int32_t>(c0);
        lt.k0 = 0;
        lt.klen = static_cast<int32_t>(m);
        lt.rows = static_cast<int32_t>(rows);
        lt.cols = static_cast<int32_t>(cols);
        lt.diag = (c0 + cols - 1 > r0) ? 1 : 0;
        lt.diag_off = static_cast<int32_t>(r0 - c0);
        lt.kind = kind;
        lt.shift = 0;
        lt.eu = static_cast<int32_t>(r0);
        lt.ev = static_cast<int32_t>(c0);
        lt.out_off = r0 * ldc + c0;
        lt.out_ld = ldc;
        lt.hbits = hbits;
        tasks[base + K] = lt;
    }
}

// Non-finite input (flagged in the status word by the column-exponent pass)
// or a device wait that ran out (flagged by the leaf): low(C) becomes NaN, so
// the caller sees the failure without a status read.
template <typename T>
__global__ void __launch_bounds__(256) nan_if_flagged_kernel(const int *status, T *C, int64_t n, int64_t ldc) {
    if (*status == 0) return;
    const T nan = static_cast<T>(__longlong_as_double(0x7FF8000000000000LL));
    const int64_t total = n * n;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j = i / n, k = i - j * n;
        if (k <= j) C[j * ldc + k] = nan;
    }
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_for_current_device(uint8_t **out, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ATA_ERR_UNSUPPORTED;
    }
    if (dev < 0 || dev >= MAX_DEVICES) return ATA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        int major = 0, minor = 0, n = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return ATA_ERR_UNSUPPORTED;
        }
        if (major != 10 || minor != 3) return ATA_ERR_UNSUPPORTED;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ATA_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_num_sms[dev] = n;
    }
    *out = static_cast<uint8_t *>(g_scratch_addr[dev]);
    *sms = g_num_sms[dev];
    return ATA_OK;
}

}  // namespace
}  // namespace ata

using namespace ata;

extern "C" int ata_lower_noalloc(int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc, int dtype,
                                 void *stream) {
    if (dtype != ATA_F64_EMU && dtype != ATA_F32 && dtype != ATA_F32_BF16) return ATA_ERR_DTYPE;
    if (m < 0 || n < 0) return ATA_ERR_INVALID;
    if (n == 0) return ATA_OK;
    if (ldc < n || !C) return ATA_ERR_INVALID;
    const bool f32 = dtype != ATA_F64_EMU;
    const size_t es = f32 ? 4 : 8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m == 0) return launch_scale_lower(C, n, ldc, f32, 0.0, s) == cudaSuccess ? ATA_OK : ATA_ERR_CUDA;
    if (lda < n || !A) return ATA_ERR_INVALID;
    {
        const uintptr_t a = reinterpret_cast<uintptr_t>(A), c = reinterpret_cast<uintptr_t>(C);
        const uintptr_t ab = static_cast<uintptr_t>(((m - 1) * lda + n) * es);
        const uintptr_t cb = static_cast<uintptr_t>(((n - 1) * ldc + n) * es);
        if (a < c + cb && c < a + ab) return ATA_ERR_INVALID;
    }
    if (m > MAX_DIGIT_K || n > (int64_t(1) << 30)) return ATA_ERR_UNSUPPORTED;
    const int slices = default_slices(dtype, m);
    // closed-form rejection first: the exact layout counts every tile
    if (plane_bytes(m, n, slices) > static_cast<int64_t>(NOALLOC_SCRATCH_BYTES)) return ATA_ERR_UNSUPPORTED;
    const Layout L = layout_for(m, n, slices);
    if (static_cast<size_t>(L.total) > NOALLOC_SCRATCH_BYTES) return ATA_ERR_UNSUPPORTED;

    uint8_t *ws = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&ws, &sms);
    if (rc != ATA_OK) return rc;

    int *status = reinterpret_cast<int *>(ws + L.status);
    unsigned long long *colmax = reinterpret_cast<unsigned long long *>(ws + L.colmax);
    int *expo = reinterpret_cast<int *>(ws + L.expo);
    OpDesc *ops = reinterpret_cast<OpDesc *>(ws + L.ops);
    OpTerm *terms = reinterpret_cast<OpTerm *>(ws + L.terms);
    LeafTask *tasks = reinterpret_cast<LeafTask *>(ws + L.tasks);

    // The scratch keeps the previous call's contents: the status word starts
    // at zero (colmax is cleared by its own launch).
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return ATA_ERR_CUDA;
    noalloc_tables_kernel<<<static_cast<unsigned>(ceil_div(n, TILE_M)), 128, 0, s>>>(
        m, n, ldc, f32 ? OUT_C_F32 : OUT_C_F64, hbits_for(m), L.fam.K_pitch, ops, terms, tasks);
    if (cudaGetLastError() != cudaSuccess) return ATA_ERR_CUDA;
    if (launch_colmax(A, m, n, lda, f32, false, colmax, expo, status, s) != cudaSuccess) return ATA_ERR_CUDA;
    if (launch_prep_digits_raw(slices, A, f32, lda, expo, ops, 1, terms, L.fam, L.prep_tiles, ws, s) !=
        cudaSuccess)
        return ATA_ERR_CUDA;
    LeafParams lp;
    lp = LeafParams{};  // zeros, alpha = 1, beta = 0
    lp.fam_base[0] = ws + L.fam.offset;
    lp.fam_ncb[0] = L.fam.cols / BLOCK_COLS;
    lp.tasks = tasks;
    lp.ntasks = static_cast<int>(L.ntasks);
    lp.C = C;
    lp.M = nullptr;
    lp.expo = expo;
    lp.status = status;
    if (launch_leaf_tc_raw(slices, lp, static_cast<int>(L.ntasks), sms, s) != cudaSuccess) return ATA_ERR_CUDA;
    const unsigned nb = static_cast<unsigned>(std::min<int64_t>(ceil_div(n * n, 256), 4 * static_cast<int64_t>(sms)));
    if (f32)
        nan_if_flagged_kernel<float><<<nb, 256, 0, s>>>(status, static_cast<float *>(C), n, ldc);
    else
        nan_if_flagged_kernel<double><<<nb, 256, 0, s>>>(status, static_cast<double *>(C), n, ldc);
    if (cudaGetLastError() != cudaSuccess) return ATA_ERR_CUDA;
    return ATA_OK;
}
