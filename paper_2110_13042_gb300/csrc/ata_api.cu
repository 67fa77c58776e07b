// C ABI (include/ata.h): handle, argument validation, plan cache, device
// workspace, tensor maps and the launch sequence of one ata_lower call.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ata.h"
#include "kernels.h"
#include "plan.h"

using namespace ata;

namespace {

using Key = std::tuple<int64_t, int64_t, int64_t, int64_t, int, int, int, int, int, int>;

struct CachedPlan {
    Plan plan;
    std::vector<uint8_t> tables;
    uint8_t *pinned = nullptr;
    uint64_t ws_generation = 0;
    LeafParams lp;
    ~CachedPlan() {
        if (pinned) cudaFreeHost(pinned);
    }
};

// The plan and pinned task tables of the last batched call, re-used while
// the same shapes and configuration come back.  The host-array form patches
// the problem pointers into the pinned table when they change (after the
// previous upload from it has completed).
struct CachedBatch {
    std::vector<int64_t> key;
    std::vector<const void *> ptrs;   // host form: the A_i, C_i in the pinned table
    BatchPlan plan;
    uint8_t *pinned = nullptr;
    size_t table_bytes = 0;
    int64_t off_expo = 0, off_probs = 0, off_tasks = 0, off_planes = 0, total = 0;
    bool any_empty_m = false;         // some problem has m == 0 and n > 0 (zero fill)
    cudaEvent_t uploaded = nullptr;   // recorded after each uncaptured upload from `pinned`
    bool recorded = false;            // `uploaded` holds a record made outside a graph capture
    ~CachedBatch() {
        if (uploaded) {
            if (recorded) cudaEventSynchronize(uploaded);
            cudaEventDestroy(uploaded);
            cudaGetLastError();
        }
        if (pinned) cudaFreeHost(pinned);
    }
};

bool is_f32_mode(int dtype) { return dtype == ATA_F32 || dtype == ATA_F32_BF16 || dtype == ATA_F32_FP8; }

bool valid_dtype(int dtype) {
    return dtype == ATA_F64 || dtype == ATA_F64_EMU || dtype == ATA_F32 || dtype == ATA_F32_BF16 ||
           dtype == ATA_F32_FP8;
}

}  // namespace

struct ata_handle_s {
    int device = 0;
    int num_sms = 0;
    ata_config cfg{};
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    uint64_t ws_generation = 1;
    int *d_status = nullptr;
    const CachedPlan *resident = nullptr;  // whose tables are in the workspace
    std::map<Key, std::unique_ptr<CachedPlan>> plans;
    std::unique_ptr<CachedBatch> batch;
    // autotuned {cutoff, depth, strassen_min} per (m, n, dtype)
    std::map<std::tuple<int64_t, int64_t, int>, std::tuple<int, int, int>> tuned;
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // static partition (ata_config.streams > 1): the side streams of the leaf
    // groups, the fork event and one join event per stream
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    std::string last_error;
};

namespace {

constexpr int MAX_STREAMS = 16;

int ensure_side_streams(ata_handle h, size_t count) {
    if (!h->fork && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        h->fork = nullptr;
        return ATA_ERR_CUDA;
    }
    while (h->side.size() < count) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return ATA_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamDestroy(st);
            return ATA_ERR_CUDA;
        }
        h->side.push_back(st);
        h->join.push_back(ev);
    }
    return ATA_OK;
}

int check_config(const ata_config *c) {
    if (!c) return ATA_OK;
    if (c->cutoff < 0 || c->strassen_depth < -1 || c->strassen_depth > ATA_MAX_STRASSEN_DEPTH || c->slices < 0 ||
        c->slices > MAX_SLICES || c->strassen_min < 0 ||
        (c->strassen_variant != ATA_STRASSEN && c->strassen_variant != ATA_WINOGRAD) || c->streams < 0 ||
        c->streams > MAX_STREAMS || c->split_k < 0 || c->split_k > SPLITK_MAX)
        return ATA_ERR_INVALID;
    for (int r : c->reserved)
        if (r != 0) return ATA_ERR_INVALID;
    return ATA_OK;
}

PlanParams params_for(const ata_config &cfg, int64_t m, int64_t n, int64_t lda, int64_t ldc, int dtype) {
    PlanParams pp;
    pp.m = m;
    pp.n = n;
    pp.lda = lda;
    pp.ldc = ldc;
    pp.mode = dtype;
    pp.cutoff = cfg.cutoff;
    pp.depth = cfg.strassen_depth;
    pp.slices = cfg.slices;
    pp.strassen_min = cfg.strassen_min;
    pp.variant = cfg.strassen_variant;
    pp.streams = cfg.streams > 1 ? cfg.streams : 1;
    pp.split_k = cfg.split_k;
    return pp;
}

int fail(ata_handle h, int status, const char *step, cudaError_t e = cudaSuccess) {
    h->last_error = step;
    if (e != cudaSuccess) {
        h->last_error += ": ";
        h->last_error += cudaGetErrorString(e);
        cudaGetLastError();
    }
    return status;
}

// Grow the workspace to `bytes`.  A new workspace is zeroed on the call's
// stream, so the zeroing is ordered before the call's table upload and
// kernels whatever kind of stream the caller uses (cudaMemset would run on
// the legacy default stream, which a non-blocking stream does not wait for).
int ensure_workspace(ata_handle h, size_t bytes, cudaStream_t s) {
    if (bytes <= h->ws_bytes) return ATA_OK;
    const char *inj = std::getenv("ATA_TEST_FAIL_ALLOC");
    if (inj && inj[0] == '1') return ATA_ERR_ALLOC;
    if (h->ws) {
        if (cudaDeviceSynchronize() != cudaSuccess) return ATA_ERR_CUDA;
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 8;  // headroom for nearby shapes
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        want = bytes;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return ATA_ERR_ALLOC;
        }
    }
    if (cudaMemsetAsync(p, 0, want, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return ATA_ERR_CUDA;
    }
    h->ws = static_cast<uint8_t *>(p);
    h->ws_bytes = want;
    h->ws_generation++;
    h->resident = nullptr;
    return ATA_OK;
}

// Tensor maps and raw family pointers for the current workspace.
int bind_plan(ata_handle h, CachedPlan &cp) {
    if (cp.ws_generation == h->ws_generation) return ATA_OK;
    const Plan &P = cp.plan;
    LeafParams &lp = cp.lp;
    lp = LeafParams{};  // zeros, alpha = 1, beta = 0
    if (P.uses_digits()) {
        for (size_t f = 0; f < P.families.size(); ++f) {
            lp.fam_base[f] = h->ws + P.families[f].offset;
            lp.fam_ncb[f] = P.families[f].cols / BLOCK_COLS;
        }
    } else {
        for (size_t f = 0; f < P.families.size(); ++f) {
            lp.fam64[f] = reinterpret_cast<const double *>(h->ws + P.families[f].offset);
            lp.fam_ld[f] = P.families[f].cols;
        }
    }
    cp.ws_generation = h->ws_generation;
    if (h->resident == &cp) h->resident = nullptr;
    return ATA_OK;
}

// The handle's configuration, with an autotuned choice for (m, n, dtype)
// applied when cutoff, depth and strassen_min are all on auto.
ata_config effective_cfg(ata_handle h, int64_t m, int64_t n, int dtype) {
    ata_config c = h->cfg;
    if (c.cutoff == 0 && c.strassen_depth == -1 && c.strassen_min == 0) {
        auto it = h->tuned.find(std::make_tuple(m, n, dtype));
        if (it != h->tuned.end()) std::tie(c.cutoff, c.strassen_depth, c.strassen_min) = it->second;
    }
    return c;
}

CachedPlan *get_plan(ata_handle h, const PlanParams &pp, int *status) {
    Key key{pp.m, pp.n, pp.lda, pp.ldc, pp.mode, pp.cutoff, pp.depth, pp.slices, pp.strassen_min,
            pp.trans | (pp.packed << 1) | (pp.variant << 2) | (pp.streams << 8) | (pp.split_k << 16)};
    auto it = h->plans.find(key);
    if (it != h->plans.end()) return it->second.get();
    std::unique_ptr<CachedPlan> cp(new CachedPlan());
    std::string err;
    if (!make_plan(pp, &cp->plan, &err)) {
        *status = ATA_ERR_INVALID;
        return nullptr;
    }
    if (cp->plan.families.size() > static_cast<size_t>(MAX_FAMILIES)) {
        *status = ATA_ERR_UNSUPPORTED;
        return nullptr;
    }
    pack_tables(cp->plan, &cp->tables);
    if (!cp->tables.empty()) {
        if (cudaMallocHost(reinterpret_cast<void **>(&cp->pinned), cp->tables.size()) != cudaSuccess) {
            cudaGetLastError();
            *status = ATA_ERR_ALLOC;
            return nullptr;
        }
        std::memcpy(cp->pinned, cp->tables.data(), cp->tables.size());
    }
    if (h->plans.size() >= 8192) h->plans.clear(), h->resident = nullptr;  // bound the cache
    CachedPlan *raw = cp.get();
    h->plans[key] = std::move(cp);
    return raw;
}

bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bbytes && y < x + abytes;
}

}  // namespace

extern "C" {

int ata_version(void) { return 100; }

const char *ata_last_error(ata_handle h) { return h ? h->last_error.c_str() : ""; }

const char *ata_status_string(int status) {
    switch (status) {
        case ATA_OK: return "ok";
        case ATA_ERR_INVALID: return "invalid argument (dimension, leading dimension, pointer, overlap or non-finite input)";
        case ATA_ERR_DTYPE: return "unknown or unsupported dtype";
        case ATA_ERR_ALLOC: return "allocation failed";
        case ATA_ERR_CUDA: return "CUDA runtime or launch error";
        case ATA_ERR_TIMEOUT: return "a device-side wait exceeded its time budget";
        case ATA_ERR_UNSUPPORTED: return "unsupported device or size";
        default: return "unknown status";
    }
}

int ata_create(ata_handle *out, const ata_config *cfg) {
    if (!out) return ATA_ERR_INVALID;
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc != ATA_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ATA_ERR_UNSUPPORTED;
    }
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return ATA_ERR_UNSUPPORTED;
    }
    if (major != 10 || minor != 3) return ATA_ERR_UNSUPPORTED;
    ata_handle h = new (std::nothrow) ata_handle_s();
    if (!h) return ATA_ERR_ALLOC;
    h->device = dev;
    h->num_sms = sms;
    if (cfg) h->cfg = *cfg;
    else {
        std::memset(&h->cfg, 0, sizeof(h->cfg));
        h->cfg.strassen_depth = -1;
    }
    // the zeroed status word is complete before any call can use it, on any stream
    if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess || cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return ATA_ERR_ALLOC;
    }
    *out = h;
    return ATA_OK;
}

int ata_set_config(ata_handle h, const ata_config *cfg) {
    if (!h) return ATA_ERR_INVALID;
    int rc = check_config(cfg);
    if (rc != ATA_OK) return rc;
    if (cfg) h->cfg = *cfg;
    else {
        std::memset(&h->cfg, 0, sizeof(h->cfg));
        h->cfg.strassen_depth = -1;
    }
    return ATA_OK;
}

int ata_destroy(ata_handle h) {
    if (!h) return ATA_ERR_INVALID;
    cudaDeviceSynchronize();
    h->plans.clear();
    h->batch.reset();
    for (cudaEvent_t &e : h->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->join) cudaEventDestroy(e);
    for (cudaStream_t st : h->side) cudaStreamDestroy(st);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->ws) cudaFree(h->ws);
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return ATA_OK;
}

int ata_plan_info(ata_handle h, int64_t m, int64_t n, int dtype, int64_t *out) {
    if (!out) return ATA_ERR_INVALID;
    if (!valid_dtype(dtype)) return ATA_ERR_DTYPE;
    ata_config cfg{};
    cfg.strassen_depth = -1;
    if (h) cfg = effective_cfg(h, m, n, dtype);
    Plan P;
    std::string err;
    if (!make_plan(params_for(cfg, m, n, n > 0 ? n : 1, n > 0 ? n : 1, dtype), &P, &err))
        return ATA_ERR_INVALID;
    out[0] = P.cutoff;
    out[1] = P.depth;
    out[2] = P.slices;
    out[3] = P.n_panels;
    out[4] = P.n_blocks;
    out[5] = P.n_products;
    out[6] = P.n_tiles;
    out[7] = P.workspace_bytes;
    out[8] = static_cast<int64_t>(P.leaf_madds);
    out[9] = static_cast<int64_t>(P.plain_madds);
    out[10] = P.split_k;
    out[11] = P.n_fused;
    out[12] = static_cast<int64_t>(P.combs.size());
    return ATA_OK;
}

int ata_plan_blocks(ata_handle h, int64_t m, int64_t n, int dtype, int64_t *out, int64_t max_blocks,
                    int64_t *count) {
    if (!count || max_blocks < 0 || (max_blocks > 0 && !out)) return ATA_ERR_INVALID;
    if (!valid_dtype(dtype)) return ATA_ERR_DTYPE;
    ata_config cfg{};
    cfg.strassen_depth = -1;
    if (h) cfg = effective_cfg(h, m, n, dtype);
    Plan P;
    std::string err;
    if (!make_plan(params_for(cfg, m, n, n > 0 ? n : 1, n > 0 ? n : 1, dtype), &P, &err))
        return ATA_ERR_INVALID;
    *count = static_cast<int64_t>(P.blocks.size());
    for (int64_t i = 0; i < max_blocks && i < *count; ++i) {
        const BlockInfo &b = P.blocks[static_cast<size_t>(i)];
        int64_t *o = out + i * ATA_BLOCK_FIELDS;
        o[0] = b.r0;
        o[1] = b.p;
        o[2] = b.c0;
        o[3] = b.q;
        o[4] = b.depth;
    }
    return ATA_OK;
}

namespace {

// low(C) <- alpha low(X^T X) + beta low(C) with X = A (flags without
// ATA_TRANS) or X = A^T (ATA_TRANS: the product A A^T); A is m x n row-major.
// ata_lower: flags 0, alpha = 1, beta = 0.
int lower_impl(ata_handle h, int flags, int64_t m, int64_t n, double alpha, const void *A, int64_t lda,
               double beta, void *C, int64_t ldc, int dtype, void *stream) {
    if (!h) return ATA_ERR_INVALID;
    h->last_error.clear();
    cudaGetLastError();  // launch checks below report this call's launches only
    if (!valid_dtype(dtype)) return ATA_ERR_DTYPE;
    if (flags & ~(ATA_TRANS | ATA_PACKED)) return ATA_ERR_INVALID;
    if (m < 0 || n < 0) return ATA_ERR_INVALID;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return ATA_ERR_INVALID;
    const bool trans = (flags & ATA_TRANS) != 0, packed = (flags & ATA_PACKED) != 0;
    // the product X^T X: contraction length mm, output nn x nn
    const int64_t mm = trans ? n : m, nn = trans ? m : n;
    if (nn == 0) return ATA_OK;
    if ((!packed && ldc < nn) || !C) return ATA_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool f32 = is_f32_mode(dtype);
    const size_t es = f32 ? 4 : 8;
    const size_t c_bytes = (packed ? nn * (nn + 1) / 2 : (nn - 1) * ldc + nn) * es;
    if (mm == 0 || alpha == 0.0) {  // no product term: low(C) <- beta low(C)
        if (beta == 1.0) return ATA_OK;
        return launch_scale_lower(C, nn, ldc, f32, beta, s, packed) == cudaSuccess ? ATA_OK : ATA_ERR_CUDA;
    }
    if (lda < n || !A) return ATA_ERR_INVALID;
    if (ranges_overlap(A, ((m - 1) * lda + n) * es, C, c_bytes)) return ATA_ERR_INVALID;

    int status = ATA_OK;
    PlanParams pp = params_for(effective_cfg(h, mm, nn, dtype), mm, nn, lda, packed ? nn : ldc, dtype);
    pp.num_ctas = h->num_sms;
    pp.trans = trans ? 1 : 0;
    pp.packed = packed ? 1 : 0;
    CachedPlan *cp = get_plan(h, pp, &status);
    if (!cp) return status;
    const Plan &P = cp->plan;
    int rc = ensure_workspace(h, static_cast<size_t>(P.workspace_bytes), s);
    if (rc != ATA_OK) return rc;
    rc = bind_plan(h, *cp);
    if (rc != ATA_OK) return rc;
    if (h->resident != cp && P.table_bytes > 0) {
        cudaError_t ce = cudaMemcpyAsync(h->ws + P.off_tables, cp->pinned, P.table_bytes,
                                         cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) return fail(h, ATA_ERR_CUDA, "task-table upload", ce);
        if (P.f0_zero) {  // the planes of A's zero padding (see Plan::f0_zero)
            const Family &f0 = P.families[0];
            ce = cudaMemsetAsync(h->ws + f0.offset, 0, static_cast<size_t>(f0.plane_elems) * 2 * P.slices, s);
            if (ce != cudaSuccess) return fail(h, ATA_ERR_CUDA, "plane padding", ce);
        }
        h->resident = cp;
    }
    uint8_t *ws = h->ws;
    const uint8_t *tables = ws + P.off_tables;
    unsigned long long *colmax = reinterpret_cast<unsigned long long *>(ws + P.off_colmax);
    int *expo = reinterpret_cast<int *>(ws + P.off_expo);
    const bool need_expo = P.uses_digits() || !P.ops.empty();

    auto mark = [&](int i) {
        if (h->timing) cudaEventRecord(h->ev[i], s);
    };
    mark(0);
    cudaError_t e;
    if (need_expo && (e = launch_colmax(A, mm, nn, lda, f32, trans, colmax, expo, h->d_status, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "column-exponent launch", e);
    mark(1);
    if ((e = launch_prep(P, A, f32, expo, tables, ws, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "operand-prep launch", e);
    mark(2);

    LeafParams &lp = cp->lp;
    lp.tasks = reinterpret_cast<const LeafTask *>(tables + P.t_tasks);
    lp.ntasks = static_cast<int>(P.tasks.size());
    lp.C = C;
    lp.M = ws + P.off_products;
    lp.expo = expo;
    lp.status = h->d_status;
    lp.A64 = static_cast<const double *>(A);
    lp.lda = lda;
    lp.alpha = alpha;
    lp.beta = beta;
    lp.a_trans = trans ? 1 : 0;
    lp.packed = packed ? 1 : 0;
    if (P.groups.empty()) {
        e = P.uses_digits() ? launch_leaf_tc(P, lp, h->num_sms, s) : launch_leaf_f64(P, lp, s);
        if (e != cudaSuccess) return fail(h, ATA_ERR_CUDA, "leaf launch", e);
    } else {  // static partition: one leaf launch per group, each on its own stream
        if ((rc = ensure_side_streams(h, P.groups.size())) != ATA_OK) return fail(h, rc, "side streams");
        if ((e = cudaEventRecord(h->fork, s)) != cudaSuccess) return fail(h, ATA_ERR_CUDA, "fork event", e);
        for (size_t g = 0; g < P.groups.size(); ++g) {
            const LeafGroup &G = P.groups[g];
            cudaStream_t sg = h->side[g];
            if ((e = cudaStreamWaitEvent(sg, h->fork, 0)) != cudaSuccess) return fail(h, ATA_ERR_CUDA, "fork", e);
            e = P.uses_digits() ? launch_leaf_tc_group(P, lp, G.first, G.count, G.ctas, sg)
                                : launch_leaf_f64_group(lp, G.first, G.count, sg);
            if (e != cudaSuccess) return fail(h, ATA_ERR_CUDA, "leaf group launch", e);
            if ((e = cudaEventRecord(h->join[g], sg)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, h->join[g], 0)) != cudaSuccess)
                return fail(h, ATA_ERR_CUDA, "join", e);
        }
    }
    mark(3);
    if ((e = launch_combine(P, tables, ws + P.off_products, C, expo, alpha, beta, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "combine launch", e);
    mark(4);
    if (h->timing) h->timed = true;
    return ATA_OK;
}

}  // namespace

int ata_lower(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc,
              int dtype, void *stream) {
    return lower_impl(h, 0, m, n, 1.0, A, lda, 0.0, C, ldc, dtype, stream);
}

int ata_syrk(ata_handle h, int64_t m, int64_t n, double alpha, const void *A, int64_t lda, double beta, void *C,
             int64_t ldc, int dtype, void *stream) {
    return lower_impl(h, 0, m, n, alpha, A, lda, beta, C, ldc, dtype, stream);
}

int ata_syrk_ex(ata_handle h, int flags, int64_t m, int64_t n, double alpha, const void *A, int64_t lda,
                double beta, void *C, int64_t ldc, int dtype, void *stream) {
    return lower_impl(h, flags, m, n, alpha, A, lda, beta, C, ldc, dtype, stream);
}

int ata_lower_aat(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc,
                  int dtype, void *stream) {
    return lower_impl(h, ATA_TRANS, m, n, 1.0, A, lda, 0.0, C, ldc, dtype, stream);
}

int ata_tune(ata_handle h, int64_t m, int64_t n, const void *A, int64_t lda, void *C, int64_t ldc, int dtype,
             void *stream, double budget_ms, int64_t *out) {
    if (!h) return ATA_ERR_INVALID;
    if (!valid_dtype(dtype)) return ATA_ERR_DTYPE;
    if (m < 0 || n < 0) return ATA_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ata_config saved = h->cfg;
    const bool saved_timing = h->timing;
    h->timing = false;
    // Candidates, plain tiles first; plans that come out identical are
    // timed once.
    struct Cand {
        int cutoff, depth, smin;
    };
    std::vector<Cand> cands{{0, 0, 0}};
    for (int d = 1; d <= 3; ++d)
        for (int smin : {4096, 2048, 1024})
            for (int cut : {0, static_cast<int>(n / 8)}) cands.push_back({cut, d, smin});
    std::vector<std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>> seen;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return ATA_ERR_CUDA;
    }
    int rc = ATA_OK, timed = 0;
    float best_ms = -1.f, spent = 0.f;
    Cand best{0, 0, 0};
    for (const Cand &c : cands) {
        ata_config cfg = saved;
        cfg.cutoff = c.cutoff;
        cfg.strassen_depth = c.depth;
        cfg.strassen_min = c.smin;
        Plan P;
        std::string err;
        if (!make_plan(params_for(cfg, m, n, lda, ldc, dtype), &P, &err)) continue;
        if (c.depth > 0 && P.n_products == 0) continue;  // no block large enough
        // plan content, not the requested knobs (a depth the blocks cannot
        // reach plans the same as a smaller one)
        auto sig = std::make_tuple(P.n_products, P.n_tiles, P.n_blocks, P.n_panels,
                                   static_cast<int64_t>(P.ops.size()));
        bool dup = false;
        for (const auto &x : seen) dup = dup || x == sig;
        if (dup) continue;
        seen.push_back(sig);
        if (timed > 0 && spent > budget_ms) break;
        h->cfg = cfg;
        float ms = 0.f;
        for (int rep = 0; rep < 3 && rc == ATA_OK; ++rep) {  // first call warms (plan, workspace)
            if (rep > 0 && cudaEventRecord(e0, s) != cudaSuccess) rc = ATA_ERR_CUDA;
            if (rc == ATA_OK) rc = ata_lower(h, m, n, A, lda, C, ldc, dtype, stream);
            if (rc == ATA_OK && rep > 0) {
                float t = 0.f;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                    rc = ATA_ERR_CUDA;
                ms = rep == 1 ? t : std::min(ms, t);
                spent += t;
            }
        }
        if (rc != ATA_OK) break;
        ++timed;
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->cfg = saved;
    h->timing = saved_timing;
    if (rc != ATA_OK) return rc;
    h->tuned[std::make_tuple(m, n, dtype)] = std::make_tuple(best.cutoff, best.depth, best.smin);
    // leave C holding the product of the chosen configuration
    rc = ata_lower(h, m, n, A, lda, C, ldc, dtype, stream);
    if (rc != ATA_OK) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ATA_ERR_CUDA;
    if (out) {
        out[0] = best.cutoff;
        out[1] = best.depth;
        out[2] = best.smin;
        out[3] = timed;
    }
    return ATA_OK;
}

int ata_tune_clear(ata_handle h) {
    if (!h) return ATA_ERR_INVALID;
    h->tuned.clear();
    return ATA_OK;
}

int ata_set_timing(ata_handle h, int enable) {
    if (!h) return ATA_ERR_INVALID;
    if (enable && !h->ev[0]) {
        for (cudaEvent_t &e : h->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return ATA_ERR_CUDA;
    }
    h->timing = enable != 0;
    h->timed = false;
    return ATA_OK;
}

int ata_phase_times(ata_handle h, double *out) {
    if (!h || !out || !h->timing || !h->timed) return ATA_ERR_INVALID;
    if (cudaEventSynchronize(h->ev[4]) != cudaSuccess) return ATA_ERR_CUDA;
    for (int i = 0; i < 4; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) != cudaSuccess) return ATA_ERR_CUDA;
        out[i] = ms;
    }
    return ATA_OK;
}

}  // extern "C"

namespace {

// Batched calls.  Host form: A_host / C_host are host arrays of device
// pointers (written into the problem table on the host).  Device form:
// A_dev / C_dev are device arrays of device pointers, copied into the problem
// table by a kernel when the call runs, so a captured graph picks up
// whatever the arrays hold at replay time.
int batched_impl(ata_handle h, int count, const int64_t *m, const int64_t *n, const void *const *A_host,
                 const int64_t *lda, void *const *C_host, const int64_t *ldc, const void *const *A_dev,
                 void *const *C_dev, int dtype, void *stream) {
    if (!h || count < 0) return ATA_ERR_INVALID;
    h->last_error.clear();
    cudaGetLastError();  // launch checks below report this call's launches only
    if (count == 0) return ATA_OK;
    const bool dev = A_dev != nullptr || C_dev != nullptr;
    if (!m || !n || !lda || !ldc || (dev ? (!A_dev || !C_dev) : (!A_host || !C_host))) return ATA_ERR_INVALID;
    if (!valid_dtype(dtype)) return ATA_ERR_DTYPE;
    if (dtype == ATA_F64 || dtype == ATA_F32_FP8)
        return fail(h, ATA_ERR_UNSUPPORTED, "batched calls take F64_EMU, F32 or F32_BF16");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool f32 = is_f32_mode(dtype);
    const size_t es = f32 ? 4 : 8;
    for (int i = 0; i < count; ++i) {
        if (m[i] < 0 || n[i] < 0) return ATA_ERR_INVALID;
        if (n[i] == 0) continue;
        if (ldc[i] < n[i]) return ATA_ERR_INVALID;
        if (m[i] > 0 && lda[i] < n[i]) return ATA_ERR_INVALID;
        if (m[i] > MAX_DIGIT_K) return fail(h, ATA_ERR_UNSUPPORTED, "contraction beyond the exact-accumulation limit");
        if (dev) continue;  // device pointers are not visible here
        if (!C_host[i]) return ATA_ERR_INVALID;
        if (m[i] == 0) continue;
        if (!A_host[i]) return ATA_ERR_INVALID;
        if (ranges_overlap(A_host[i], ((m[i] - 1) * lda[i] + n[i]) * es, C_host[i], ((n[i] - 1) * ldc[i] + n[i]) * es))
            return ATA_ERR_INVALID;
    }

    // Plan (and its pinned tables) for this problem set: shapes only.
    std::vector<int64_t> key;
    key.reserve(4 + 4 * static_cast<size_t>(count));
    key.push_back(dtype);
    key.push_back(h->cfg.slices);
    key.push_back(h->num_sms);
    key.push_back(count);
    for (int i = 0; i < count; ++i) {
        key.push_back(m[i]);
        key.push_back(n[i]);
        key.push_back(lda[i]);
        key.push_back(ldc[i]);
    }
    if (!h->batch || h->batch->key != key) {
        h->batch.reset();
        std::unique_ptr<CachedBatch> cb(new (std::nothrow) CachedBatch());
        if (!cb) return ATA_ERR_ALLOC;
        std::string err;
        if (!make_batch_plan(dtype, h->cfg.slices, h->num_sms, count, m, n, lda, ldc, nullptr, nullptr, &cb->plan,
                             &err))
            return fail(h, ATA_ERR_INVALID, err.c_str());
        const BatchPlan &B = cb->plan;
        auto align = [](int64_t x) { return (x + 1023) & ~int64_t(1023); };
        const int64_t probs_bytes = static_cast<int64_t>(B.probs.size() * sizeof(BatchProb));
        const int64_t tasks_bytes = static_cast<int64_t>(B.tasks.size() * sizeof(LeafTask));
        cb->off_expo = 0;
        cb->off_probs = align(B.total_cols * 4);
        cb->off_tasks = cb->off_probs + align(probs_bytes);
        cb->off_planes = cb->off_tasks + align(tasks_bytes);
        cb->total = cb->off_planes + align(B.plane_bytes);
        cb->table_bytes = static_cast<size_t>(cb->off_planes - cb->off_probs);
        for (int i = 0; i < count; ++i) cb->any_empty_m = cb->any_empty_m || (m[i] == 0 && n[i] > 0);
        if (cudaMallocHost(reinterpret_cast<void **>(&cb->pinned), cb->table_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, ATA_ERR_ALLOC, "pinned batch tables");
        }
        if (cudaEventCreateWithFlags(&cb->uploaded, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, ATA_ERR_CUDA, "batch upload event");
        }
        std::memset(cb->pinned, 0, cb->table_bytes);
        std::memcpy(cb->pinned, B.probs.data(), static_cast<size_t>(probs_bytes));
        std::memcpy(cb->pinned + (cb->off_tasks - cb->off_probs), B.tasks.data(), static_cast<size_t>(tasks_bytes));
        cb->key.swap(key);
        h->batch = std::move(cb);
    }
    CachedBatch &cb = *h->batch;
    const BatchPlan &B = cb.plan;
    if (!dev) {  // patch the problem pointers into the pinned table when they changed
        bool same = cb.ptrs.size() == 2 * static_cast<size_t>(count);
        for (int i = 0; same && i < count; ++i) same = cb.ptrs[2 * i] == A_host[i] && cb.ptrs[2 * i + 1] == C_host[i];
        if (!same) {
            if (cb.recorded && cudaEventSynchronize(cb.uploaded) != cudaSuccess)
                return fail(h, ATA_ERR_CUDA, "batch table reuse");
            BatchProb *pp = reinterpret_cast<BatchProb *>(cb.pinned);
            cb.ptrs.resize(2 * static_cast<size_t>(count));
            for (int i = 0; i < count; ++i) {
                pp[i].A = A_host[i];
                pp[i].C = C_host[i];
                cb.ptrs[2 * i] = A_host[i];
                cb.ptrs[2 * i + 1] = C_host[i];
            }
        }
    }
    int rc = ensure_workspace(h, static_cast<size_t>(cb.total), s);
    if (rc != ATA_OK) return fail(h, rc, "workspace");
    h->resident = nullptr;  // the batch overwrites the single-call tables
    uint8_t *ws = h->ws;
    BatchProb *probs = reinterpret_cast<BatchProb *>(ws + cb.off_probs);
    int *expo = reinterpret_cast<int *>(ws + cb.off_expo);
    cudaError_t e = cudaMemcpyAsync(ws + cb.off_probs, cb.pinned, cb.table_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(h, ATA_ERR_CUDA, "table upload", e);
    // Remember the upload (to wait for it before the pinned table is
    // rewritten) only outside a graph capture: a captured upload belongs to
    // the graph, and an event recorded in a capture cannot be waited on.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return fail(h, ATA_ERR_CUDA, "capture status", e);
    if (cap == cudaStreamCaptureStatusNone) {
        if ((e = cudaEventRecord(cb.uploaded, s)) != cudaSuccess) return fail(h, ATA_ERR_CUDA, "table upload event", e);
        cb.recorded = true;
    }
    // phase events (ata_set_timing): exponents, digit prep, leaf; no combine
    auto mark = [&](int i) {
        if (h->timing) cudaEventRecord(h->ev[i], s);
    };
    if (dev && (e = launch_batched_ptrs(probs, count, A_dev, C_dev, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "batched pointer gather", e);
    if (cb.any_empty_m && (e = launch_batched_zero(probs, count, f32, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "zero fill", e);
    mark(0);
    if ((e = launch_batched_expo(B, probs, f32, expo, h->d_status, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "batched exponents", e);
    mark(1);
    if ((e = launch_batched_prep(B, probs, f32, expo, ws + cb.off_planes, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "batched digit prep", e);
    mark(2);
    LeafParams lp;
    lp = LeafParams{};  // zeros, alpha = 1, beta = 0
    lp.tasks = reinterpret_cast<const LeafTask *>(ws + cb.off_tasks);
    lp.ntasks = static_cast<int>(B.tasks.size());
    lp.expo = expo;
    lp.status = h->d_status;
    lp.probs = probs;
    lp.batch_planes = ws + cb.off_planes;
    if ((e = launch_leaf_tc_raw(B.slices, lp, lp.ntasks, h->num_sms, s)) != cudaSuccess)
        return fail(h, ATA_ERR_CUDA, "batched leaf", e);
    mark(3);
    mark(4);
    if (h->timing) h->timed = true;
    return ATA_OK;
}

}  // namespace

extern "C" {

int ata_batched(ata_handle h, int count, const int64_t *m, const int64_t *n, const void *const *A,
                const int64_t *lda, void *const *C, const int64_t *ldc, int dtype, void *stream) {
    return batched_impl(h, count, m, n, A, lda, C, ldc, nullptr, nullptr, dtype, stream);
}

int ata_batched_dev(ata_handle h, int count, const int64_t *m, const int64_t *n, const void *const *A_dev,
                    const int64_t *lda, void *const *C_dev, const int64_t *ldc, int dtype, void *stream) {
    if (!A_dev || !C_dev) return count == 0 && h ? ATA_OK : ATA_ERR_INVALID;
    return batched_impl(h, count, m, n, nullptr, lda, nullptr, ldc, A_dev, C_dev, dtype, stream);
}
int ata_check_wait_timeout(ata_handle h, int64_t budget_ns, void *stream) {
    if (!h || budget_ns < 1000 || budget_ns > 10000000000LL) return ATA_ERR_INVALID;
    cudaError_t e = launch_wait_check(h->d_status, static_cast<unsigned long long>(budget_ns),
                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ATA_OK : fail(h, ATA_ERR_CUDA, "wait self-test launch", e);
}

int ata_sync(ata_handle h, void *stream) {
    if (!h) return ATA_ERR_INVALID;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return ATA_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ATA_ERR_CUDA;
    if (st != 0 && (cudaMemsetAsync(h->d_status, 0, sizeof(int), static_cast<cudaStream_t>(stream)) != cudaSuccess ||
                    cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess))
        return ATA_ERR_CUDA;
    return st;
}

}  // extern "C"
