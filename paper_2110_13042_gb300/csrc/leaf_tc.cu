// tcgen05 leaf engine: every 128 x 96 output tile of every leaf product
// (diagonal panels, classical tiles, Strassen products) in one persistent
// launch.
//
// Arithmetic (split-digit emulation of a wide product on BF16 tensor cores):
// each operand column is a fixed-point number written as S balanced digits,
//   u = 2^-8 sum_q x_q 2^(-9 (q - 1)),  |x_1| <= 256, x_q in [-256, 255],
// stored in BF16 as x_q 2^(-9 (q - 1)) (exact).  The digit products
// x_p y_q 2^(-9 (p + q - 2)) (|x_p y_q| <= 2^16) are summed by the tensor core
// into FP32 accumulators in TMEM; products with the same p + q share one:
//   acc0: p + q = 2 (1 pair)   |partial| <= 1 * 256 * 2^16 = 2^24 (256 rows)
//   acc1: p + q = 3 (2 pairs)  |partial| <= 2 * 128 * 2^16 = 2^24 (128 rows)
//   acc2: p + q = 4 (3 pairs)  |partial| <= 3 *  64 * 2^16 < 2^24  (64 rows)
//   acc3: p + q = 5 (4 pairs)  |partial| <= 4 *  64 * 2^16 = 2^24  (64 rows)
//   acc4: p + q >= 6 (the rest, weight <= 2^-36 of acc0's unit; not exact)
// Each of acc0..acc3 holds integers (in its unit) of magnitude <= 2^24, which
// FP32 represents exactly, and is drained at the interval shown into a
// per-element int64 sum T in units of 2^-(27 + h) (acc4 is rounded to that
// unit); h = min(9, 19 - log2 K) extra bits keep short contractions as
// accurate as long ones.  The tile's value is T * 2^(-43 - h + shift + e_row + e_col).
//
// Tile 128 x 96: five 96-column FP32 accumulators fit the 512 TMEM columns.
// One digit (FP8, and one BF16 digit when every contraction is at most
// ONE_DIGIT_WIDE_MAX_K rows): tile 128 x 192, whose single accumulator has two
// 192-column buffers, filled and drained in turn by alternate 16-step chunks;
// these leaves are bound by operand delivery, and the wide tile moves 10 KB
// per K step instead of 2 x 7 KB for the same work.  One BF16 digit keeps its
// exact sums in 32 bits there (at most 2^24 per 256-row chunk).
// K step 16 (one MMA per digit pair per stage, 32-byte swizzle) keeps stages
// small, so 4-10 of them are in flight.
//
// Pipeline (one CTA per SM, persistent over a static round-robin task list):
//   warp 0       TMA producer: per stage and digit, one bulk copy of the
//                operand rows' 4 KB (A) and 3 KB (B) pre-swizzled images.
//   warp 1       TMEM allocator + single-thread tcgen05.mma issuer; with
//                5+ digits warps 1, 2, 3 each issue the MMAs of their own
//                accumulators ({4}, {0, 1}, {2, 3}).
//   warps 4..15  epilogue: tcgen05.ld drains, int64 accumulation, stores
//                (3 warps per TMEM lane quadrant, 32 columns each).
//   (16 warps keep the 4 SM sub-partitions balanced at 4 warps each, a
//    budget of 128 registers per thread; warps 2, 3 are idle below 5 digits.)
// The issuers and the epilogue visit the accumulators in the same fixed order
// (4, 0, 1, 2, 3): the ones drained every chunk come last, so the tensor core
// keeps working on the others while they are drained.
// The tensor core queues only a few instructions, so every instruction an
// issuing thread spends between MMAs can idle it (measured: the issuing
// thread, not memory or the MMA rate, bounds the leaf).  Steps with no
// accumulator pending or fresh take a branch-free path that merges pairs
// with adjacent accumulators of the same issuer into N = 192 MMAs; up to 3
// digits the bookkeeping runs once per multi-step stage.
// All mbarrier waits are bounded (ptx.cuh).
#include <cuda_bf16.h>
#include <cstdint>
#include <type_traits>

#include "fixconv.h"
#include "kernels.h"
#include "ptx.cuh"

namespace ata {
namespace {

constexpr int NUM_THREADS = 512;
constexpr int EPI_WARP0 = 4;
constexpr int NUM_EPI = 384;                          // 12 epilogue warps, 3 per lane quadrant
constexpr int EPI_COLS = TILE_N / 3;                  // 32 columns per epilogue thread
constexpr int A_SLICE_BYTES = TILE_M * KSTEP * 2;     // 4 KB
constexpr int B_SLICE_BYTES = TILE_N * KSTEP * 2;     // 3 KB
constexpr int MAX_ACC = 5;
constexpr int MAX_STAGES = 10;
constexpr uint32_t IDESC = idesc_bf16_f32(TILE_M, TILE_N);
constexpr uint32_t IDESC2 = idesc_bf16_f32(TILE_M, 2 * TILE_N);
constexpr uint32_t IDESC8 = idesc_e4m3_f32(TILE_M, TILE_N8);  // the FP8 mode's 128 x 192 tile

// W1: one BF16 digit on the wide 128 x 192 tile with 32-bit sums (plans
// whose leaf contractions are at most ONE_DIGIT_WIDE_MAX_K rows).
template <int S, bool F8 = false, bool W1 = false>
struct Cfg {
    // Tile columns (one-digit wide tiles: 192, TILE_N8), the B slice of one
    // K step (32-byte rows: 16 BF16 or 32 E4M3 values) and the columns each
    // epilogue thread owns (a third of the tile).
    static constexpr int TN = (F8 || W1) ? TILE_N8 : TILE_N;
    static constexpr int B_SLICE = TN * 32;
    static constexpr int EPI = TN / 3;
    // K steps per pipeline stage.  Up to 3 digits the issuing thread does
    // its bookkeeping once per stage (see the issuer), so longer stages pay:
    // measured at 8192^2, one digit 8 steps (-38% leaf time against 1-step
    // bookkeeping), two and three digits 4 steps (-24% / -19%, although only
    // 2-4 stages fit).  From 4 digits on, drains fall inside 16-step spans
    // and every step is a stage.  FP8 (twice the work per step): 4 steps.
    static constexpr int KPS = (F8 || W1) ? 4 : S == 1 ? 8 : S <= 3 ? 4 : 1;
    static constexpr int STEP_BYTES = S * (A_SLICE_BYTES + B_SLICE);
    static constexpr int STAGE_BYTES = KPS * STEP_BYTES;
    static constexpr int STAGES_FIT = 229000 / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT < MAX_STAGES ? STAGES_FIT : MAX_STAGES;
    static constexpr int NACC = S >= MAX_ACC ? MAX_ACC : S;
    // One digit: two TMEM buffers for the one accumulator, used by
    // alternate drain chunks, so the tensor core fills one while the
    // epilogue drains the other (with one buffer every drain idled it).
    static constexpr int NBUF = S == 1 ? 2 : NACC;
    static constexpr int TMEM_COLS = NBUF * TN <= 128 ? 128 : NBUF * TN <= 256 ? 256 : 512;
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + BAR_BYTES;
    static_assert(STAGES >= 2, "pipeline depth");
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
    static_assert(NBUF * TN <= TMEM_COLS, "TMEM budget");
    static_assert(EPI % 16 == 0, "16-column TMEM loads");
};

__host__ __device__ constexpr int acc_of(int p, int q) {
    return (p + q - 2) < MAX_ACC - 1 ? (p + q - 2) : MAX_ACC - 1;
}

// Accumulators due for draining at the end of 64-row chunk `c`.  The most
// frequently drained accumulator present is in every non-empty mask.
// With at most 3 digits (the FP32 modes, whose stated bound is 5e-5 or the
// one-digit rounding bound) only acc0 must stay exact: acc1 and acc2 (weights
// 2^-9 and 2^-18) are drained with it every 256 rows, where they stay below
// 2^31 in their units (2 and 3 pairs x 256 rows x 2^16) so the 32-bit
// conversion still applies, and their FP32 rounding is ~2^-33 relative.
__device__ __forceinline__ uint32_t due_mask(int c, bool last, int nacc) {
    if (nacc <= 3) return ((c & 3) == 3 || last) ? (1u << nacc) - 1u : 0u;
    uint32_t m = (1u << 2) | (1u << 3);             // acc2, acc3 every chunk
    if ((c & 1) == 1 || last) m |= 1u << 1;          // acc1 every 2 chunks
    if ((c & 3) == 3 || last) m |= 1u | (1u << 4);   // acc0, acc4 every 4 chunks
    return m & ((1u << nacc) - 1u);
}

struct Shared {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t accf[3];  // due accumulators handed to the epilogue, one barrier per issuer
    uint64_t acce[MAX_ACC];
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ void spin_ns(unsigned long long ns) {
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < ns) {
    }
}

// Element offset in C of column 0 of tile row `row`: row-major C, or a packed
// lower triangle (entry (j, k) at j (j + 1) / 2 + k; the task then holds the
// tile's first row and column in out_off / out_ld).
__device__ __forceinline__ int64_t c_row_offset(const LeafTask &t, int row, int packed) {
    if (packed) {
        const int64_t j = t.out_off + row;
        return j * (j + 1) / 2 + t.out_ld;
    }
    return t.out_off + static_cast<int64_t>(row) * t.out_ld;
}

// 16-byte vector stores and loads of C / M values.
__device__ __forceinline__ void st16(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st16(int64_t *p, const int64_t (&v)[2]) {
    *reinterpret_cast<longlong2 *>(p) = make_longlong2(v[0], v[1]);
}
__device__ __forceinline__ void ld16(const float *p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
}
__device__ __forceinline__ void ld16(const double *p, double (&v)[2]) {
    const double2 x = *reinterpret_cast<const double2 *>(p);
    v[0] = x.x, v[1] = x.y;
}
__device__ __forceinline__ void ld16(const int64_t *, int64_t (&v)[2]) { v[0] = v[1] = 0; }  // (never scaled)
// alpha * v + beta * old, as store_scaled computes it
__device__ __forceinline__ float scaled_val(float v, float old, double alpha, double beta) {
    const float r = static_cast<float>(alpha) * v;
    return beta != 0.0 ? fmaf(static_cast<float>(beta), old, r) : r;
}
__device__ __forceinline__ double scaled_val(double v, double old, double alpha, double beta) {
    const double r = alpha * v;
    return beta != 0.0 ? fma(beta, old, r) : r;
}
__device__ __forceinline__ int64_t scaled_val(int64_t v, int64_t, double, double) { return v; }

// Write columns [colbase, colbase + EC) of one tile row, those below lim:
// out[colbase + i] = val(i) (SCALED: alpha * val(i) + beta * out, the old
// value read only when beta != 0).  A thread owns a row, so each warp store
// instruction touches 32 rows of C; 16-byte vectors (where the row segment is
// 16-byte aligned and the whole vector lies below lim) cut those instructions
// two- to fourfold.  Other columns are written one at a time.
template <int EC, bool SCALED, typename O, typename F>
__device__ __forceinline__ void store_row(O *out, int colbase, int lim, const F &val, double alpha, double beta) {
    constexpr int VW = 16 / static_cast<int>(sizeof(O));
    static_assert(EC % VW == 0, "whole vectors");
    const bool vec = (reinterpret_cast<uintptr_t>(out + colbase) & 15u) == 0;
#pragma unroll
    for (int g = 0; g < EC; g += VW) {
        O *dst = out + colbase + g;
        if (vec && colbase + g + VW <= lim) {
            O v[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) v[j] = val(g + j);
            if constexpr (SCALED) {
                if (alpha != 1.0 || beta != 0.0) {  // (alpha = 1, beta = 0 store v as it is)
                    O old[VW];
                    if (beta != 0.0) {
                        ld16(dst, old);
                    } else {
#pragma unroll
                        for (int j = 0; j < VW; ++j) old[j] = O(0);
                    }
#pragma unroll
                    for (int j = 0; j < VW; ++j) v[j] = scaled_val(v[j], old[j], alpha, beta);
                }
            }
            st16(dst, v);
        } else {
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                if (colbase + g + j < lim) {
                    if constexpr (SCALED)
                        store_scaled(dst + j, val(g + j), alpha, beta);
                    else
                        dst[j] = val(g + j);
                }
            }
        }
    }
}

__device__ __forceinline__ double exp2d(int x) {
    if (x >= -1022 && x <= 1023) return __longlong_as_double(static_cast<long long>(x + 1023) << 52);
    return scalbn(1.0, x);
}
__device__ __forceinline__ float exp2f_(int x) {
    if (x >= -126 && x <= 127) return __uint_as_float(static_cast<unsigned>(x + 127) << 23);
    return scalbnf(1.0f, x);
}
// v * 2^x: one multiply while 2^x is a normal number, else scalbn (one
// exact scaling and a single rounding, where 2^x alone would under- or
// overflow although v * 2^x need not: tiny or subnormal columns).
__device__ __forceinline__ double scale2d(double v, int x) {
    return (x >= -1022 && x <= 1023) ? v * exp2d(x) : scalbn(v, x);
}
__device__ __forceinline__ float scale2f(float v, int x) {
    return (x >= -126 && x <= 127) ? v * exp2f_(x) : scalbnf(v, x);
}

// All digit pairs (P, Q) of accumulator ACC, unrolled at compile time.  The
// shared-memory descriptors of digit P / Q differ from the stage's first by
// the slice offset (in 16-byte units of the start-address field).
template <int S, int ACC, int P = 1, int Q = 1>
__device__ __forceinline__ void issue_pairs(uint32_t d_tmem, uint64_t da0, uint64_t db0, uint32_t &accum) {
    if constexpr (P <= S) {
        if constexpr (P + Q <= S + 1) {
            if constexpr (acc_of(P, Q) == ACC) {
                umma_f16(d_tmem, da0 + static_cast<uint64_t>((P - 1) * (A_SLICE_BYTES >> 4)),
                         db0 + static_cast<uint64_t>((Q - 1) * (B_SLICE_BYTES >> 4)), IDESC, accum);
                accum = 1u;
            }
            issue_pairs<S, ACC, P, Q + 1>(d_tmem, da0, db0, accum);
        } else {
            issue_pairs<S, ACC, P + 1, 1>(d_tmem, da0, db0, accum);
        }
    }
}

// Accumulators 2 and 3 are the ones drained every 64 rows.
__host__ __device__ constexpr bool in_b(int acc) { return acc == 2 || acc == 3; }

// Several issuing threads (5+ digits): the issuer that owns an accumulator.
// Two: {4, 0, 1}, {2, 3}.  Three: {4}, {0, 1}, {2, 3}.
template <int NI>
__host__ __device__ constexpr int issuer_of(int acc) {
    return NI == 2 ? (in_b(acc) ? 1 : 0) : (acc == 4 ? 0 : (acc <= 1 ? 1 : 2));
}
template <int NI>
__host__ __device__ constexpr uint32_t issuer_mask(int g) {
    uint32_t m = 0;
    for (int a = 0; a < MAX_ACC; ++a)
        if (issuer_of<NI>(a) == g) m |= 1u << a;
    return m;
}

// Every pair whose accumulator belongs to issuer G, with (p, q), (p, q + 1)
// sharing one N = 192 MMA when their accumulators are adjacent and both G's.
template <int S, int NI, int G, int P = 1, int Q = 1>
__device__ __forceinline__ void issue_own(uint32_t tmem, uint64_t da0, uint64_t db0) {
    if constexpr (P <= S) {
        if constexpr (P + Q <= S + 1) {
            constexpr int ACC = acc_of(P, Q);
            constexpr bool has_next = P + Q + 1 <= S + 1;
            constexpr int NEXT = has_next ? acc_of(P, Q + 1) : -1;
            constexpr bool own = issuer_of<NI>(ACC) == G;
            constexpr bool merge = own && has_next && NEXT == ACC + 1 && issuer_of<NI>(NEXT) == G;
            const uint64_t da = da0 + static_cast<uint64_t>((P - 1) * (A_SLICE_BYTES >> 4));
            const uint64_t db = db0 + static_cast<uint64_t>((Q - 1) * (B_SLICE_BYTES >> 4));
            if constexpr (own) umma_f16(tmem + ACC * TILE_N, da, db, merge ? IDESC2 : IDESC, 1u);
            issue_own<S, NI, G, P, Q + (merge ? 2 : 1)>(tmem, da0, db0);
        } else {
            issue_own<S, NI, G, P + 1, 1>(tmem, da0, db0);
        }
    }
}

// With at most 4 digits every K step takes one path (no first-write case:
// the epilogue zeroes an accumulator when it drains it), in two groups.
// Group A (GB = false): pairs whose accumulator is 0, 1 or 4, with (p, q),
// (p, q + 1) sharing one N = 192 MMA when both accumulators are adjacent in
// TMEM and outside {2, 3}.  Group B (GB = true): pairs into acc2 / acc3, each
// merged with its right neighbour when adjacent.  The issuer waits for the
// drains of group A's accumulators before it, and of 2 and 3 only before
// group B, so that drain overlaps group A.  (Measured: 6-11% faster for 1-4
// digits.  With 5-7 digits one issuing thread cannot keep the pipe busy, and
// the accumulators are split over several issuers instead: issue_own above.)
template <int S, bool GB, int P = 1, int Q = 1>
__device__ __forceinline__ void issue_group(uint32_t tmem, uint64_t da0, uint64_t db0) {
    if constexpr (P <= S) {
        if constexpr (P + Q <= S + 1) {
            constexpr int ACC = acc_of(P, Q);
            constexpr bool has_next = P + Q + 1 <= S + 1;
            constexpr int NEXT = has_next ? acc_of(P, Q + 1) : -1;
            constexpr bool merge = has_next && NEXT == ACC + 1 && in_b(ACC) == in_b(NEXT);
            const uint64_t da = da0 + static_cast<uint64_t>((P - 1) * (A_SLICE_BYTES >> 4));
            const uint64_t db = db0 + static_cast<uint64_t>((Q - 1) * (B_SLICE_BYTES >> 4));
            if constexpr (in_b(ACC) == GB) umma_f16(tmem + ACC * TILE_N, da, db, merge ? IDESC2 : IDESC, 1u);
            issue_group<S, GB, P, Q + (merge ? 2 : 1)>(tmem, da0, db0);
        } else {
            issue_group<S, GB, P + 1, 1>(tmem, da0, db0);
        }
    }
}

struct IssueState {
    uint32_t acce_phase;  // bit a: parity of the next acce[a] wait
    uint32_t pending;     // bit a: accumulator a handed to the epilogue
    uint32_t fresh;       // bit a: next MMA into a overwrites
};

// Wait until the epilogue has drained every accumulator in `mask`.
template <int NACC>
__device__ __forceinline__ bool wait_drained(IssueState &st, uint32_t mask, Shared *sh, volatile int *abort_flag,
                                             int *status) {
    mask &= st.pending;
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
        const uint32_t bit = 1u << a;
        if (mask & bit) {
            if (!mbar_wait(&sh->acce[a], (st.acce_phase >> a) & 1u, abort_flag, status)) return false;
            st.acce_phase ^= bit;
            st.pending &= ~bit;
        }
    }
    tc_fence_after();
    return true;
}

template <int S, int ACC>
__device__ __forceinline__ bool step_acc(IssueState &st, Shared *sh, uint32_t tmem, uint64_t da0,
                                         uint64_t db0, volatile int *abort_flag, int *status) {
    if constexpr (ACC >= Cfg<S, false>::NACC) {
        return true;
    } else {
        constexpr uint32_t bit = 1u << ACC;
        if (st.pending & bit) {
            if (!mbar_wait(&sh->acce[ACC], (st.acce_phase >> ACC) & 1u, abort_flag, status)) return false;
            st.acce_phase ^= bit;
            st.pending &= ~bit;
            tc_fence_after();
        }
        uint32_t accum = (st.fresh & bit) ? 0u : 1u;
        issue_pairs<S, ACC>(tmem + ACC * TILE_N, da0, db0, accum);
        st.fresh &= ~bit;
        return true;
    }
}

// Slow step of issuer G: its accumulators in the order 4, 0, 1, 2, 3.
template <int S, int NI, int G>
__device__ __forceinline__ bool step_own(IssueState &st, Shared *sh, uint32_t tmem, uint64_t da0, uint64_t db0,
                                         volatile int *abort_flag, int *status) {
    return (issuer_of<NI>(4) != G || step_acc<S, 4>(st, sh, tmem, da0, db0, abort_flag, status)) &&
           (issuer_of<NI>(0) != G || step_acc<S, 0>(st, sh, tmem, da0, db0, abort_flag, status)) &&
           (issuer_of<NI>(1) != G || step_acc<S, 1>(st, sh, tmem, da0, db0, abort_flag, status)) &&
           (issuer_of<NI>(2) != G || step_acc<S, 2>(st, sh, tmem, da0, db0, abort_flag, status)) &&
           (issuer_of<NI>(3) != G || step_acc<S, 3>(st, sh, tmem, da0, db0, abort_flag, status));
}

// T += a * b as one 32 x 32 -> 64-bit signed multiply-add instruction (on
// the multiply-add pipe: no integer-ALU shift or carry chain).
__device__ __forceinline__ void mad_wide(int64_t &t, int32_t a, int32_t b) {
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(t) : "r"(a), "r"(b));
}

// Add one drained accumulator (16 columns) into T, kept in units of
// 2^-(27 + h) of the leading digit product (h extra bits for short K).  The
// scaled value x is an exact integer (|x| <= 2^24).  Three equivalent forms
// (bit-identical T), chosen by measurement:
//   FORM 0: x << s added to T (integer-ALU shift and 64-bit add);
//   FORM 1: x * 2^s + T as one widening multiply-add written in C++ (s <= 30
//           for acc1..acc3): fewer instructions where drains dominate (S <= 3);
//   FORM 2: every accumulator as mad.wide.s32 (x rescaled so both factors fit
//           32 bits), no integer-ALU work: the three-issuer path (5-7 digits),
//           where the drains' ALU work delays the issuers (leaf -1.4 to -1.9 %
//           at 8192^2; FORM 1 spilled there, and FORM 2 is 2-3 % slower below 4
//           digits).
template <int ACC, int FORM>
__device__ __forceinline__ void absorb(int64_t *T, const uint32_t (&r)[16], int h, float fold_scale) {
    if constexpr (FORM == 2) {
        // x = round(v 2^c) exact with |x| <= 2^30, s = (27 + h) - c <= 30:
        // acc0 c = 6 (|v| <= 2^24), acc1..3 their unit (c = 9, 18, 27), acc4
        // the fold scale (s = 0).
        constexpr int C = ACC == 0 ? 6 : ACC == 1 ? 9 : ACC == 2 ? 18 : ACC == 3 ? 27 : 0;
        const int32_t mul = ACC == 4 ? 1 : (1 << (27 - C + h));
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float v = __uint_as_float(r[i]);
            const int32_t x = __float2int_rn(ACC == 4 ? v * fold_scale : v * static_cast<float>(1 << C));
            mad_wide(T[i], x, mul);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float v = __uint_as_float(r[i]);
        if (ACC == 0) {
            T[i] += static_cast<int64_t>(__float2int_rn(v)) << (27 + h);
        } else if (ACC == 4) {
            // |acc4| * 2^(27 + h) < 2^27 (p + q >= 6 terms over <= 256 rows,
            // h <= 9), so the 32-bit conversion is exact in range; the
            // 64-bit one runs at a small fraction of its rate.
            T[i] += static_cast<int64_t>(__float2int_rn(v * fold_scale));
        } else {
            constexpr float sc = ACC == 1 ? 512.0f : ACC == 2 ? 262144.0f : 134217728.0f;
            constexpr int s0 = ACC == 1 ? 18 : ACC == 2 ? 9 : 0;
            const int x = __float2int_rn(v * sc);
            if constexpr (FORM == 1)
                T[i] += static_cast<int64_t>(x) * static_cast<int64_t>(1 << (s0 + h));
            else
                T[i] += static_cast<int64_t>(x) << (s0 + h);
        }
    }
}

// Drain one accumulator: both TMEM loads are issued before a single wait,
// and the accumulator is handed back to the MMA issuer before the (longer)
// conversion work.
// ZERO: also clear what was read, so the next MMA into ACC accumulates onto
// zero (the grouped issue path of S <= 4).
// buf: the one-digit accumulator's TMEM buffer (0 for every other case).
template <int ACC, int FORM, bool ZERO>
__device__ __forceinline__ void drain_one(int64_t (&T)[EPI_COLS], uint32_t tbase, int colbase, Shared *sh,
                                          int h, float fold_scale, int buf = 0) {
    static_assert(EPI_COLS == 32, "two 16-column loads");
    const uint32_t col = static_cast<uint32_t>((ACC + buf) * TILE_N + colbase);
    uint32_t r0[16], r1[16];
    tmem_ld_32x32b_x16(tbase + col, r0);
    tmem_ld_32x32b_x16(tbase + col + 16, r1);
    tmem_ld_wait();
    if constexpr (ZERO) {
        tmem_st_zero_32x32b_x16(tbase + col);
        tmem_st_zero_32x32b_x16(tbase + col + 16);
        tmem_st_wait();
    }
    tc_fence_before();
    mbar_arrive(&sh->acce[ACC + buf]);
    absorb<ACC, FORM>(T, r0, h, fold_scale);
    absorb<ACC, FORM>(T + 16, r1, h, fold_scale);
}

// FP8 mode: drain the single accumulator (FP32 partial sums of E4M3
// products over the chunk) from TMEM buffer `buf` into the thread's FP32
// sums (its EC columns of the 192-column tile), zeroing what it read.
template <int EC>
__device__ __forceinline__ void drain_f8(float (&T)[EC], uint32_t tbase, int colbase, Shared *sh, int buf) {
    const uint32_t col = static_cast<uint32_t>(buf * TILE_N8 + colbase);
    uint32_t r[EC / 16][16];
#pragma unroll
    for (int g = 0; g < EC / 16; ++g) tmem_ld_32x32b_x16(tbase + col + 16 * g, r[g]);
    tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < EC / 16; ++g) tmem_st_zero_32x32b_x16(tbase + col + 16 * g);
    tmem_st_wait();
    tc_fence_before();
    mbar_arrive(&sh->acce[buf]);
#pragma unroll
    for (int g = 0; g < EC / 16; ++g)
#pragma unroll
        for (int i = 0; i < 16; ++i) T[16 * g + i] += __uint_as_float(r[g][i]);
}

// One BF16 digit on the wide tile: drain the accumulator (exact integer
// digit-product sums of at most 2^24 over the 256-row chunk) from TMEM
// buffer `buf` into the thread's 32-bit sums, zeroing what it read.
template <int EC>
__device__ __forceinline__ void drain_w1(int32_t (&T)[EC], uint32_t tbase, int colbase, Shared *sh, int buf) {
    const uint32_t col = static_cast<uint32_t>(buf * TILE_N8 + colbase);
    uint32_t r[EC / 16][16];
#pragma unroll
    for (int g = 0; g < EC / 16; ++g) tmem_ld_32x32b_x16(tbase + col + 16 * g, r[g]);
    tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < EC / 16; ++g) tmem_st_zero_32x32b_x16(tbase + col + 16 * g);
    tmem_st_wait();
    tc_fence_before();
    mbar_arrive(&sh->acce[buf]);
#pragma unroll
    for (int g = 0; g < EC / 16; ++g)
#pragma unroll
        for (int i = 0; i < 16; ++i) T[16 * g + i] += __float2int_rn(__uint_as_float(r[g][i]));
}

// F8: one E4M3 plane per operand (S == 1), K steps of 32 rows, FP32 sums.
// W1: one BF16 digit on the 128 x 192 tile, 32-bit exact sums.
template <int S, bool F8 = false, bool W1 = false>
__global__ void __launch_bounds__(NUM_THREADS, 1) leaf_tc_kernel(const __grid_constant__ LeafParams p) {
    using C = Cfg<S, F8, W1>;
    static_assert(!F8 || S == 1, "the FP8 mode has one plane");
    static_assert(!W1 || (S == 1 && !F8), "wide 32-bit sums: one BF16 digit");
    constexpr int KS = F8 ? KSTEP8 : KSTEP;  // contraction rows per K step
    // 5+ digits: three issuing threads (warps 1, 2, 3) owning accumulators
    // {4}, {0, 1}, {2, 3} (issuer_of), so a drain wait stalls only the issuer
    // of the accumulator being drained while the others keep the tensor core
    // fed, and the per-step bookkeeping is split between them.  Measured at
    // 8192^2, S = 6: one issuer 9.81 ms, two 8.87-8.98, three 8.19.
    constexpr bool MULTI = S >= 5;
    constexpr int NI = MULTI ? 3 : 1;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Shared *sh = reinterpret_cast<Shared *>(smem + C::STAGES * C::STAGE_BYTES);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], NI);  // every issuer releases the stage
        }
        for (int g = 0; g < 3; ++g) mbar_init(&sh->accf[g], 1);
        for (int a = 0; a < MAX_ACC; ++a) mbar_init(&sh->acce[a], NUM_EPI);
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&sh->tmem_base, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort_flag = &sh->abort_flag;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
                const LeafTask t = p.tasks[ti];
                const int nsteps = (t.klen + KS - 1) / KS;
                // Digit images: ((kstep * S + digit) * ncb + column block) KB; the
                // tile's TILE_M (TILE_N) columns are 4 (3) consecutive blocks.
                const uint8_t *ubase = p.fam_base[t.fam_u], *vbase = p.fam_base[t.fam_v];
                int64_t uncb = p.fam_ncb[t.fam_u], vncb = p.fam_ncb[t.fam_v];
                if (p.probs) {  // batched: both operands are the planes of problem t.prob
                    const BatchProb &bp = p.probs[t.prob];
                    ubase = vbase = p.batch_planes + bp.plane_off;
                    uncb = vncb = bp.ncb;
                }
                const uint8_t *ua = ubase + static_cast<int64_t>(t.col_u / BLOCK_COLS) * BLOCK_BYTES;
                const uint8_t *vb = vbase + static_cast<int64_t>(t.col_v / BLOCK_COLS) * BLOCK_BYTES;
                const int64_t ua_step = uncb * BLOCK_BYTES;  // per digit plane
                const int64_t vb_step = vncb * BLOCK_BYTES;
                for (int s0 = 0; s0 < nsteps; s0 += C::KPS) {
                    const int cnt = nsteps - s0 < C::KPS ? nsteps - s0 : C::KPS;
                    if (!mbar_wait(&sh->empty[stage], phase ^ 1u, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->full[stage], cnt * C::STEP_BYTES);
                    for (int kk = 0; kk < cnt; ++kk) {
                        uint8_t *a_dst = smem + stage * C::STAGE_BYTES + kk * C::STEP_BYTES;
                        uint8_t *b_dst = a_dst + S * A_SLICE_BYTES;
                        const int64_t ku = (t.k0 / KS) + s0 + kk, kv = (t.k0v / KS) + s0 + kk;
#pragma unroll
                        for (int q = 0; q < S; ++q) {
                            bulk_load(a_dst + q * A_SLICE_BYTES, ua + (ku * S + q) * ua_step, A_SLICE_BYTES,
                                      &sh->full[stage]);
                            bulk_load(b_dst + q * C::B_SLICE, vb + (kv * S + q) * vb_step, C::B_SLICE,
                                      &sh->full[stage]);
                        }
                    }
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) spin_ns(2000000);  // let copies already in flight land
        }
    } else if (MULTI && warp >= 1 && warp <= NI) {
        // ------------------------------------- NI MMA issuers (5+ digits) --
        if (lane == 0) {
            const int g = warp - 1;
            const uint32_t mine = g == 0 ? issuer_mask<NI>(0) : g == 1 ? issuer_mask<NI>(1) : issuer_mask<NI>(2);
            uint64_t *my_accf = &sh->accf[g];
            int stage = 0;
            uint32_t phase = 0;
            IssueState st{0u, 0u, mine};  // every accumulator starts fresh
            bool ok = true;
            const uint32_t smem_base = smem_u32(smem);
            for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
                const int nsteps = (p.tasks[ti].klen + KS - 1) / KS;
                for (int step = 0; step < nsteps; ++step) {
                    if (!mbar_wait(&sh->full[stage], phase, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = smem_base + stage * C::STAGE_BYTES;
                    const uint64_t da0 = sdesc_kmajor_sw32(a_base);
                    const uint64_t db0 = sdesc_kmajor_sw32(a_base + S * A_SLICE_BYTES);
                    if (((st.pending | st.fresh) & mine) == 0u) {
                        if (g == 0)
                            issue_own<S, NI, 0>(tmem, da0, db0);
                        else if (g == 1)
                            issue_own<S, NI, 1>(tmem, da0, db0);
                        else
                            issue_own<S, NI, 2>(tmem, da0, db0);
                    } else {
                        ok = g == 0   ? step_own<S, NI, 0>(st, sh, tmem, da0, db0, abort_flag, p.status)
                             : g == 1 ? step_own<S, NI, 1>(st, sh, tmem, da0, db0, abort_flag, p.status)
                                      : step_own<S, NI, 2>(st, sh, tmem, da0, db0, abort_flag, p.status);
                    }
                    if (!ok) break;
                    const bool last = step == nsteps - 1;
                    const uint32_t due = (last || (step % CHUNK_STEPS) == CHUNK_STEPS - 1)
                                             ? due_mask(step / CHUNK_STEPS, last, C::NACC) & mine
                                             : 0u;
                    if (due) {  // hand this issuer's due accumulators to the epilogue
                        umma_commit(my_accf);
                        st.pending |= due;
                        st.fresh |= due;
                    }
                    umma_commit(&sh->empty[stage]);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) spin_ns(2000000);  // let MMAs already issued retire
        }
    } else if (!MULTI && warp == 1) {
        // ------------------------------------- one MMA issuer (1-4 digits) --
        if constexpr (!MULTI) {
            if (lane == 0) {
                int stage = 0;
                uint32_t phase = 0;
                // every accumulator starts out with the epilogue, which zeroes it
                // (grouped issue path, see issue_group)
                IssueState st{0u, (1u << C::NBUF) - 1u, 0u};
                bool ok = true;
                bool ready = false;  // the current stage's full barrier was already seen complete
                int dbuf = 0;        // one digit: the accumulator buffer of the current drain chunk
                const uint32_t smem_base = smem_u32(smem);
                for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
                    const int nsteps = (p.tasks[ti].klen + KS - 1) / KS;
                    for (int s0 = 0; s0 < nsteps; s0 += C::KPS) {
                        const int cnt = nsteps - s0 < C::KPS ? nsteps - s0 : C::KPS;
                        if (!ready && !mbar_wait(&sh->full[stage], phase, abort_flag, p.status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        // Up to 3 digits, probe the next stage now (the test's
                        // latency hides behind this stage's MMA issue); with one
                        // step per stage (4+ digits) it measured 1% slower at 6.
                        if constexpr (S <= 3) {
                            const int nstage = stage + 1 == C::STAGES ? 0 : stage + 1;
                            const uint32_t nphase = nstage == 0 ? phase ^ 1u : phase;
                            ready = mbar_test_wait(&sh->full[nstage], nphase);
                        }
                        if constexpr (S <= 3) {
                            static_assert((4 * CHUNK_STEPS) % C::KPS == 0, "every 16-step drain point ends a stage");
                            // At most 3 digits: every accumulator is drained every
                            // 16 steps, at the end of a stage, so the drain waits
                            // come before the stage's first step and the due check
                            // after its last; the stage's MMAs go out back to back
                            // from descriptors built once.  (Per-step bookkeeping
                            // in the issuing thread measured ~275 cycles against a
                            // 56-cycle MMA; the pipe idles meanwhile.)
                            const uint32_t a_base = smem_base + stage * C::STAGE_BYTES;
                            const uint64_t da0 = sdesc_kmajor_sw32(a_base);
                            const uint64_t db0 = sdesc_kmajor_sw32(a_base + S * A_SLICE_BYTES);
                            // one digit: only the current buffer must be drained
                            const uint32_t need_a = S == 1 ? (1u << dbuf) : ~0x0Cu;
                            const uint32_t tacc = S == 1 ? tmem + static_cast<uint32_t>(dbuf * C::TN) : tmem;
#pragma unroll
                            for (int kk = 0; kk < C::KPS; ++kk) {
                                if (kk < cnt) {
                                    const uint64_t off = static_cast<uint64_t>(kk * (C::STEP_BYTES >> 4));
                                    if (kk == 0 && (st.pending & need_a)) {
                                        ok = wait_drained<C::NBUF>(st, need_a, sh, abort_flag, p.status);
                                        if (!ok) break;
                                    }
                                    if constexpr (F8)
                                        umma_f8(tacc, da0 + off, db0 + off, IDESC8, 1u);
                                    else if constexpr (W1)
                                        umma_f16(tacc, da0 + off, db0 + off, IDESC2, 1u);  // N = 192
                                    else
                                        issue_group<S, false>(tacc, da0 + off, db0 + off);
                                    if (kk == 0 && (st.pending & 0x0Cu)) {
                                        ok = wait_drained<C::NACC>(st, 0x0Cu, sh, abort_flag, p.status);
                                        if (!ok) break;
                                    }
                                    issue_group<S, true>(tmem, da0 + off, db0 + off);
                                }
                            }
                            if (!ok) break;
                            const int end = s0 + cnt;  // drains fall on 16-step boundaries and task ends
                            const uint32_t due =
                                (end % (4 * CHUNK_STEPS) == 0 || end >= nsteps)
                                    ? due_mask((end - 1) / CHUNK_STEPS, end >= nsteps, C::NACC)
                                    : 0u;
                            if (due) {  // hand the accumulators to the epilogue
                                if constexpr (S == 1) {  // each buffer has its own barrier
                                    umma_commit(&sh->accf[dbuf]);
                                    st.pending |= 1u << dbuf;
                                    dbuf ^= 1;
                                } else {
                                    umma_commit(&sh->accf[0]);
                                    st.pending |= due;
                                }
                            }
                        } else {
                            for (int kk = 0; kk < cnt; ++kk) {
                                const int step = s0 + kk;
                                const uint32_t a_base = smem_base + stage * C::STAGE_BYTES + kk * C::STEP_BYTES;
                                const uint64_t da0 = sdesc_kmajor_sw32(a_base);
                                const uint64_t db0 = sdesc_kmajor_sw32(a_base + S * A_SLICE_BYTES);
                                if (st.pending & ~0x0Cu) {
                                    ok = wait_drained<C::NACC>(st, ~0x0Cu, sh, abort_flag, p.status);
                                    if (!ok) break;
                                }
                                issue_group<S, false>(tmem, da0, db0);
                                if (st.pending & 0x0Cu) {
                                    ok = wait_drained<C::NACC>(st, 0x0Cu, sh, abort_flag, p.status);
                                    if (!ok) break;
                                }
                                issue_group<S, true>(tmem, da0, db0);
                                const bool last = step == nsteps - 1;
                                const uint32_t due = (last || (step % CHUNK_STEPS) == CHUNK_STEPS - 1)
                                                         ? due_mask(step / CHUNK_STEPS, last, C::NACC)
                                                         : 0u;
                                if (due) {  // hand the due accumulators to the epilogue
                                    umma_commit(&sh->accf[0]);
                                    st.pending |= due;
                                }
                            }
                        }
                        if (!ok) break;
                        umma_commit(&sh->empty[stage]);
                        if (++stage == C::STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
                if (!ok) spin_ns(2000000);  // let MMAs already issued retire
            }
        }
    } else if (warp >= EPI_WARP0) {
        // --------------------------------------------------- epilogue --
        const int q = warp & 3;                      // TMEM lane quadrant of this warp
        const int third = (warp - EPI_WARP0) >> 2;   // which third of the tile's columns
        const int row = 32 * q + lane;               // tile row == TMEM lane
        const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16);
        constexpr int EC = C::EPI;                   // columns per thread: 32 (FP8: 64)
        const int colbase = EC * third;
        uint32_t accf_phase = 0;  // bit g: parity of the next wait on accf[g]
        int ebuf = 0;             // one digit: the buffer of the next drain
        bool ok = true;
        constexpr bool ZERO = S <= 4;  // the grouped issue path (see issue_group)
        if constexpr (ZERO) {
            // zero every accumulator once and hand it to the issuer
            for (int a = 0; a < C::NBUF; ++a)
#pragma unroll
                for (int g = 0; g < EC / 16; ++g) tmem_st_zero_32x32b_x16(tbase + a * C::TN + colbase + 16 * g);
            tmem_st_wait();
            tc_fence_before();
            for (int a = 0; a < C::NBUF; ++a) mbar_arrive(&sh->acce[a]);
        }
        for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
            // Only the chunk count stays live across the K loop; the rest of
            // the task record is re-read for the store (register budget).
            const int nsteps = (p.tasks[ti].klen + KS - 1) / KS;
            const int nchunks = (nsteps + CHUNK_STEPS - 1) / CHUNK_STEPS;
            const int h = p.tasks[ti].hbits;
            const float fold_scale = __uint_as_float(static_cast<unsigned>(127 + 27 + h) << 23);
            using Sum = typename std::conditional<F8, float,
                                                  typename std::conditional<W1, int32_t, int64_t>::type>::type;
            Sum T[EC];
#pragma unroll
            for (int i = 0; i < EC; ++i) T[i] = 0;
            for (int c = 0; c < nchunks; ++c) {
                const bool last = c == nchunks - 1;
                const uint32_t due = due_mask(c, last, C::NACC);
                if (!due) continue;
                if constexpr (MULTI) {
                    // issuer by issuer, each issuer's accumulators in the order 4, 0, 1, 2, 3
                    bool good = true;
#pragma unroll
                    for (int gi = 0; gi < NI; ++gi) {
                        const uint32_t m = issuer_mask<NI>(gi) & due;
                        if (!m) continue;
                        // every lane of the warp takes the same decision before
                        // the warp-collective TMEM loads
                        if (!__all_sync(0xffffffffu,
                                        mbar_wait(&sh->accf[gi], (accf_phase >> gi) & 1u, abort_flag, p.status))) {
                            good = false;
                            break;
                        }
                        accf_phase ^= 1u << gi;
                        tc_fence_after();
                        if (m & 16u) drain_one<4, 2, false>(T, tbase, colbase, sh, h, fold_scale);
                        if (m & 1u) drain_one<0, 2, false>(T, tbase, colbase, sh, h, fold_scale);
                        if (m & 2u) drain_one<1, 2, false>(T, tbase, colbase, sh, h, fold_scale);
                        if (m & 4u) drain_one<2, 2, false>(T, tbase, colbase, sh, h, fold_scale);
                        if (m & 8u) drain_one<3, 2, false>(T, tbase, colbase, sh, h, fold_scale);
                    }
                    if (!good) {
                        ok = false;
                        break;
                    }
                    continue;
                }
                const int bar = S == 1 ? ebuf : 0;
                if (!__all_sync(0xffffffffu,
                                mbar_wait(&sh->accf[bar], (accf_phase >> bar) & 1u, abort_flag, p.status))) {
                    ok = false;
                    break;
                }
                accf_phase ^= 1u << bar;
                tc_fence_after();
                if constexpr (F8) {
                    drain_f8(T, tbase, colbase, sh, ebuf);
                } else if constexpr (W1) {
                    drain_w1(T, tbase, colbase, sh, ebuf);
                } else {
                    if (due & 16u) drain_one<4, (S <= 3 ? 1 : 0), ZERO>(T, tbase, colbase, sh, h, fold_scale);
                    if (due & 1u) drain_one<0, (S <= 3 ? 1 : 0), ZERO>(T, tbase, colbase, sh, h, fold_scale, S == 1 ? ebuf : 0);
                    if (due & 2u) drain_one<1, (S <= 3 ? 1 : 0), ZERO>(T, tbase, colbase, sh, h, fold_scale);
                    if (due & 4u) drain_one<2, (S <= 3 ? 1 : 0), ZERO>(T, tbase, colbase, sh, h, fold_scale);
                    if (due & 8u) drain_one<3, (S <= 3 ? 1 : 0), ZERO>(T, tbase, colbase, sh, h, fold_scale);
                }
                if constexpr (S == 1) ebuf ^= 1;
            }
            if (!ok) break;
            const LeafTask t = p.tasks[ti];
            if constexpr (F8) {
                // T holds sum_k q_u q_v of E4M3 values scaled by 2^(FP8_TOP - t - e)
                if (row < t.rows) {
                    const int lim0 = t.diag ? min(t.cols, row + t.diag_off + 1) : t.cols;
                    const int lim = lim0 < 0 ? 0 : lim0;
                    if (t.kind == OUT_M_F64) {  // Strassen product, in units of the scaled columns
                        double *out = static_cast<double *>(p.M) + t.out_off + static_cast<int64_t>(row) * t.out_ld;
                        const double sc = exp2d(t.shift - 2 * FP8_TOP);
                        store_row<EC, false>(out, colbase, lim, [&](int i) { return static_cast<double>(T[i]) * sc; },
                                             p.alpha, p.beta);
                    } else {
                        const int er = -2 * FP8_TOP + t.shift + (t.eu >= 0 ? p.expo[t.eu + row] : 0);
                        const int *ev = t.ev >= 0 ? p.expo + t.ev : nullptr;
                        float *out = static_cast<float *>(p.C) + c_row_offset(t, row, p.packed);
                        store_row<EC, true>(
                            out, colbase, lim, [&](int i) { return scale2f(T[i], er + (ev ? ev[colbase + i] : 0)); },
                            p.alpha, p.beta);
                    }
                }
            } else if (row < t.rows) {
                const int lim0 = t.diag ? min(t.cols, row + t.diag_off + 1) : t.cols;
                const int lim = lim0 < 0 ? 0 : lim0;
                // W1 sums are in units of the digit product, 2^(27 + h) of T's unit
                const int wsh = W1 ? 27 + t.hbits : 0;
                if (t.kind == OUT_M_I64) {
                    int64_t *out = static_cast<int64_t *>(p.M) + t.out_off + static_cast<int64_t>(row) * t.out_ld;
                    const int64_t wmul = int64_t(1) << wsh;
                    store_row<EC, false>(out, colbase, lim, [&](int i) { return static_cast<int64_t>(T[i]) * wmul; },
                                         p.alpha, p.beta);
                } else {
                    const int er = -(T_FRAC + 2 * DIGIT_TOP_BITS) - t.hbits + t.shift + wsh +
                                   (t.eu >= 0 ? p.expo[t.eu + row] : 0);
                    const int *ev = t.ev >= 0 ? p.expo + t.ev : nullptr;
                    void *cbase = p.probs ? p.probs[t.prob].C : p.C;
                    if (t.kind == OUT_C_F64) {
                        double *out = static_cast<double *>(cbase) + c_row_offset(t, row, p.packed);
                        store_row<EC, true>(
                            out, colbase, lim,
                            [&](int i) {
                                // T 2^x rounded once, on the integer pipe (GB300's FP64 rate is low)
                                const int x = er + (ev ? ev[colbase + i] : 0);
                                double v;
                                if (!ldexp_i64_rn(static_cast<int64_t>(T[i]), x, v))
                                    v = scale2d(static_cast<double>(T[i]), x);
                                return v;
                            },
                            p.alpha, p.beta);
                    } else {
                        float *out = static_cast<float *>(cbase) + c_row_offset(t, row, p.packed);
                        // (W1's sums are 32-bit: the 32-bit conversion)
                        store_row<EC, true>(
                            out, colbase, lim,
                            [&](int i) {
                                const float v = W1 ? __int2float_rn(static_cast<int32_t>(T[i]))
                                                   : __ll2float_rn(static_cast<int64_t>(T[i]));
                                return scale2f(v, er + (ev ? ev[colbase + i] : 0));
                            },
                            p.alpha, p.beta);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        // After an abort, MMAs committed to barriers nobody waited for may
        // still be writing TMEM: give them time to retire before the release.
        if (*abort_flag) spin_ns(2000000);
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing
// arrives at, with the given budget, so the wait runs out, records the
// timeout status and the kernel returns.
__global__ void wait_check_kernel(int *status, unsigned long long budget_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
    mbar_wait_for(&bar, 0u, &abort_flag, status, budget_ns);
}

// The shared-memory opt-in of leaf_tc_kernel<S>, set once per device (a
// later call, e.g. inside a graph capture, needs no attribute change).
template <int S, bool F8 = false, bool W1 = false>
cudaError_t ensure_leaf_attr() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(leaf_tc_kernel<S, F8, W1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg<S, F8, W1>::SMEM_BYTES);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <int S, bool F8 = false, bool W1 = false>
cudaError_t launch_s(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s) {
    using C = Cfg<S, F8, W1>;
    cudaError_t ea = ensure_leaf_attr<S, F8, W1>();
    if (ea != cudaSuccess) return ea;
    const int ntasks = static_cast<int>(P.tasks.size());
    const int grid = ntasks < num_sms ? ntasks : num_sms;
    leaf_tc_kernel<S, F8, W1><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(lp);
    return cudaGetLastError();
}

}  // namespace

int leaf_tc_smem_bytes(int slices) {
    switch (slices) {
        case 1: return Cfg<1>::SMEM_BYTES;
        case 2: return Cfg<2>::SMEM_BYTES;
        case 3: return Cfg<3>::SMEM_BYTES;
        case 4: return Cfg<4>::SMEM_BYTES;
        case 5: return Cfg<5>::SMEM_BYTES;
        case 6: return Cfg<6>::SMEM_BYTES;
        case 7: return Cfg<7>::SMEM_BYTES;
        default: return 0;
    }
}

cudaError_t launch_leaf_tc(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s) {
    if (P.tasks.empty()) return cudaSuccess;
    if (P.p.mode == MODE_F32_FP8) return launch_s<1, true>(P, lp, num_sms, s);
    if (P.slices == 1 && P.tile_n == TILE_N8) return launch_s<1, false, true>(P, lp, num_sms, s);
    switch (P.slices) {
        case 1: return launch_s<1>(P, lp, num_sms, s);
        case 2: return launch_s<2>(P, lp, num_sms, s);
        case 3: return launch_s<3>(P, lp, num_sms, s);
        case 4: return launch_s<4>(P, lp, num_sms, s);
        case 5: return launch_s<5>(P, lp, num_sms, s);
        case 6: return launch_s<6>(P, lp, num_sms, s);
        case 7: return launch_s<7>(P, lp, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ata

namespace ata {

// One group of a static partition: tasks [first, first + count) of the plan,
// laid out for `ctas` persistent CTAs.
cudaError_t launch_leaf_tc_group(const Plan &P, const LeafParams &lp, int64_t first, int64_t count, int ctas,
                                 cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    LeafParams g = lp;
    g.tasks = lp.tasks + first;
    g.ntasks = static_cast<int>(count);
    if (P.p.mode == MODE_F32_FP8) {
        cudaError_t e = ensure_leaf_attr<1, true>();
        if (e != cudaSuccess) return e;
        leaf_tc_kernel<1, true><<<count < ctas ? static_cast<int>(count) : ctas, NUM_THREADS,
                                  Cfg<1, true>::SMEM_BYTES, s>>>(g);
        return cudaGetLastError();
    }
    if (P.slices == 1 && P.tile_n == TILE_N8) {
        cudaError_t e = ensure_leaf_attr<1, false, true>();
        if (e != cudaSuccess) return e;
        leaf_tc_kernel<1, false, true><<<count < ctas ? static_cast<int>(count) : ctas, NUM_THREADS,
                                         Cfg<1, false, true>::SMEM_BYTES, s>>>(g);
        return cudaGetLastError();
    }
    return launch_leaf_tc_raw(P.slices, g, g.ntasks, ctas, s);
}

cudaError_t launch_wait_check(int *status, unsigned long long budget_ns, cudaStream_t s) {
    wait_check_kernel<<<1, 32, 0, s>>>(status, budget_ns);
    return cudaGetLastError();
}

// Leaf launch from an explicit task count (allocation-free and batched entry
// points).
cudaError_t launch_leaf_tc_raw(int slices, const LeafParams &lp, int ntasks, int num_sms, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    const int grid = ntasks < num_sms ? ntasks : num_sms;
#define ATA_LEAF_RAW(SS)                                                                                     \
    case SS: {                                                                                               \
        cudaError_t e = ensure_leaf_attr<SS>();                                                              \
        if (e != cudaSuccess) return e;                                                                      \
        leaf_tc_kernel<SS><<<grid, NUM_THREADS, Cfg<SS>::SMEM_BYTES, s>>>(lp);                              \
        return cudaGetLastError();                                                                           \
    }
    switch (slices) {
        ATA_LEAF_RAW(1)
        ATA_LEAF_RAW(2)
        ATA_LEAF_RAW(3)
        ATA_LEAF_RAW(4)
        ATA_LEAF_RAW(5)
        ATA_LEAF_RAW(6)
        ATA_LEAF_RAW(7)
        default: return cudaErrorInvalidValue;
    }
#undef ATA_LEAF_RAW
}

}  // namespace ata
