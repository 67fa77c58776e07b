// Auxiliary device kernels: column exponents (equilibration), operand
// preparation (exact fixed-point Strassen operand sums + digit slicing),
// Strassen result sums (exact int64 combine), the native-FP64 DMMA leaf, and
// the m == 0 zero fill.
//
// GB300 note: FP64 arithmetic runs at a small fraction of the integer and
// FP32 rates on this part, so every exact step here (scaling, operand sums,
// digit extraction, result sums) is done in 64-bit INTEGER arithmetic on a
// fixed-point representation; FP64 is used only to form the final values.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cstdint>
#include <type_traits>

#include "fixconv.h"
#include "kernels.h"
#include "ptx.cuh"

namespace ata {
namespace {

constexpr int STATUS_NONFINITE = 1;  // == ATA_ERR_INVALID

// 2^x as a double (exact for -1074 <= x <= 1023).
__device__ __forceinline__ double exp2i(int x) {
    if (x >= -1022 && x <= 1023) return __longlong_as_double(static_cast<long long>(x + 1023) << 52);
    return scalbn(1.0, x);
}

__device__ __forceinline__ float exp2f_i(int x) {
    if (x >= -126 && x <= 127) return __uint_as_float(static_cast<unsigned>(x + 127) << 23);
    return scalbnf(1.0f, x);
}

// v * 2^x: one multiply while 2^x is a normal number, else scalbn (one
// exact scaling and a single rounding, where 2^x alone would under- or
// overflow although v * 2^x need not: tiny or subnormal columns).
__device__ __forceinline__ double scale2d(double v, int x) {
    return (x >= -1022 && x <= 1023) ? v * exp2i(x) : scalbn(v, x);
}
__device__ __forceinline__ float scale2f(float v, int x) {
    return (x >= -126 && x <= 127) ? v * exp2f_i(x) : scalbnf(v, x);
}

// round(a * 2^sh) as int64 (round half away from zero), computed from the
// bits of a with integer operations only.  Requires |a * 2^sh| < 2^62.
__device__ __forceinline__ int64_t fixed_of(double a, int sh) {
    const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(a));
    const int eb = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
    const uint64_t M = eb ? (mant | (1ull << 52)) : mant;
    const int s = (eb ? eb - 1075 : -1074) + sh;  // value = M * 2^s
    uint64_t r;
    if (s >= 0)
        r = M << s;
    else if (s < -62)
        r = 0;
    else
        r = (M + (1ull << (-s - 1))) >> (-s);
    return (bits >> 63) ? -static_cast<int64_t>(r) : static_cast<int64_t>(r);
}

__device__ __forceinline__ int64_t fixed_of(float a, int sh) {
    const uint32_t bits = __float_as_uint(a);
    const int eb = static_cast<int>((bits >> 23) & 0xFF);
    const uint64_t mant = bits & 0x7FFFFFu;
    const uint64_t M = eb ? (mant | 0x800000u) : mant;
    const int s = (eb ? eb - 150 : -149) + sh;
    uint64_t r;
    if (s >= 0)
        r = M << s;
    else if (s < -62)
        r = 0;
    else
        r = (M + (1ull << (-s - 1))) >> (-s);
    return (bits >> 31) ? -static_cast<int64_t>(r) : static_cast<int64_t>(r);
}

__device__ __forceinline__ unsigned long long abs_bits(double a) {
    return static_cast<unsigned long long>(__double_as_longlong(a)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float a) {
    return __float_as_uint(a) & 0x7FFFFFFFu;
}

// ------------------------------------------------------------ exponents --
// colmax[j] = bits of max_i |a_ij| (order-preserving for non-negative IEEE).
template <typename T>
__global__ void __launch_bounds__(256) colmax_kernel(const T *__restrict__ A, int64_t m, int64_t n,
                                                     int64_t lda, int rows_per_block,
                                                     unsigned long long *colmax) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x;
    if (j >= n) return;
    const int64_t i0 = static_cast<int64_t>(blockIdx.y) * rows_per_block;
    const int64_t i1 = i0 + rows_per_block < m ? i0 + rows_per_block : m;
    unsigned long long mx = 0;
    for (int64_t i = i0; i < i1; ++i) {
        unsigned long long b = abs_bits(A[i * lda + j]);
        mx = b > mx ? b : mx;
    }
    if (mx) atomicMax(colmax + j, mx);
}

// e_j = smallest integer with max_i |a_ij| < 2^e_j (0 for a zero column),
// from the bits b of max_i |a_ij|; a non-finite column sets *status.
template <typename T>
__device__ __forceinline__ int column_exponent(unsigned long long b, int *status) {
    int e = 0;
    if (sizeof(T) == 8) {
        const int eb = static_cast<int>(b >> 52);
        if (eb == 0x7FF) atomicExch(status, STATUS_NONFINITE);
        if (b == 0)
            e = 0;
        else if (eb == 0)
            e = (64 - __clzll(static_cast<long long>(b & 0xFFFFFFFFFFFFFull))) - 1074;
        else
            e = eb - 1022;
    } else {
        const unsigned bb = static_cast<unsigned>(b);
        const int eb = static_cast<int>(bb >> 23);
        if (eb == 0xFF) atomicExch(status, STATUS_NONFINITE);
        if (bb == 0)
            e = 0;
        else if (eb == 0)
            e = (32 - __clz(static_cast<int>(bb & 0x7FFFFFu))) - 149;
        else
            e = eb - 126;
    }
    return e;
}

template <typename T>
__global__ void expo_kernel(const unsigned long long *colmax, int64_t n, int *expo, int *status) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    expo[j] = column_exponent<T>(colmax[j], status);
}

// Transposed operand (the A A^T product): the exponent of operand column j
// is taken over row j of A, which is contiguous.  One warp per row (coalesced
// loads, four in flight per lane), a warp maximum, no atomics.
template <typename T>
__global__ void __launch_bounds__(256) rowmax_expo_kernel(const T *__restrict__ A, int64_t rows, int64_t len,
                                                          int64_t lda, int *expo, int *status) {
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= rows) return;  // whole warps
    const T *r = A + j * lda;
    unsigned long long mx = 0;
    int64_t i = lane;
    for (; i + 96 < len; i += 128) {
        const unsigned long long b0 = abs_bits(r[i]), b1 = abs_bits(r[i + 32]);
        const unsigned long long b2 = abs_bits(r[i + 64]), b3 = abs_bits(r[i + 96]);
        mx = max(mx, max(max(b0, b1), max(b2, b3)));
    }
    for (; i < len; i += 32) mx = max(mx, abs_bits(r[i]));
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) expo[j] = column_exponent<T>(mx, status);
}

// Element offset of entry (j, k), k <= j, of a packed lower triangle.
__device__ __forceinline__ int64_t packed_at(int64_t j, int64_t k) { return j * (j + 1) / 2 + k; }

// -------------------------------------------------------- operand prep --
struct Families {
    Family f[MAX_FAMILIES];
};

// The operand a prep tile belongs to, and the tile's index within it
// (interleaved groups: see OpDesc::ilv_n).
__device__ __forceinline__ int find_desc(const OpDesc *ops, int nops, int64_t tile);
__device__ __forceinline__ int op_of_tile(const OpDesc *ops, int nops, int64_t tile, int64_t *local) {
    int i = find_desc(ops, nops, tile);
    const int64_t g = tile - ops[i].tile_base;
    const int n = ops[i].ilv_n;
    if (ops[i].fuse_ns > 0) {  // fused range: sub-group g mod nsub, tile g / nsub of every member
        const int nsub = ops[i].fuse_nsub;
        const int sub = static_cast<int>(g % nsub);
        while (ops[i].fuse_isub > sub) i -= ops[i].ilv_i + 1;  // back to the sub-group's last member
        *local = g / nsub;
        return i - ops[i].ilv_i;  // its first member
    }
    if (n > 1) {  // tile counts fit 32 bits (checked at launch): 32-bit division
        const uint32_t g32 = static_cast<uint32_t>(g);
        const uint32_t q = g32 / static_cast<uint32_t>(n);
        i = i - ops[i].ilv_i + static_cast<int>(g32 - q * static_cast<uint32_t>(n));
        *local = q;
    } else {
        *local = g;
    }
    return i;
}

__device__ __forceinline__ int find_desc(const OpDesc *ops, int nops, int64_t tile) {
    int lo = 0, hi = nops - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ops[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// round(a * 2^sh) (half away from zero) without branches, for |a * 2^sh| <=
// 2^F (guaranteed by the column exponents).  With a = M 2^s', s = s' + sh and
// P = max(F - mantissa bits, 0): r = (X + 2^u) >> (u + 1), X = M 2^(P + 1 + L),
// L = max(s - P, 0) (only a subnormal a in a column whose maximum is
// subnormal too has s > P), u = max(P - s, 0) clamped to 62 (fixconv.h, which
// the CPU tests check against the exact definition).
template <int F, typename T>
struct FastFixed {
    static constexpr int MB = sizeof(T) == 8 ? 52 : 23;
    static constexpr int P = F - MB > 0 ? F - MB : 0;
    static constexpr bool ok = MB + 1 + P + 1 <= 62;
};

template <int F>
__device__ __forceinline__ int64_t fixed_of_fast(double a, int sh) {
    return fixed_of_f64<FastFixed<F, double>::P>(a, sh);
}

template <int F>
__device__ __forceinline__ int64_t fixed_of_fast(float a, int sh) {
    return fixed_of_f32<FastFixed<F, float>::P>(a, sh);
}

// 32-bit form for FP32 inputs and F <= 29 fraction bits (one to three
// digits); same result as the 64-bit form.
template <int F>
__device__ __forceinline__ int32_t fixed32_of_fast(float a, int sh) {
    static_assert(F <= 29, "32-bit fixed point");
    return fixed32_of_f32<(F - 23 > 0 ? F - 23 : 0)>(a, sh);
}

// Digit q of w = V + sum_{j < S-1} 256 * 512^j as the BF16-exact float
// x_q * 2^(-9 (q - 1)).  Adding that constant turns the balanced digits of V
// into plain 9-bit fields of w: x = field - 256 for the S - 1 low digits, and
// the top digit x_1 is w >> 9 (S - 1).  Both are built from their bits: the
// field is or-ed into the mantissa of 2^23 and one exact FMA removes 2^23 + 256
// and applies the digit's power-of-two scale.
template <int S, int Q, typename W>
__device__ __forceinline__ float digit_value(W w) {
    if constexpr (Q == 0) {
        const int x = static_cast<int>(w >> (DIGIT_BITS * (S - 1)));  // |x| <= 256
        return __int_as_float(0x4B400000 + x) - 12582912.0f;         // 1.5 * 2^23
    } else {
        constexpr int J = S - 1 - Q;  // field index from the least significant
        const uint32_t f = static_cast<uint32_t>(w >> (DIGIT_BITS * J)) & 511u;
        constexpr float sc = 1.0f / static_cast<float>(1ull << (DIGIT_BITS * Q));
        return fmaf(__uint_as_float(0x4B000000u | f), sc, -8388864.0f * sc);
    }
}

template <int S, int Q, typename W>
__device__ __forceinline__ void store_digit_row(const W (&w)[KSTEP], uint8_t *img_row, int swz) {
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(digit_value<S, Q>(w[2 * i]), digit_value<S, Q>(w[2 * i + 1]));
        pk[i] = *reinterpret_cast<const uint32_t *>(&v);
    }
    // chunk h (contraction values 8h .. 8h + 7) sits at 16-byte slot h ^ swz
    *reinterpret_cast<uint4 *>(img_row + (swz << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(img_row + ((swz ^ 1) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

template <int S, int Q = 0, typename W>
__device__ __forceinline__ void store_digits(const W (&w)[KSTEP], uint8_t *row0, int64_t plane_step,
                                             int swz) {
    if constexpr (Q < S) {
        store_digit_row<S, Q, W>(w, row0 + Q * plane_step, swz);
        store_digits<S, Q + 1, W>(w, row0, plane_step, swz);
    }
}

// Digit planes.  For operand o and its 64 x 64 tile (k0, c0):
//   V[k][c] = sum_t coef_t * round(a(row0_t + k, col0_t + c) * 2^(F - t - e))
// with F = 8 + 9 (S - 1) fraction bits, exact in int64.  V is then written as
// S balanced digits x_1 (|x_1| <= 256) and x_q in [-256, 255] (q >= 2) with
// V = sum_q x_q 2^(9 (S - q)); digit q is stored as the BF16 value
// x_q * 2^(-9 (q - 1)) (exact: at most 8 significant bits), K-major: plane q,
// column c, contraction k.
// Read phase: each warp loads 32 consecutive columns of one row (coalesced);
// all 16 loads of a term are issued before the column exponent is needed.
// Write phase: thread (c, ks) owns column c of contraction step ks and writes
// its 32-byte image row of every digit plane as two 16-byte stores, so one
// warp fills each 1 KB image.  Blocks are persistent (grid-stride over the
// tiles) and keep the operand tables in shared memory when they fit, so a
// tile starts with no dependent global loads before its data loads.
constexpr int PREP_SMEM_OPS = 64;
constexpr int PREP_SMEM_TERMS = 128;

// sv[it * ld] = sum over the op's terms of coef * round(a * 2^sh) for the 16
// rows k0 + it of column c0 + cc (one thread per column and 16-row group; a
// warp loads 32 consecutive columns of a row).  NT > 0 (1, 2 or 4 terms; a missing fourth
// reads nothing): the rows go in groups of 16 / NT, every term's loads of a
// group are issued before any is used (16 loads in flight per thread whatever
// the term count), and a group's sums go to shared memory as soon as they are
// complete.  NT = 0: any count, groups of four rows, one term at a time.
// trans: the operand is the transpose of A (element (r, c) at A[c * lda + r]);
// each thread then reads 16 consecutive elements of one row of A.
template <int S, int NT, typename T, bool F8>
__device__ __forceinline__ void read_terms(const T *__restrict__ A, int64_t lda, bool trans,
                                           const int *__restrict__ expo, const OpDesc &od, const OpTerm *terms,
                                           int k0, int c0, int cc, int64_t *sv, int ld) {
    const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;  // strides of an operand row / column
    constexpr int F = F8 ? FP8_FIX : DIGIT_TOP_BITS + DIGIT_BITS * (S - 1);
    // FP32 input with up to 3 digits: every value and sum fits 32 bits.
    constexpr bool NARROW = sizeof(T) == 4 && !F8 && F <= 29;
    using V = typename std::conditional<NARROW, int32_t, int64_t>::type;
    auto fixed = [](T a, int sh) -> V {
        if constexpr (NARROW)
            return fixed32_of_fast<F>(static_cast<float>(a), sh);
        else if constexpr (FastFixed<F, T>::ok)
            return fixed_of_fast<F>(a, sh);
        else
            return fixed_of(a, sh);
    };
    const int c = c0 + cc;
    if constexpr (NT > 0) {
        constexpr int G = PREP_TK / NT;  // rows per group
        const T *base[NT];               // element (k0, column) of each term
        int lim[NT], sh[NT], neg[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const bool present = t < od.nterms;
            const OpTerm tm = present ? terms[od.first_term + t] : OpTerm{};
            const bool cv = present && c < tm.cols;
            base[t] = A + (tm.row0 + k0) * rs + (tm.col0 + c) * cs;
            lim[t] = cv ? tm.rows - k0 : 0;  // rows it < lim are inside the term
            sh[t] = cv ? F - od.t_shift - expo[tm.col0 + c] : 0;
            neg[t] = tm.coef < 0;
        }
#pragma unroll
        for (int g = 0; g < PREP_TK; g += G) {
            T raw[NT][G];
#pragma unroll
            for (int t = 0; t < NT; ++t)
#pragma unroll
                for (int j = 0; j < G; ++j) raw[t][j] = (g + j) < lim[t] ? base[t][(g + j) * rs] : T(0);
#pragma unroll
            for (int j = 0; j < G; ++j) {
                V v = 0;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    const V x = fixed(raw[t][j], sh[t]);
                    v += neg[t] ? -x : x;
                }
                sv[(g + j) * ld] = v;
            }
        }
    } else {
#pragma unroll 1
        for (int g = 0; g < PREP_TK; g += 4) {
            V v[4] = {0, 0, 0, 0};
            for (int t = 0; t < od.nterms; ++t) {
                const OpTerm tm = terms[od.first_term + t];
                const bool cvalid = c < tm.cols;
                const T *col = A + (tm.col0 + c) * cs;
                T raw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = k0 + g + j;
                    raw[j] = (cvalid && k < tm.rows) ? col[(tm.row0 + k) * rs] : T(0);
                }
                const int sh = cvalid ? F - od.t_shift - expo[tm.col0 + c] : 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const V x = fixed(raw[j], sh);
                    v[j] += tm.coef > 0 ? x : -x;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) sv[(g + j) * ld] = v[j];
        }
    }
}

// One prep tile of an operand: (4096 / tc) contraction rows x tc columns,
// tc = 2^lgtc in {64, 128, 256}.  Thread t owns column t mod tc and the
// 16-row group (one K step) t / tc: it reads that column segment (above) and
// writes its 32-byte image row of every digit plane as two 16-byte stores,
// so a warp fills one 1 KB image per digit.
constexpr int PREP_SV = 4096 + 256;  // shared sums: (4096 / tc) x (tc + 1) entries at most

// E4M3 code of V * 2^(FP8_TOP - FP8_FIX), rounded to nearest even: V is
// first rounded to odd at FP32's 24 bits (truncate, then set the last bit if
// anything was dropped), which keeps the final rounding to E4M3's 4 bits (or
// its subnormal grid) exact (Boldo and Melquiond, "Emulation of FMA and
// correctly rounded sums: proved algorithms using rounding to odd", 2008).
// |V| <= 2^FP8_FIX, so the scaled value stays below 2^FP8_TOP.
// The truncation and the sticky bit are taken from the integer's bits (its
// top 24 significant bits, and whether any bit below them is set), so the
// only conversion is a 32-bit one: the 64-bit integer-float conversions ran
// at a small fraction of the rate and bounded this kernel (same codes).
__device__ __forceinline__ uint32_t e4m3_of_fixed(int64_t V) {
    const unsigned long long mag = V < 0 ? 0ull - static_cast<unsigned long long>(V) : static_cast<unsigned long long>(V);
    const int p = 63 - __clzll(static_cast<long long>(mag | 1ull));  // leading bit (mag < 2^48)
    const int sh = p > 23 ? p - 23 : 0;
    uint32_t m24 = static_cast<uint32_t>(mag >> sh);                  // truncated to 24 bits
    if (sh > 0 && (mag & ((1ull << sh) - 1ull)) != 0ull) m24 |= 1u;   // round to odd
    float f = __uint2float_rn(m24);                                    // exact: m24 < 2^24
    f *= __uint_as_float(static_cast<unsigned>(127 + sh + FP8_TOP - FP8_FIX) << 23);
    return static_cast<uint32_t>(__nv_cvt_float_to_fp8(V < 0 ? -f : f, __NV_SATFINITE, __NV_E4M3));
}

template <int S, typename T, bool F8 = false>
__device__ __forceinline__ void prep_tile(const T *__restrict__ A, int64_t lda, bool trans,
                                          const int *__restrict__ expo, const OpDesc &od, const OpTerm *terms,
                                          int64_t tile, const Family &fam, uint8_t *ws, int64_t *sV, int lgtc) {
    const int tc = 1 << lgtc, tk = 4096 >> lgtc, ld = tc + 1;
    const int64_t local = tile - od.tile_base;
    const int tiles_k = od.K_pitch / tk;
    const int k0 = static_cast<int>(local % tiles_k) * tk;
    const int c0 = static_cast<int>(local / tiles_k) * tc;
    const int cc = threadIdx.x & (tc - 1);  // column within the tile
    const int rg = threadIdx.x >> lgtc;     // 16-row group (K step) within the tile
    int64_t *sv = sV + rg * KSTEP * ld + cc;
    switch (od.nterms) {
        case 1: read_terms<S, 1, T, F8>(A, lda, trans, expo, od, terms, k0 + rg * KSTEP, c0, cc, sv, ld); break;
        case 2: read_terms<S, 2, T, F8>(A, lda, trans, expo, od, terms, k0 + rg * KSTEP, c0, cc, sv, ld); break;
        case 3:
        case 4: read_terms<S, 4, T, F8>(A, lda, trans, expo, od, terms, k0 + rg * KSTEP, c0, cc, sv, ld); break;
        default: read_terms<S, 0, T, F8>(A, lda, trans, expo, od, terms, k0 + rg * KSTEP, c0, cc, sv, ld); break;
    }
    __syncthreads();

    if constexpr (F8) {
        // One E4M3 plane: the thread's 16 rows are one 16-byte half of its
        // column's 32-byte image row (rows 32 ks .. 32 ks + 31); half h sits
        // at 16-byte slot h ^ swz.
        if (c0 + cc < od.P_pad) {
            const int64_t ncb = fam.cols / BLOCK_COLS;
            const int r = cc & (BLOCK_COLS - 1);
            const int kk = k0 + rg * KSTEP;
            const int64_t cblk = (od.out_col + c0 + cc) / BLOCK_COLS;
            uint32_t pk[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                pk[i] = e4m3_of_fixed(sv[(4 * i) * ld]) | (e4m3_of_fixed(sv[(4 * i + 1) * ld]) << 8) |
                        (e4m3_of_fixed(sv[(4 * i + 2) * ld]) << 16) | (e4m3_of_fixed(sv[(4 * i + 3) * ld]) << 24);
            const int slot = ((kk / KSTEP) & 1) ^ ((r >> 2) & 1);
            uint8_t *dst = ws + fam.offset + (static_cast<int64_t>(kk / KSTEP8) * ncb + cblk) * BLOCK_BYTES + r * 32 +
                           slot * 16;
            *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    } else if (c0 + cc < od.P_pad) {
        const int64_t ncb = fam.cols / BLOCK_COLS;
        const int r = cc & (BLOCK_COLS - 1);
        constexpr int64_t CADD = [] {
            int64_t v = 0;
            for (int j = 0; j < S - 1; ++j) v += int64_t(256) << (DIGIT_BITS * j);
            return v;
        }();
        // up to 3 digits the shifted value fits 32 bits (|V| <= 2^26 + CADD)
        using W = typename std::conditional<(S <= 3), int32_t, int64_t>::type;
        W w[KSTEP];
#pragma unroll
        for (int i = 0; i < KSTEP; ++i) w[i] = static_cast<W>(sv[i * ld]) + static_cast<W>(CADD);
        const int64_t kstep = k0 / KSTEP + rg;
        const int64_t cblk = (od.out_col + c0 + cc) / BLOCK_COLS;
        uint8_t *row0 = ws + fam.offset + ((kstep * S) * ncb + cblk) * BLOCK_BYTES + r * 32;
        store_digits<S>(w, row0, ncb * BLOCK_BYTES, (r >> 2) & 1);
    }
    __syncthreads();  // sV is reused by the block's next tile
}

// prep_tile for FP32 inputs with up to 3 digits, whose fixed-point values
// and sums fit 32 bits: the thread keeps its 16 sums in registers, so there
// is no shared-memory round trip and no block barrier, and each term's 16
// loads are in flight together.  Same values as prep_tile.
template <int S, typename T>
__device__ __forceinline__ void prep_tile_narrow(const T *__restrict__ A, int64_t lda, bool trans,
                                                 const int *__restrict__ expo, const OpDesc &od,
                                                 const OpTerm *terms, int64_t tile, const Family &fam, uint8_t *ws,
                                                 int lgtc) {
    constexpr int F = DIGIT_TOP_BITS + DIGIT_BITS * (S - 1);
    static_assert(sizeof(T) == 4 && S <= 3 && F <= 29, "32-bit fixed point");
    const int tc = 1 << lgtc, tk = 4096 >> lgtc;
    const int64_t local = tile - od.tile_base;
    const int tiles_k = od.K_pitch / tk;
    const int k0 = static_cast<int>(local % tiles_k) * tk;
    const int c0 = static_cast<int>(local / tiles_k) * tc;
    const int cc = threadIdx.x & (tc - 1);
    const int rg = threadIdx.x >> lgtc;
    const int c = c0 + cc;
    if (c >= od.P_pad) return;
    const int kk = k0 + rg * KSTEP;
    const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;
    int32_t v[KSTEP];
#pragma unroll
    for (int j = 0; j < KSTEP; ++j) v[j] = 0;
    for (int t = 0; t < od.nterms; ++t) {
        const OpTerm tm = terms[od.first_term + t];
        const bool cv = c < tm.cols;
        const T *base = A + (tm.row0 + kk) * rs + (tm.col0 + c) * cs;
        const int lim = cv ? tm.rows - kk : 0;
        T raw[KSTEP];
#pragma unroll
        for (int j = 0; j < KSTEP; ++j) raw[j] = j < lim ? base[j * rs] : T(0);
        const int sh = cv ? F - od.t_shift - expo[tm.col0 + c] : 0;
#pragma unroll
        for (int j = 0; j < KSTEP; ++j) {
            const int32_t x = fixed32_of_fast<F>(static_cast<float>(raw[j]), sh);
            v[j] += tm.coef > 0 ? x : -x;
        }
    }
    constexpr int32_t CADD = [] {
        int32_t a = 0;
        for (int j = 0; j < S - 1; ++j) a += int32_t(256) << (DIGIT_BITS * j);
        return a;
    }();
    int32_t w[KSTEP];
#pragma unroll
    for (int j = 0; j < KSTEP; ++j) w[j] = v[j] + CADD;
    const int64_t ncb = fam.cols / BLOCK_COLS;
    const int r = cc & (BLOCK_COLS - 1);
    const int64_t cblk = (od.out_col + c) / BLOCK_COLS;
    uint8_t *row0 = ws + fam.offset + ((static_cast<int64_t>(kk / KSTEP) * S) * ncb + cblk) * BLOCK_BYTES + r * 32;
    store_digits<S>(w, row0, ncb * BLOCK_BYTES, (r >> 2) & 1);
}

// FP8 prep tile (32 contraction rows x 128 columns) of a single-term
// operand: each E4M3 value is the scaled entry a 2^(FP8_TOP - e) rounded to
// nearest even directly.  The scaling is exact in FP32 (an entry that leaves
// FP32's normal range lies far below E4M3's smallest subnormal), so this is
// the same rounding as the oracle's quantisation; only sums of several
// blocks (Strassen operands) need the exact fixed-point detour of prep_tile.
// Each thread converts 16 rows of one column, with its 16 loads in flight,
// and writes its 16-byte half of the column's 32-byte image row.
template <typename T>
__device__ __forceinline__ void prep_tile_f8_single(const T *__restrict__ A, int64_t lda, bool trans,
                                                    const int *__restrict__ expo, const OpDesc &od,
                                                    const OpTerm *terms, int64_t tile, const Family &fam,
                                                    uint8_t *ws) {
    constexpr int lgtc = 7, tc = 1 << lgtc, tk = 4096 >> lgtc;
    const int64_t local = tile - od.tile_base;
    const int tiles_k = od.K_pitch / tk;
    const int k0 = static_cast<int>(local % tiles_k) * tk;
    const int c0 = static_cast<int>(local / tiles_k) * tc;
    const int cc = threadIdx.x & (tc - 1);
    const int rg = threadIdx.x >> lgtc;
    const int c = c0 + cc;
    if (c >= od.P_pad) return;
    const int kk = k0 + rg * KSTEP;
    const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;
    const OpTerm tm = terms[od.first_term];
    const bool cv = c < tm.cols;
    const int lim = cv ? tm.rows - kk : 0;
    const T *base = A + (tm.row0 + kk) * rs + (tm.col0 + c) * cs;
    float raw[KSTEP];
#pragma unroll
    for (int j = 0; j < KSTEP; ++j) raw[j] = j < lim ? static_cast<float>(base[j * rs]) : 0.0f;
    // 2^(FP8_TOP - e) (and the term's sign) as two factors built from their
    // exponent bits: x reaches 156 for a column whose maximum is subnormal,
    // and each half stays in range; both products are exact power-of-two
    // scalings (an intermediate underflow only hits values that round to 0).
    const int x = cv ? FP8_TOP - expo[tm.col0 + c] : 0;
    const float sc = exp2f_i(x >> 1) * (tm.coef < 0 ? -1.0f : 1.0f), sc2 = exp2f_i(x - (x >> 1));
    uint32_t pk[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w |= static_cast<uint32_t>(__nv_cvt_float_to_fp8(raw[4 * i + j] * sc * sc2, __NV_SATFINITE, __NV_E4M3))
                 << (8 * j);
        pk[i] = w;
    }
    const int64_t ncb = fam.cols / BLOCK_COLS;
    const int r = cc & (BLOCK_COLS - 1);
    const int64_t cblk = (od.out_col + c) / BLOCK_COLS;
    const int slot = ((kk / KSTEP) & 1) ^ ((r >> 2) & 1);
    uint8_t *dst = ws + fam.offset + (static_cast<int64_t>(kk / KSTEP8) * ncb + cblk) * BLOCK_BYTES + r * 32 + slot * 16;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

// One-digit BF16 prep tile (16 contraction rows x 256 columns) of a
// single-term operand: the digit is round(a 2^(8 - e)) (half away from zero,
// as the fixed-point path rounds), an integer of at most 256 in magnitude
// that BF16 holds exactly, computed directly from the scaled FP32 value (the
// scaling is exact, and an entry below FP32's normal range scales to well
// under 1/2, i.e. a zero digit).  Each thread converts 16 rows of one column
// and writes its 32-byte image row as two 16-byte stores.
template <typename T>
__device__ __forceinline__ void prep_tile_bf16_single(const T *__restrict__ A, int64_t lda, bool trans,
                                                      const int *__restrict__ expo, const OpDesc &od,
                                                      const OpTerm *terms, int64_t tile, const Family &fam,
                                                      uint8_t *ws, int lgtc) {
    const int tc = 1 << lgtc, tk = 4096 >> lgtc;
    const int64_t local = tile - od.tile_base;
    const int tiles_k = od.K_pitch / tk;
    const int k0 = static_cast<int>(local % tiles_k) * tk;
    const int c0 = static_cast<int>(local / tiles_k) * tc;
    const int cc = threadIdx.x & (tc - 1);
    const int rg = threadIdx.x >> lgtc;
    const int c = c0 + cc;
    if (c >= od.P_pad) return;
    const int kk = k0 + rg * KSTEP;
    const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;
    const OpTerm tm = terms[od.first_term];
    const bool cv = c < tm.cols;
    const int lim = cv ? tm.rows - kk : 0;
    const T *base = A + (tm.row0 + kk) * rs + (tm.col0 + c) * cs;
    float raw[KSTEP];
#pragma unroll
    for (int j = 0; j < KSTEP; ++j) raw[j] = j < lim ? static_cast<float>(base[j * rs]) : 0.0f;
    // 2^(8 - e) as two exact factors (see prep_tile_f8_single)
    const int x = cv ? DIGIT_TOP_BITS - expo[tm.col0 + c] : 0;
    const float sc = exp2f_i(x >> 1) * (tm.coef < 0 ? -1.0f : 1.0f), sc2 = exp2f_i(x - (x >> 1));
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 v =
            __floats2bfloat162_rn(roundf(raw[2 * i] * sc * sc2), roundf(raw[2 * i + 1] * sc * sc2));
        pk[i] = *reinterpret_cast<const uint32_t *>(&v);
    }
    const int64_t ncb = fam.cols / BLOCK_COLS;
    const int r = cc & (BLOCK_COLS - 1);
    const int swz = (r >> 2) & 1;
    const int64_t cblk = (od.out_col + c) / BLOCK_COLS;
    uint8_t *row0 = ws + fam.offset + (static_cast<int64_t>(kk / KSTEP) * ncb + cblk) * BLOCK_BYTES + r * 32;
    // rows 8h .. 8h + 7 sit at 16-byte slot h ^ swz
    *reinterpret_cast<uint4 *>(row0 + (swz << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(row0 + ((swz ^ 1) << 4)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Half an image row: contraction values 8h .. 8h + 7 of one column, digits
// Q .. S - 1, one 16-byte store per digit plane at byte `off` (slot h ^ swz)
// of the column's 32-byte image row.
template <int S, int Q = 0, typename W>
__device__ __forceinline__ void store_digits_half(const W (&w)[8], uint8_t *row0, int64_t plane_step, int off) {
    if constexpr (Q < S) {
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 v =
                __floats2bfloat162_rn(digit_value<S, Q>(w[2 * i]), digit_value<S, Q>(w[2 * i + 1]));
            pk[i] = *reinterpret_cast<const uint32_t *>(&v);
        }
        *reinterpret_cast<uint4 *>(row0 + Q * plane_step + off) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        store_digits_half<S, Q + 1, W>(w, row0, plane_step, off);
    }
}

// One prep tile (16 contraction rows x FUSED_TC columns) of every operand of
// a fused group (OpDesc::fuse_ns <= FUSE_MAX_SRC sources).  Lanes 2l and
// 2l + 1 of a warp own one column and rows 0-7 / 8-15 of the tile: each loads
// its rows of every source block once and writes its half of the column's
// 32-byte image row of every member's digit planes, so one warp store fills
// 16 whole image rows (512 contiguous bytes).  Each member's value is the one prep_tile
// writes: every term rounded with the member's t_shift and the terms summed
// exactly; with fuse_uni (one t_shift for the whole group) each source value
// is rounded once for all members.
template <int S, typename T, bool UNI>
__device__ __forceinline__ void prep_fused_tile(const T *__restrict__ A, int64_t lda, bool trans,
                                                const int *__restrict__ expo, const OpDesc *o, int lead,
                                                const OpTerm *__restrict__ fsrc, int64_t local,
                                                const Families &fams, uint8_t *ws) {
    constexpr int F = DIGIT_TOP_BITS + DIGIT_BITS * (S - 1);
    constexpr bool NARROW = sizeof(T) == 4 && F <= 29;
    using V = typename std::conditional<NARROW, int32_t, int64_t>::type;
    using W = typename std::conditional<(S <= 3), int32_t, int64_t>::type;
    constexpr int NS = FUSE_MAX_SRC;
    constexpr int R = 8;            // contraction rows per lane
    constexpr int LPC = KSTEP / R;  // lanes per column
    auto fixed = [](T a, int sh) -> V {
        if constexpr (NARROW)
            return fixed32_of_fast<F>(static_cast<float>(a), sh);
        else if constexpr (FastFixed<F, T>::ok)
            return fixed_of_fast<F>(a, sh);
        else
            return fixed_of(a, sh);
    };
    constexpr int64_t CADD = [] {
        int64_t v = 0;
        for (int j = 0; j < S - 1; ++j) v += int64_t(256) << (DIGIT_BITS * j);
        return v;
    }();
    const OpDesc &L = o[lead];
    const int ns = L.fuse_ns, nm = L.ilv_n;
    const int tiles_k = L.K_pitch / KSTEP;
    const int k0 = static_cast<int>(local % tiles_k) * KSTEP;
    const int c0 = static_cast<int>(local / tiles_k) * FUSED_TC;
    const int lane = threadIdx.x & 31;
    const int cc = (threadIdx.x >> 5) * (32 / LPC) + lane / LPC;
    const int part = lane % LPC;  // rows R part .. R part + R - 1 of the tile
    const int c = c0 + cc;
    if (c >= L.P_pad) return;  // every member has the group's P_pad
    const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;
    const int kh = k0 + R * part;
    T raw[NS][R];
    int ex[NS];
    int64_t arow[NS], acol[NS];  // A position of this lane's first element of block q (-1: none)
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const bool present = q < ns;
        const OpTerm sb = present ? fsrc[L.fuse_src + q] : OpTerm{};
        const bool cv = present && c < sb.cols;
        const T *base = A + (sb.row0 + kh) * rs + (sb.col0 + c) * cs;
        const int lim = cv ? sb.rows - kh : 0;
#pragma unroll
        for (int j = 0; j < R; ++j) raw[q][j] = j < lim ? base[j * rs] : T(0);
        ex[q] = cv ? expo[sb.col0 + c] : 0;
        arow[q] = lim > 0 ? sb.row0 + kh : -1;
        acol[q] = sb.col0 + c;
    }
    // The planes of A itself (family 0, no operand sum: t = 0) for the
    // blocks' own elements: each block starts on a K step, so this lane's 8
    // rows are half of one image row of A's planes; rows past a block's end
    // belong to the next block (or are A's zero padding).
    const Family &f0 = fams.f[0];
    const int64_t ncb0 = f0.cols / BLOCK_COLS;
    auto store_f0 = [&](int q, const W (&w0)[R]) {
        const int r0 = static_cast<int>(acol[q] & (BLOCK_COLS - 1));
        uint8_t *dst = ws + f0.offset + (((arow[q] / KSTEP) * S) * ncb0 + acol[q] / BLOCK_COLS) * BLOCK_BYTES +
                       r0 * 32;
        store_digits_half<S>(w0, dst, ncb0 * BLOCK_BYTES, (part ^ ((r0 >> 2) & 1)) << 4);
    };
    // UNI: every source value rounded once, for all members
    V x[UNI ? NS : 1][R];
    // FP64 sources with the planes of A and members at t_shift 1 (depth 1):
    // both roundings of each value from one truncation (fixed_pair_f64,
    // bit-identical to two conversions)
    constexpr bool PAIR = UNI && sizeof(T) == 8 && !NARROW && FastFixed<F, T>::ok;
    bool paired = false;
    if constexpr (PAIR) {
        if (L.fuse_f0 && L.t_shift == 1) {
            paired = true;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                W w0[R];
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    int64_t xf, xh;
                    fixed_pair_f64<FastFixed<F, T>::P>(static_cast<double>(raw[q][j]), F - ex[q], xf, xh);
                    x[q][j] = xh;
                    w0[j] = static_cast<W>(xf) + static_cast<W>(CADD);
                }
                if (arow[q] >= 0) store_f0(q, w0);
            }
        }
    }
    if (!paired) {
        if (L.fuse_f0) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                if (arow[q] < 0) continue;
                W w0[R];
#pragma unroll
                for (int j = 0; j < R; ++j) w0[j] = static_cast<W>(fixed(raw[q][j], F - ex[q])) + static_cast<W>(CADD);
                store_f0(q, w0);
            }
        }
        if constexpr (UNI) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const int sh = F - L.t_shift - ex[q];
#pragma unroll
                for (int j = 0; j < R; ++j) x[q][j] = fixed(raw[q][j], sh);
            }
        }
    }
    const Family &fam = fams.f[L.family];
    const int64_t ncb = fam.cols / BLOCK_COLS;
    const int64_t plane_step = ncb * BLOCK_BYTES;
    const int r = c & (BLOCK_COLS - 1);  // out_col is a multiple of BLOCK_COLS
    // rows 8h .. 8h + 7 are 16-byte slot h ^ swz of the image row
    const int off = (part ^ ((r >> 2) & 1)) << 4;
    const int64_t kstep = k0 / KSTEP;
#pragma unroll 1
    for (int mi = 0; mi < nm; ++mi) {
        const OpDesc &od = o[lead + mi];
        V v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = 0;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            // 2-bit coefficient of source q (uniform over the block)
            const int cf = static_cast<int>(static_cast<uint32_t>(od.fuse_coef) << (30 - 2 * q)) >> 30;
            if (cf == 0) continue;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                V y;
                if constexpr (UNI)
                    y = x[q][j];
                else
                    y = fixed(raw[q][j], F - od.t_shift - ex[q]);
                v[j] += cf > 0 ? y : -y;
            }
        }
        W w[R];
#pragma unroll
        for (int j = 0; j < R; ++j) w[j] = static_cast<W>(v[j]) + static_cast<W>(CADD);
        const int64_t cblk = (od.out_col + c) / BLOCK_COLS;
        uint8_t *row0 = ws + fam.offset + ((kstep * S) * ncb + cblk) * BLOCK_BYTES + r * 32;
        store_digits_half<S>(w, row0, plane_step, off);
    }
}

// Prep tiles [tile_begin, ntiles) outside the fused groups.
template <int S, typename T, bool F8 = false>
__global__ void __launch_bounds__(256, 4) prep_digits_kernel(const T *__restrict__ A, int64_t lda, bool trans,
                                                             const int *__restrict__ expo,
                                                             const OpDesc *__restrict__ ops, int nops,
                                                             const OpTerm *__restrict__ terms, int nterms,
                                                             int64_t tile_begin, int64_t ntiles, Families fams,
                                                             uint8_t *ws) {
    __shared__ int64_t sV[PREP_SV];
    __shared__ OpDesc s_ops[PREP_SMEM_OPS];
    __shared__ OpTerm s_terms[PREP_SMEM_TERMS];
    const bool cached = nops <= PREP_SMEM_OPS && nterms <= PREP_SMEM_TERMS;
    if (cached) {
        for (int i = threadIdx.x; i < nops; i += blockDim.x) s_ops[i] = ops[i];
        for (int i = threadIdx.x; i < nterms; i += blockDim.x) s_terms[i] = terms[i];
        __syncthreads();
    }
    const OpDesc *o = cached ? s_ops : ops;
    const OpTerm *tt = cached ? s_terms : terms;
    for (int64_t tile = tile_begin + blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t local;
        const OpDesc &od = o[op_of_tile(o, nops, tile, &local)];  // read where used (register budget)
        if constexpr (!F8 && S == 1 && sizeof(T) == 4) {  // (FP64 inputs keep the exact fixed point)
            if (od.nterms == 1) {
                prep_tile_bf16_single<T>(A, lda, trans, expo, od, tt, od.tile_base + local, fams.f[od.family], ws, 8);
                continue;
            }
        }
        if constexpr (!F8 && sizeof(T) == 4 && S <= 3) {
            prep_tile_narrow<S, T>(A, lda, trans, expo, od, tt, od.tile_base + local, fams.f[od.family], ws, 8);
            continue;
        }
        if constexpr (F8) {
            if (od.nterms == 1) {
                prep_tile_f8_single<T>(A, lda, trans, expo, od, tt, od.tile_base + local, fams.f[od.family], ws);
                continue;
            }
        }
        // 16 x 256 tiles; FP8: 32 x 128 (one K step of the plane)
        prep_tile<S, T, F8>(A, lda, trans, expo, od, tt, od.tile_base + local, fams.f[od.family], ws, sV,
                            F8 ? 7 : 8);
    }
}

// Prep tiles [0, ntiles) of the fused groups (which come first in the tile
// range).  A thread holds 8 rows of up to four source blocks (64 registers
// for FP64) while it writes every member's digits: two blocks per SM (three
// spill).
constexpr int FUSED_PREP_BLOCKS = 2;
template <int S, typename T>
__global__ void __launch_bounds__(256, FUSED_PREP_BLOCKS) prep_fused_kernel(
    const T *__restrict__ A, int64_t lda, bool trans, const int *__restrict__ expo,
    const OpDesc *__restrict__ ops, int nops, const OpTerm *__restrict__ fsrc, int64_t ntiles, Families fams,
    uint8_t *ws) {
    constexpr int SMEM_OPS = 192;  // Strassen depth 2: about 2 x 49 operands per block
    __shared__ OpDesc s_ops[SMEM_OPS];
    const bool cached = nops <= SMEM_OPS;
    if (cached) {
        for (int i = threadIdx.x; i < nops; i += blockDim.x) s_ops[i] = ops[i];
        __syncthreads();
    }
    const OpDesc *o = cached ? s_ops : ops;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t local;
        const int lead = op_of_tile(o, nops, tile, &local);
        if (o[lead].fuse_uni)
            prep_fused_tile<S, T, true>(A, lda, trans, expo, o, lead, fsrc, local, fams, ws);
        else
            prep_fused_tile<S, T, false>(A, lda, trans, expo, o, lead, fsrc, local, fams, ws);
    }
}

// Batched calls: the prep tiles of all problems in one persistent grid.  A
// block walks its tiles in increasing order and keeps a cursor on the
// problem table (prefix prep_base), so locating a tile's problem costs one
// binary search per block.
// FP32 inputs with up to 3 digits (32-bit arithmetic, sums kept in
// registers: prep_tile_narrow) take no shared memory and run six resident
// blocks per SM (40 registers); others four.
template <typename T, int S>
__host__ __device__ constexpr bool batched_narrow() { return sizeof(T) == 4 && S <= 3; }
template <typename T, int S>
constexpr int batched_prep_blocks() { return batched_narrow<T, S>() ? 6 : 4; }

template <int S, typename T>
__global__ void __launch_bounds__(256, batched_prep_blocks<T, S>()) batched_prep_kernel(const BatchProb *__restrict__ probs, int64_t count,
                                                              const int *__restrict__ expo, int64_t ntiles,
                                                              uint8_t *planes) {
    __shared__ int64_t sV[batched_narrow<T, S>() ? 1 : PREP_SV];
    // Each block takes a contiguous range of tiles, so its problem cursor
    // moves by at most a few problems over the whole range (a grid-stride
    // walk would skip gridDim.x tiles, i.e. several small problems, per step,
    // each skip a dependent load before the tile's data loads can start).
    const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
    int64_t tile = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t tile_end = tile + per < ntiles ? tile + per : ntiles;
    if (tile >= tile_end) return;
    int64_t lo = 0, hi = count - 1;  // last problem with prep_base <= tile
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (probs[mid].prep_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    int64_t pi = lo;
    for (; tile < tile_end; ++tile) {
        while (pi + 1 < count && probs[pi + 1].prep_base <= tile) ++pi;
        const BatchProb &bp = probs[pi];
        OpDesc od{};
        od.nterms = 1;
        od.K_pitch = static_cast<int32_t>(bp.K_pitch);
        od.P_pad = static_cast<int32_t>(bp.P_pad);
        od.tile_base = bp.prep_base;
        const OpTerm term{0, 0, static_cast<int32_t>(bp.m), static_cast<int32_t>(bp.n), 1, 0};
        Family fam{};
        fam.K_pitch = bp.K_pitch;
        fam.cols = bp.ncb * BLOCK_COLS;
        fam.offset = bp.plane_off;
        const int lgtc = bp.tc == 64 ? 6 : (bp.tc == 128 ? 7 : 8);
        if constexpr (batched_narrow<T, S>())
            prep_tile_narrow<S, T>(static_cast<const T *>(bp.A), bp.lda, false, expo + bp.col_off, od, &term, tile,
                                   fam, planes, lgtc);
        else
            prep_tile<S, T>(static_cast<const T *>(bp.A), bp.lda, false, expo + bp.col_off, od, &term, tile, fam,
                            planes, sV, lgtc);
    }
}

// Batched calls: exponents of every column of every problem.  Block (x, y):
// problem y (then y + gridDim.y, ...), columns 64 x .. 64 x + 63; the four
// warps of each column pair split the rows and combine their maxima in
// shared memory (narrow problems waste no 256-column blocks).
template <typename T>
__global__ void __launch_bounds__(256) batched_expo_kernel(const BatchProb *__restrict__ probs, int64_t count,
                                                           int *expo, int *status) {
    __shared__ unsigned long long smax[4][64];
    const int cl = threadIdx.x & 63, rg = threadIdx.x >> 6;
    for (int64_t pi = blockIdx.y; pi < count; pi += gridDim.y) {
        const BatchProb &bp = probs[pi];
        const int64_t j = static_cast<int64_t>(blockIdx.x) * 64 + cl;
        if (static_cast<int64_t>(blockIdx.x) * 64 >= bp.n || bp.m == 0) continue;  // block-uniform
        unsigned long long mx = 0;
        if (j < bp.n) {
            const T *a = static_cast<const T *>(bp.A) + j;
            int64_t i = rg;
            for (; i + 12 < bp.m; i += 16) {  // four independent loads in flight
                const unsigned long long b0 = abs_bits(a[(i + 0) * bp.lda]), b1 = abs_bits(a[(i + 4) * bp.lda]);
                const unsigned long long b2 = abs_bits(a[(i + 8) * bp.lda]), b3 = abs_bits(a[(i + 12) * bp.lda]);
                mx = max(mx, max(max(b0, b1), max(b2, b3)));
            }
            for (; i < bp.m; i += 4) mx = max(mx, abs_bits(a[i * bp.lda]));
        }
        smax[rg][cl] = mx;
        __syncthreads();
        if (rg == 0 && j < bp.n) {
            const unsigned long long m = max(max(smax[0][cl], smax[1][cl]), max(smax[2][cl], smax[3][cl]));
            expo[bp.col_off + j] = column_exponent<T>(m, status);
        }
        __syncthreads();
    }
}

// Batched calls with device-resident pointer arrays: copy the problems' A_i
// and C_i into the problem table (every call, so a replayed graph reads the
// arrays as they are at replay time).
__global__ void batched_ptrs_kernel(BatchProb *probs, int64_t count, const void *const *A, void *const *C) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        probs[i].A = A[i];
        probs[i].C = C[i];
    }
}

// Batched calls: low(C_i) <- 0 for the problems with m_i == 0 (one block per
// problem, grid-stride over problems).
template <typename T>
__global__ void __launch_bounds__(256) batched_zero_kernel(const BatchProb *probs, int64_t count) {
    for (int64_t pi = blockIdx.x; pi < count; pi += gridDim.x) {
        const BatchProb &bp = probs[pi];
        if (bp.m != 0 || bp.n == 0) continue;
        T *C = static_cast<T *>(bp.C);
        const int64_t total = bp.n * (bp.n + 1) / 2;
        for (int64_t x = threadIdx.x; x < total; x += blockDim.x) {
            // x = j (j + 1) / 2 + k, k <= j
            int64_t j = static_cast<int64_t>((sqrt(8.0 * static_cast<double>(x) + 1.0) - 1.0) * 0.5);
            while (j * (j + 1) / 2 > x) --j;
            while ((j + 1) * (j + 2) / 2 <= x) ++j;
            C[j * bp.ldc + (x - j * (j + 1) / 2)] = T(0);
        }
    }
}

// Persistent grid: four 256-thread blocks per SM (64 registers each).
static unsigned prep_grid(int64_t ntiles, int per_sm = 4) {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!sms[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = n > 0 ? n : 1;
    }
    const int64_t cap = per_sm * static_cast<int64_t>(sms[dev]);
    return static_cast<unsigned>(ntiles < cap ? ntiles : cap);
}

// Native FP64 operands: U[k][c] = sum_t coef_t * a * 2^-e  (FP64, row-major
// [k][col] with leading dimension fam.cols).
template <typename T>
__global__ void __launch_bounds__(256) prep_f64_kernel(const T *__restrict__ A, int64_t lda, bool trans,
                                                       const int *__restrict__ expo,
                                                       const OpDesc *__restrict__ ops, int nops,
                                                       const OpTerm *__restrict__ terms,
                                                       Families fams, uint8_t *ws) {
    const int64_t tile = blockIdx.x;
    int64_t local;
    const OpDesc od = ops[op_of_tile(ops, nops, tile, &local)];
    const int tiles_k = od.K_pitch / PREP_K;
    const int k0 = static_cast<int>(local % tiles_k) * PREP_K;
    const int c0 = static_cast<int>(local / tiles_k) * PREP_C;
    const int cc = threadIdx.x & 63;
    const int kr0 = threadIdx.x >> 6;
    double V[16];
#pragma unroll
    for (int it = 0; it < 16; ++it) V[it] = 0.0;
    for (int t = 0; t < od.nterms; ++t) {
        const OpTerm tm = terms[od.first_term + t];
        const int c = c0 + cc;
        if (c < tm.cols) {
            const int x = -expo[tm.col0 + c];
            const int64_t rs = trans ? 1 : lda, cs = trans ? lda : 1;
            const T *col = A + (tm.col0 + c) * cs;
#pragma unroll
            for (int it = 0; it < 16; ++it) {
                const int k = k0 + kr0 + 4 * it;
                if (k < tm.rows) {
                    const double v = scale2d(static_cast<double>(col[(tm.row0 + k) * rs]), x);
                    V[it] = tm.coef > 0 ? V[it] + v : V[it] - v;
                }
            }
        }
    }
    const Family fam = fams.f[od.family];
    double *out = reinterpret_cast<double *>(ws + fam.offset);
#pragma unroll
    for (int it = 0; it < 16; ++it)
        out[(k0 + kr0 + 4 * it) * fam.cols + od.out_col + c0 + cc] = V[it];
}

// ------------------------------------------------------------- combine --
__device__ __forceinline__ int find_comb(const CombDesc *d, int nd, int64_t tile) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Combine tile of a block: COMB_ROWS x COMB_COLS entries of one region; the
// thread owns column lane and rows warp + 8 i (i < 8).  Every term's eight
// loads are issued together, and the term table is read straight from
// global memory (the same entries for the whole block).
constexpr int COMB_RPT = COMB_ROWS / 8;  // rows per thread

// An int128 as the nearest double: the top 64 significant bits with a
// sticky bit for the rest are rounded once by the 64-bit conversion (the
// sticky bit lies 11 places below the rounding point, so ties stay exact).
__device__ __forceinline__ double i128_to_double(__int128 s) {
    const bool neg = s < 0;
    const unsigned __int128 u = neg ? static_cast<unsigned __int128>(0) - static_cast<unsigned __int128>(s)
                                    : static_cast<unsigned __int128>(s);
    const uint64_t hi = static_cast<uint64_t>(u >> 64), lo = static_cast<uint64_t>(u);
    double r;
    if (hi == 0) {
        r = __ull2double_rn(lo);
    } else {
        const int sh = 64 - __clzll(static_cast<long long>(hi));  // 1..64
        const uint64_t below = sh == 64 ? lo : lo & ((1ull << sh) - 1);
        const uint64_t top = static_cast<uint64_t>(u >> sh) | (below != 0 ? 1ull : 0ull);
        r = __ull2double_rn(top) * exp2i(sh);
    }
    return neg ? -r : r;
}

// v * 2^sh in the accumulator type: int128, or uint64 for the sums taken
// modulo 2^64 (the shift done on the unsigned bits).
template <typename Acc>
__device__ __forceinline__ Acc shl(int64_t v, int sh) {
    if constexpr (sizeof(Acc) == 16)
        return static_cast<__int128>(static_cast<unsigned __int128>(static_cast<__int128>(v)) << sh);
    else
        return static_cast<uint64_t>(v) << sh;
}

// The accumulated sum as a signed value (a uint64 sum is the two's
// complement of the exact result, which fits in int64).
template <typename Acc>
__device__ __forceinline__ double acc_to_double(Acc s) {
    if constexpr (sizeof(Acc) == 16) return i128_to_double(s);
    else return static_cast<double>(static_cast<int64_t>(s));
}

template <typename Acc>
__device__ __forceinline__ float acc_to_float(Acc s) {
    if constexpr (sizeof(Acc) == 16) return static_cast<float>(i128_to_double(s));
    else return __ll2float_rn(static_cast<int64_t>(s));
}

// Exact Strassen result sums: region = sum_r coef_r * T_r * 2^(shift_r),
// added in units of 2^smin (the smallest term shift), then one rounding to
// the output type and the column scale 2^(e_j + e_k).  The sum is exact.
// The terms can be far larger than the result (deep recursion and
// Winograd's operands give products up to 2^(t_u + t_v) above a plain one,
// and they cancel), but the result itself is an entry of A^T A, at most m
// in scaled units.  Where that bound is below 2^63 in units of 2^smin, the
// sum is taken modulo 2^64 (uint64 wraps; the exact result is its two's
// complement value); else (d.wide) in int128.
template <typename Acc, typename TOut>
__device__ __forceinline__ void combine_region(const CombDesc &d, int r0, int col,
                                               const CombTerm *__restrict__ cterms,
                                               const int64_t *__restrict__ M, TOut *C, int64_t ldc, bool packed,
                                               const int *__restrict__ expo, double alpha, double beta) {
    Acc sum[COMB_RPT];
#pragma unroll
    for (int i = 0; i < COMB_RPT; ++i) sum[i] = 0;
    // (issuing the next term's loads before adding the current one doubled
    // the registers, halved the resident blocks and measured 0.23 against
    // 0.14 ms at 8192^2 depth 1)
    for (int t = 0; t < d.nterms; ++t) {
        const CombTerm ct = cterms[d.first_term + t];
        const int64_t *src = M + ct.src_off + col;
        int64_t v[COMB_RPT];
#pragma unroll
        for (int i = 0; i < COMB_RPT; ++i) {
            const int row = r0 + 8 * i;
            v[i] = row < d.rows ? src[static_cast<int64_t>(row) * ct.ld] : 0;
        }
        const int dsh = ct.shift - d.smin;  // >= 0
#pragma unroll
        for (int i = 0; i < COMB_RPT; ++i) {
            const Acc x = shl<Acc>(v[i], dsh);
            sum[i] += ct.coef > 0 ? x : -x;
        }
    }
    const int xc = -(T_FRAC + 2 * DIGIT_TOP_BITS) + d.smin + expo[d.e_col0 + col];
#pragma unroll
    for (int i = 0; i < COMB_RPT; ++i) {
        const int row = r0 + 8 * i;
        if (row >= d.rows) break;
        if (d.diag && col > row + d.diag_off) continue;  // upper triangle: never written
        const int x = xc + expo[d.e_row0 + row];
        TOut *c = packed ? C + packed_at(d.e_row0 + row, d.e_col0 + col)
                         : C + d.c_off + static_cast<int64_t>(row) * ldc + col;
        // A 64-bit sum goes to FP64 on the integer pipe (GB300's FP64 rate is
        // low); int128 sums and results outside the normal range take the
        // FP64 route.  FP32 output keeps the hardware conversion, which
        // measured faster than the integer construction.
        if constexpr (sizeof(TOut) == 8) {
            double r;
            if (sizeof(Acc) == 16 || !ldexp_i64_rn(static_cast<int64_t>(sum[i]), x, r))
                r = scale2d(acc_to_double(sum[i]), x);
            store_scaled(c, r, alpha, beta);
        } else {
            store_scaled(c, scale2f(acc_to_float(sum[i]), x), alpha, beta);
        }
    }
}

template <typename TOut>
__global__ void __launch_bounds__(256) combine_i64_kernel(const CombDesc *__restrict__ descs, int nd,
                                                          const CombTerm *__restrict__ cterms,
                                                          const int64_t *__restrict__ M, TOut *C,
                                                          int64_t ldc, bool packed, const int *__restrict__ expo,
                                                          double alpha, double beta) {
    const CombDesc d = descs[find_comb(descs, nd, blockIdx.x)];
    const int64_t local = blockIdx.x - d.tile_base;
    const int tcols = (d.cols + COMB_COLS - 1) / COMB_COLS;
    const int r0 = static_cast<int>(local / tcols) * COMB_ROWS + (threadIdx.x >> 5);
    const int col = static_cast<int>(local % tcols) * COMB_COLS + (threadIdx.x & 31);
    if (col >= d.cols) return;
    if (d.wide)
        combine_region<__int128>(d, r0, col, cterms, M, C, ldc, packed, expo, alpha, beta);
    else
        combine_region<uint64_t>(d, r0, col, cterms, M, C, ldc, packed, expo, alpha, beta);
}

// Native FP64 (and FP8-mode) result sums, in the fixed term order, then the
// column scales.
template <typename TOut>
__global__ void __launch_bounds__(256) combine_f64_kernel(const CombDesc *__restrict__ descs, int nd,
                                                          const CombTerm *__restrict__ cterms,
                                                          const double *__restrict__ M, TOut *C,
                                                          int64_t ldc, bool packed, const int *__restrict__ expo,
                                                          double alpha, double beta) {
    const CombDesc d = descs[find_comb(descs, nd, blockIdx.x)];
    const int64_t local = blockIdx.x - d.tile_base;
    const int tcols = (d.cols + COMB_COLS - 1) / COMB_COLS;
    const int r0 = static_cast<int>(local / tcols) * COMB_ROWS + (threadIdx.x >> 5);
    const int col = static_cast<int>(local % tcols) * COMB_COLS + (threadIdx.x & 31);
    if (col >= d.cols) return;
    double sum[COMB_RPT];
#pragma unroll
    for (int i = 0; i < COMB_RPT; ++i) sum[i] = 0.0;
    for (int t = 0; t < d.nterms; ++t) {
        const CombTerm ct = cterms[d.first_term + t];
        const double *src = M + ct.src_off + col;
        double v[COMB_RPT];
#pragma unroll
        for (int i = 0; i < COMB_RPT; ++i) {
            const int row = r0 + 8 * i;
            v[i] = row < d.rows ? src[static_cast<int64_t>(row) * ct.ld] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < COMB_RPT; ++i) sum[i] = ct.coef > 0 ? sum[i] + v[i] : sum[i] - v[i];
    }
    const int ec = expo[d.e_col0 + col];
#pragma unroll
    for (int i = 0; i < COMB_RPT; ++i) {
        const int row = r0 + 8 * i;
        if (row >= d.rows) break;
        if (d.diag && col > row + d.diag_off) continue;  // upper triangle: never written
        store_scaled(packed ? C + packed_at(d.e_row0 + row, d.e_col0 + col)
                            : C + d.c_off + static_cast<int64_t>(row) * ldc + col,
                     static_cast<TOut>(scale2d(sum[i], expo[d.e_row0 + row] + ec)), alpha, beta);
    }
}

// ---------------------------------------------------- native FP64 leaf --
// One TILE_M x TILE_N (128 x 96) tile per block with FP64 tensor-core MMA
// (m8n8k4); 8 warps, each 32 rows x 48 columns.
__device__ __forceinline__ void dmma_8x8x4(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256) leaf_f64_kernel(const __grid_constant__ LeafParams p) {
    constexpr int KT = 16, LDU = TILE_M + 4, LDV = TILE_N + 4;
    __shared__ double Us[KT][LDU];
    __shared__ double Vs[KT][LDV];
    const LeafTask t = p.tasks[blockIdx.x];
    const double *U = t.fam_u < 0 ? p.A64 : p.fam64[t.fam_u];
    const double *V = t.fam_v < 0 ? p.A64 : p.fam64[t.fam_v];
    // operand (row k, column c) at base[k * rstride + c * cstride]: families are
    // [k][col] arrays; A itself may be the transpose of the operand
    const bool tu = t.fam_u < 0 && p.a_trans, tv = t.fam_v < 0 && p.a_trans;
    const int64_t ldu = t.fam_u < 0 ? p.lda : p.fam_ld[t.fam_u];
    const int64_t ldv = t.fam_v < 0 ? p.lda : p.fam_ld[t.fam_v];
    const int64_t urs = tu ? 1 : ldu, ucs = tu ? ldu : 1, vrs = tv ? 1 : ldv, vcs = tv ? ldv : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 48;
    double acc[4][6][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

    const int lc = threadIdx.x & 127, lk = threadIdx.x >> 7;
    for (int k0 = 0; k0 < t.klen; k0 += KT) {
#pragma unroll
        for (int i = 0; i < KT / 2; ++i) {
            const int kk = lk + 2 * i;
            const int64_t ku = static_cast<int64_t>(t.k0) + k0 + kk, kv = static_cast<int64_t>(t.k0v) + k0 + kk;
            const bool kin = (k0 + kk) < t.klen;
            Us[kk][lc] = (kin && lc < t.rows) ? U[ku * urs + (t.col_u + lc) * ucs] : 0.0;
            if (lc < TILE_N) Vs[kk][lc] = (kin && lc < t.cols) ? V[kv * vrs + (t.col_v + lc) * vcs] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k4 = 0; k4 < KT; k4 += 4) {
            double a[4], b[6];
#pragma unroll
            for (int fm = 0; fm < 4; ++fm) a[fm] = Us[k4 + (lane & 3)][wm + 8 * fm + (lane >> 2)];
#pragma unroll
            for (int fn = 0; fn < 6; ++fn) b[fn] = Vs[k4 + (lane & 3)][wn + 8 * fn + (lane >> 2)];
#pragma unroll
            for (int fm = 0; fm < 4; ++fm)
#pragma unroll
                for (int fn = 0; fn < 6; ++fn) dmma_8x8x4(acc[fm][fn], a[fm], b[fn]);
        }
        __syncthreads();
    }
    const bool to_m = t.kind == OUT_M_F64;
    double *out = reinterpret_cast<double *>(to_m ? p.M : p.C) + (p.packed && !to_m ? 0 : t.out_off);
#pragma unroll
    for (int fm = 0; fm < 4; ++fm) {
        const int row = wm + 8 * fm + (lane >> 2);
#pragma unroll
        for (int fn = 0; fn < 6; ++fn) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = wn + 8 * fn + 2 * (lane & 3) + h;
                if (row < t.rows && col < t.cols && (!t.diag || col <= row + t.diag_off)) {
                    double *o = p.packed && !to_m ? out + packed_at(t.out_off + row, t.out_ld + col)
                                                  : out + static_cast<int64_t>(row) * t.out_ld + col;
                    if (t.kind == OUT_M_F64)
                        *o = acc[fm][fn][h];
                    else
                        store_scaled(o, acc[fm][fn][h], p.alpha, p.beta);
                }
            }
        }
    }
}

template <typename T>
__global__ void scale_lower_kernel(T *C, int64_t n, int64_t ldc, bool packed, double beta) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y + static_cast<int64_t>(blockIdx.z) * 65535;
    if (j < n && k <= j) {
        T *c = packed ? C + packed_at(j, k) : C + j * ldc + k;
        *c = beta != 0.0 ? static_cast<T>(beta * *c) : T(0);
    }
}

}  // namespace

// ------------------------------------------------------------- launchers --
cudaError_t launch_batched_expo(const BatchPlan &B, const BatchProb *probs, bool is_f32, int *expo, int *status,
                                cudaStream_t s) {
    if (B.count == 0 || B.max_col_chunks == 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>(B.max_col_chunks), static_cast<unsigned>(B.count < 65535 ? B.count : 65535));
    if (is_f32)
        batched_expo_kernel<float><<<grid, 256, 0, s>>>(probs, B.count, expo, status);
    else
        batched_expo_kernel<double><<<grid, 256, 0, s>>>(probs, B.count, expo, status);
    return cudaGetLastError();
}

cudaError_t launch_batched_ptrs(BatchProb *probs, int64_t count, const void *const *A, void *const *C,
                                cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const unsigned g = static_cast<unsigned>(count < 256 * 1024 ? (count + 255) / 256 : 1024);
    batched_ptrs_kernel<<<g, 256, 0, s>>>(probs, count, A, C);
    return cudaGetLastError();
}

cudaError_t launch_batched_zero(const BatchProb *probs, int64_t count, bool is_f32, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const unsigned g = static_cast<unsigned>(count < 65535 ? count : 65535);
    if (is_f32)
        batched_zero_kernel<float><<<g, 256, 0, s>>>(probs, count);
    else
        batched_zero_kernel<double><<<g, 256, 0, s>>>(probs, count);
    return cudaGetLastError();
}

cudaError_t launch_batched_prep(const BatchPlan &B, const BatchProb *probs, bool is_f32, const int *expo,
                                uint8_t *planes, cudaStream_t s) {
    if (B.prep_tiles == 0) return cudaSuccess;
#define ATA_PREP_B(SS)                                                                                        \
    case SS:                                                                                                  \
        if (is_f32)                                                                                           \
            batched_prep_kernel<SS, float><<<prep_grid(B.prep_tiles, batched_prep_blocks<float, SS>()), 256, 0, \
                                            s>>>(probs, B.count, expo, B.prep_tiles, planes);                 \
        else                                                                                                  \
            batched_prep_kernel<SS, double><<<prep_grid(B.prep_tiles, batched_prep_blocks<double, SS>()), 256, \
                                             0, s>>>(probs, B.count, expo, B.prep_tiles, planes);             \
        break;
    switch (B.slices) {
        ATA_PREP_B(1)
        ATA_PREP_B(2)
        ATA_PREP_B(3)
        ATA_PREP_B(4)
        ATA_PREP_B(5)
        ATA_PREP_B(6)
        ATA_PREP_B(7)
        default: return cudaErrorInvalidValue;
    }
#undef ATA_PREP_B
    return cudaGetLastError();
}

cudaError_t launch_colmax(const void *A, int64_t m, int64_t n, int64_t lda, bool is_f32, bool trans,
                          unsigned long long *colmax, int *expo, int *status, cudaStream_t s) {
    if (trans) {  // operand column j is row j of A: one warp per row, exponents written directly
        const unsigned g = static_cast<unsigned>((n + 7) / 8);
        if (is_f32)
            rowmax_expo_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(A), n, m, lda, expo, status);
        else
            rowmax_expo_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(A), n, m, lda, expo, status);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * n, s);
    if (e != cudaSuccess) return e;
    const int rows_per_block = 64;
    const int64_t gy = (m + rows_per_block - 1) / rows_per_block;
    int rpb = rows_per_block;
    int64_t gyy = gy;
    while (gyy > 65535) {  // keep grid.y legal
        rpb *= 2;
        gyy = (m + rpb - 1) / rpb;
    }
    dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(gyy > 0 ? gyy : 1));
    if (is_f32)
        colmax_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(A), m, n, lda, rpb, colmax);
    else
        colmax_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(A), m, n, lda, rpb, colmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g = static_cast<unsigned>((n + 255) / 256);
    if (is_f32)
        expo_kernel<float><<<g, 256, 0, s>>>(colmax, n, expo, status);
    else
        expo_kernel<double><<<g, 256, 0, s>>>(colmax, n, expo, status);
    return cudaGetLastError();
}

template <int S>
static void prep_digits_dispatch(const Plan &P, const void *A, bool is_f32, const int *expo,
                                 const uint8_t *tables, uint8_t *ws, const Families &F,
                                 cudaStream_t s) {
    const OpDesc *ops = reinterpret_cast<const OpDesc *>(tables + P.t_ops);
    const OpTerm *terms = reinterpret_cast<const OpTerm *>(tables + P.t_terms);
    const OpTerm *fsrc = reinterpret_cast<const OpTerm *>(tables + P.t_fsrc);
    const int nops = static_cast<int>(P.ops.size()), nterms = static_cast<int>(P.terms.size());
    const bool tr = P.p.trans != 0;
    const int64_t t0 = P.fused_tiles, nt = P.prep_tiles;
    if (t0 > 0) {  // fused groups (digit modes other than FP8)
        const unsigned gf = prep_grid(t0, FUSED_PREP_BLOCKS);
        if (is_f32)
            prep_fused_kernel<S, float><<<gf, 256, 0, s>>>(static_cast<const float *>(A), P.p.lda, tr, expo, ops,
                                                            nops, fsrc, t0, F, ws);
        else
            prep_fused_kernel<S, double><<<gf, 256, 0, s>>>(static_cast<const double *>(A), P.p.lda, tr, expo,
                                                             ops, nops, fsrc, t0, F, ws);
    }
    if (nt <= t0) return;
    const unsigned g = prep_grid(nt - t0);
    if (S == 1 && P.p.mode == MODE_F32_FP8)  // FP8 mode: float A, one E4M3 plane
        prep_digits_kernel<1, float, true><<<g, 256, 0, s>>>(static_cast<const float *>(A), P.p.lda, tr, expo,
                                                              ops, nops, terms, nterms, t0, nt, F, ws);
    else if (is_f32)
        prep_digits_kernel<S, float><<<g, 256, 0, s>>>(static_cast<const float *>(A), P.p.lda, tr, expo, ops,
                                                        nops, terms, nterms, t0, nt, F, ws);
    else
        prep_digits_kernel<S, double><<<g, 256, 0, s>>>(static_cast<const double *>(A), P.p.lda, tr, expo, ops,
                                                         nops, terms, nterms, t0, nt, F, ws);
}

cudaError_t launch_prep(const Plan &P, const void *A, bool is_f32, const int *expo,
                        const uint8_t *tables, uint8_t *ws, cudaStream_t s) {
    if (P.ops.empty() || P.prep_tiles == 0) return cudaSuccess;
    if (P.prep_tiles > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
    Families F{};
    for (size_t i = 0; i < P.families.size() && i < MAX_FAMILIES; ++i) F.f[i] = P.families[i];
    if (P.p.mode == MODE_F64) {
        const OpDesc *ops = reinterpret_cast<const OpDesc *>(tables + P.t_ops);
        const OpTerm *terms = reinterpret_cast<const OpTerm *>(tables + P.t_terms);
        prep_f64_kernel<double><<<static_cast<unsigned>(P.prep_tiles), 256, 0, s>>>(
            static_cast<const double *>(A), P.p.lda, P.p.trans != 0, expo, ops, static_cast<int>(P.ops.size()),
            terms, F, ws);
        return cudaGetLastError();
    }
    switch (P.slices) {
        case 1: prep_digits_dispatch<1>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 2: prep_digits_dispatch<2>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 3: prep_digits_dispatch<3>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 4: prep_digits_dispatch<4>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 5: prep_digits_dispatch<5>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 6: prep_digits_dispatch<6>(P, A, is_f32, expo, tables, ws, F, s); break;
        case 7: prep_digits_dispatch<7>(P, A, is_f32, expo, tables, ws, F, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_leaf_f64(const Plan &P, const LeafParams &lp, cudaStream_t s) {
    if (P.tasks.empty()) return cudaSuccess;
    leaf_f64_kernel<<<static_cast<unsigned>(P.tasks.size()), 256, 0, s>>>(lp);
    return cudaGetLastError();
}

cudaError_t launch_leaf_f64_group(const LeafParams &lp, int64_t first, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    LeafParams g = lp;
    g.tasks = lp.tasks + first;
    g.ntasks = static_cast<int>(count);
    leaf_f64_kernel<<<static_cast<unsigned>(count), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_combine(const Plan &P, const uint8_t *tables, const void *M, void *C,
                           const int *expo, double alpha, double beta, cudaStream_t s) {
    if (P.combs.empty() || P.comb_tiles == 0) return cudaSuccess;
    const CombDesc *d = reinterpret_cast<const CombDesc *>(tables + P.t_combs);
    const CombTerm *t = reinterpret_cast<const CombTerm *>(tables + P.t_cterms);
    const unsigned g = static_cast<unsigned>(P.comb_tiles);
    const int nd = static_cast<int>(P.combs.size());
    const bool pk = P.p.packed != 0;
    if (P.p.mode == MODE_F64)
        combine_f64_kernel<double><<<g, 256, 0, s>>>(d, nd, t, static_cast<const double *>(M),
                                                      static_cast<double *>(C), P.p.ldc, pk, expo, alpha, beta);
    else if (P.p.mode == MODE_F32_FP8)  // FP8 products are FP32 sums, stored as double
        combine_f64_kernel<float><<<g, 256, 0, s>>>(d, nd, t, static_cast<const double *>(M),
                                                     static_cast<float *>(C), P.p.ldc, pk, expo, alpha, beta);
    else if (P.p.mode == MODE_F64_EMU)
        combine_i64_kernel<double><<<g, 256, 0, s>>>(d, nd, t, static_cast<const int64_t *>(M),
                                                      static_cast<double *>(C), P.p.ldc, pk, expo, alpha, beta);
    else
        combine_i64_kernel<float><<<g, 256, 0, s>>>(d, nd, t, static_cast<const int64_t *>(M),
                                                     static_cast<float *>(C), P.p.ldc, pk, expo, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_scale_lower(void *C, int64_t n, int64_t ldc, bool is_f32, double beta, cudaStream_t s,
                               bool packed) {
    if (n <= 0) return cudaSuccess;
    dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(n < 65535 ? n : 65535),
              static_cast<unsigned>((n + 65534) / 65535));
    if (is_f32)
        scale_lower_kernel<float><<<grid, 256, 0, s>>>(static_cast<float *>(C), n, ldc, packed, beta);
    else
        scale_lower_kernel<double><<<grid, 256, 0, s>>>(static_cast<double *>(C), n, ldc, packed, beta);
    return cudaGetLastError();
}

}  // namespace ata

namespace ata {

// Prep launch from explicit tables (used by the allocation-free entry point,
// whose tables live in its fixed device scratch rather than in a plan).
cudaError_t launch_prep_digits_raw(int slices, const void *A, bool is_f32, int64_t lda, const int *expo,
                                   const OpDesc *ops, int nops, const OpTerm *terms, const Family &fam0,
                                   int64_t prep_tiles, uint8_t *ws, cudaStream_t s) {
    if (prep_tiles <= 0) return cudaSuccess;
    if (prep_tiles > 0x7FFFFFFF) return cudaErrorInvalidConfiguration;
    Families F{};
    F.f[0] = fam0;
    const unsigned g = prep_grid(prep_tiles);
#define ATA_PREP_RAW(SS)                                                                                   \
    case SS:                                                                                               \
        if (is_f32)                                                                                        \
            prep_digits_kernel<SS, float><<<g, 256, 0, s>>>(static_cast<const float *>(A), lda, false, expo, ops, \
                                                             nops, terms, 1, 0, prep_tiles, F, ws);           \
        else                                                                                               \
            prep_digits_kernel<SS, double><<<g, 256, 0, s>>>(static_cast<const double *>(A), lda, false, expo, \
                                                              ops, nops, terms, 1, 0, prep_tiles, F, ws);     \
        break;
    switch (slices) {
        ATA_PREP_RAW(1)
        ATA_PREP_RAW(2)
        ATA_PREP_RAW(3)
        ATA_PREP_RAW(4)
        ATA_PREP_RAW(5)
        ATA_PREP_RAW(6)
        ATA_PREP_RAW(7)
        default: return cudaErrorInvalidValue;
    }
#undef ATA_PREP_RAW
    return cudaGetLastError();
}

}  // namespace ata
