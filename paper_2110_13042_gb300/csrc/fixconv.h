// Conversions between IEEE binary64 and scaled integers, with integer
// operations only.
//
// binary64 -> fixed point (the digit prep): round(a * 2^sh), half away from
// zero, from a's bits.
//
// fixed point -> binary64 (the leaf's epilogue and the combine): each exact
// integer sum T becomes T * 2^e.  GB300 runs FP64 arithmetic (and conversions to FP64) at a small
// fraction of its integer rate, so the rounded result is built from T's bits
// instead: normalise, keep the leading 53 bits, round to nearest with ties
// to even on the bits below (IEEE 754-2019, 4.3.1 roundTiesToEven), and add
// the biased exponent.  Where the result would not be a normal number the
// function returns false and the caller takes the floating-point route.
// Host and device code share these functions (the CPU tests check them
// against the exact definitions and the host's correctly rounded conversion).  FP32 output keeps the hardware
// int64-to-float conversion, which measured faster than this construction.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define ATA_HD __host__ __device__ __forceinline__
#else
#define ATA_HD inline
#endif

namespace ata {

ATA_HD int clz64_(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll(static_cast<long long>(x));
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

ATA_HD double bits_to_double_(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(static_cast<long long>(b));
#else
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// round(a * 2^sh), half away from zero, for |a * 2^sh| <= 2^(53 + P) with
// P in {0, 1}.  With a = M 2^s' (M the 53-bit significand, s' its exponent)
// and s = s' + sh: r = (X + 2^u) / 2^(u + 1) (floor) with X = M 2^(P + 1 + L),
// L = max(s - P, 0) and u = max(P - s, 0) clamped to 62.  L > 0 only for a
// subnormal a in a column whose maximum is subnormal too; then u = 0 and r =
// M 2^s exactly.  X < 2^55 either way, so a clamped u gives 0, as the exact
// value below 1/2 requires.
template <int P>
ATA_HD int64_t fixed_of_f64(double a, int sh) {
    static_assert(P == 0 || P == 1, "X stays below 2^55");
    uint64_t bits;
#ifdef __CUDA_ARCH__
    bits = static_cast<uint64_t>(__double_as_longlong(a));
#else
    std::memcpy(&bits, &a, sizeof bits);
#endif
    const int eb = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
    const uint64_t M = eb ? (mant | (1ull << 52)) : mant;
    const int s = (eb ? eb - 1075 : -1074) + sh;
    const int L = s > P ? s - P : 0;
    const int u = (P - s < 0 ? 0 : P - s) > 62 ? 62 : (P - s < 0 ? 0 : P - s);
    const uint64_t r = ((M << (P + 1 + L)) + (1ull << u)) >> (u + 1);
    return (bits >> 63) ? -static_cast<int64_t>(r) : static_cast<int64_t>(r);
}

// Both round(a * 2^sh) and round(a * 2^(sh - 1)) (half away from zero) from
// one truncation q = floor(|a| 2^(sh + 1)): for v >= 0 with q = floor(2 v),
// floor(v + 1/2) = floor((q + 1) / 2) and floor(v / 2 + 1/2) = floor((q + 2) / 4),
// whatever fraction q dropped.  Same bound as fixed_of_f64: |a 2^sh| <= 2^(53 + P),
// so q < 2^(55 + P).
template <int P>
ATA_HD void fixed_pair_f64(double a, int sh, int64_t &x, int64_t &x_half) {
    static_assert(P == 0 || P == 1, "q stays below 2^56");
    uint64_t bits;
#ifdef __CUDA_ARCH__
    bits = static_cast<uint64_t>(__double_as_longlong(a));
#else
    std::memcpy(&bits, &a, sizeof bits);
#endif
    const int eb = static_cast<int>((bits >> 52) & 0x7FF);
    const uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
    const uint64_t M = eb ? (mant | (1ull << 52)) : mant;
    const int s1 = (eb ? eb - 1075 : -1074) + sh + 1;  // |a| 2^(sh + 1) = M 2^s1
    const int L = s1 > 0 ? s1 : 0;
    const int u = s1 < 0 ? (-s1 > 63 ? 63 : -s1) : 0;
    const uint64_t q = (M << L) >> u;
    const uint64_t r = (q + 1u) >> 1, rh = (q + 2u) >> 2;
    const bool neg = (bits >> 63) != 0;
    x = neg ? -static_cast<int64_t>(r) : static_cast<int64_t>(r);
    x_half = neg ? -static_cast<int64_t>(rh) : static_cast<int64_t>(rh);
}

// The same for an FP32 value (24-bit significand M, subnormal exponent -149),
// with P <= 37: X = M 2^(P + 1 + L) <= 2^(P + 25) or M 2^(s + 1) <= 2^(F + 1)
// with F = P + 23, so X < 2^62.
template <int P>
ATA_HD int64_t fixed_of_f32(float a, int sh) {
    static_assert(P >= 0 && P <= 37, "X stays below 2^62");
    uint32_t bits;
#ifdef __CUDA_ARCH__
    bits = __float_as_uint(a);
#else
    std::memcpy(&bits, &a, sizeof bits);
#endif
    const int eb = static_cast<int>(bits >> 23) & 0xFF;
    const uint64_t M = (bits & 0x7FFFFFu) | (static_cast<uint64_t>(eb != 0) << 23);
    const int s = (eb > 1 ? eb : 1) - 150 + sh;
    const int L = s > P ? s - P : 0;
    const int u = (P - s < 0 ? 0 : P - s) > 62 ? 62 : (P - s < 0 ? 0 : P - s);
    const uint64_t r = ((M << (P + 1 + L)) + (1ull << u)) >> (u + 1);
    return (bits >> 31) ? -static_cast<int64_t>(r) : static_cast<int64_t>(r);
}

// 32-bit form for |a 2^sh| <= 2^(P + 23) with P <= 6: X <= 2^(P + 24) < 2^31,
// and a rounding position past bit 30 leaves |a 2^sh| < 1/2, i.e. 0.
template <int P>
ATA_HD int32_t fixed32_of_f32(float a, int sh) {
    static_assert(P >= 0 && P <= 6, "X stays below 2^31");
    uint32_t bits;
#ifdef __CUDA_ARCH__
    bits = __float_as_uint(a);
#else
    std::memcpy(&bits, &a, sizeof bits);
#endif
    const int eb = static_cast<int>(bits >> 23) & 0xFF;
    const uint32_t M = (bits & 0x7FFFFFu) | (static_cast<uint32_t>(eb != 0) << 23);
    const int s = (eb > 1 ? eb : 1) - 150 + sh;
    const int L = s > P ? s - P : 0;
    const int u = P - s > 0 ? P - s : 0;
    const uint32_t r = u > 30 ? 0u : ((M << (P + 1 + L)) + (1u << u)) >> (u + 1);
    return (bits >> 31) ? -static_cast<int32_t>(r) : static_cast<int32_t>(r);
}

// out = T * 2^e rounded to the nearest double (ties to even).  Returns false
// (out untouched) unless the result is 0 or a normal number below 2^1023.
ATA_HD bool ldexp_i64_rn(int64_t T, int e, double &out) {
    if (T == 0) {
        out = 0.0;
        return true;
    }
    const uint64_t neg = T < 0 ? 1u : 0u;
    const uint64_t mag = neg ? 0ull - static_cast<uint64_t>(T) : static_cast<uint64_t>(T);
    const int lz = clz64_(mag);
    const uint64_t m = mag << lz;     // leading one at bit 63
    uint64_t mant = m >> 11;          // 53 bits, leading one at bit 52
    const uint64_t rest = m & 0x7FFu;  // the 11 bits rounded away
    mant += (rest > 0x400u || (rest == 0x400u && (mant & 1u))) ? 1u : 0u;
    const int E = 63 - lz + e;        // |T 2^e| = (mant / 2^52) 2^E before the carry
    if (E < -1022 || E > 1022) return false;
    // The leading one (bit 52, or bit 53 after a rounding carry) adds 1 (2)
    // to the exponent field E + 1022.
    out = bits_to_double_((neg << 63) | ((static_cast<uint64_t>(E + 1022) << 52) + mant));
    return true;
}

}  // namespace ata
