// Scaled integers to IEEE binary64 with integer operations only.
//
// The leaf's epilogue and the combine turn each exact integer sum T into
// T * 2^e.  GB300 runs FP64 arithmetic (and conversions to FP64) at a small
// fraction of its integer rate, so the rounded result is built from T's bits
// instead: normalise, keep the leading 53 bits, round to nearest with ties
// to even on the bits below (IEEE 754-2019, 4.3.1 roundTiesToEven), and add
// the biased exponent.  Where the result would not be a normal number the
// function returns false and the caller takes the floating-point route.
// Host and device code share this function (the CPU tests check it against
// the host's correctly rounded conversion).  FP32 output keeps the hardware
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
