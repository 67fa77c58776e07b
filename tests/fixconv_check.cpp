// Checks the integer-only conversions of csrc/fixconv.h:
// - ldexp_i64_rn against the host's conversion: (double)T rounds to nearest,
//   ties to even, and ldexp by a power of two is exact while the result stays
//   normal;
// - fixed_of_f64, fixed_of_f32 and fixed32_of_f32 against round(a 2^sh),
//   half away from zero, computed exactly in 128-bit integers from a's
//   significand and exponent.
// Prints "<cases> <mismatches> <missed> <fixed cases> <fixed mismatches>" and
// exits 0.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "fixconv.h"

static uint64_t s = 0x243F6A8885A308D3ull;
static uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static long cases = 0, bad = 0, missed = 0;

static void check(int64_t T, int e) {
    ++cases;
    const double want = std::ldexp(static_cast<double>(T), e);
    double got = 1.5;
    const bool ok = ata::ldexp_i64_rn(T, e, got);
    const bool normal = T == 0 || (std::fabs(want) >= DBL_MIN && std::fabs(want) < 0x1p1023);
    if (ok && !(got == want && std::signbit(got) == std::signbit(want))) ++bad;
    if (!ok && normal) ++missed;
}

static long fcases = 0, fbad = 0;

// round(|a| 2^sh) half away from zero, exactly, for |a 2^sh| < 2^62
static uint64_t exact_fixed_mag(double a, int sh) {
    uint64_t bits;
    std::memcpy(&bits, &a, sizeof bits);
    const int eb = static_cast<int>(bits >> 52) & 0x7FF;
    const uint64_t M = (bits & 0xFFFFFFFFFFFFFull) | (eb ? (1ull << 52) : 0ull);
    const int s = (eb ? eb - 1075 : -1074) + sh;
    if (s >= 0) return M << s;
    if (-s > 120) return 0;
    const unsigned __int128 v = static_cast<unsigned __int128>(M);
    return static_cast<uint64_t>((v + (static_cast<unsigned __int128>(1) << (-s - 1))) >> (-s));
}

template <int P>
static void check_fixed(double a, int sh) {
    ++fcases;
    const uint64_t mag = exact_fixed_mag(a, sh);
    const int64_t want = std::signbit(a) ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
    if (ata::fixed_of_f64<P>(a, sh) != want) ++fbad;
    // the pair form: round(a 2^sh) and round(a 2^(sh - 1)) from one truncation
    const uint64_t mag_h = exact_fixed_mag(a, sh - 1);
    const int64_t want_h = std::signbit(a) ? -static_cast<int64_t>(mag_h) : static_cast<int64_t>(mag_h);
    int64_t x = 0, xh = 0;
    ata::fixed_pair_f64<P>(a, sh, x, xh);
    if (x != want || xh != want_h) ++fbad;
}

// a random double with exponent field eb (0: subnormal) and sign
static double make_double(int eb, bool neg) {
    const uint64_t bits = (static_cast<uint64_t>(neg) << 63) | (static_cast<uint64_t>(eb) << 52) |
                          (next() & 0xFFFFFFFFFFFFFull);
    double d;
    std::memcpy(&d, &bits, sizeof d);
    return d;
}

// every sh that keeps |a 2^sh| <= 2^(53 + P) (as the column exponents do), and
// a few far below it
template <int P>
static void fixed_cases(double a) {
    const int e = a == 0.0 ? -1074 : std::ilogb(a) + 1;  // |a| < 2^e
    const int top = 53 + P - e;                         // |a 2^top| < 2^(53 + P)
    for (int d = 0; d < 70; ++d) check_fixed<P>(a, top - d);
    check_fixed<P>(a, top - 200);
}

template <int P, bool NARROW>
static void check_fixed_f32(float a, int sh) {
    ++fcases;
    const uint64_t mag = exact_fixed_mag(static_cast<double>(a), sh);  // a float is exact as a double
    const int64_t want = std::signbit(a) ? -static_cast<int64_t>(mag) : static_cast<int64_t>(mag);
    int64_t got;
    if constexpr (NARROW)
        got = ata::fixed32_of_f32<P>(a, sh);
    else
        got = ata::fixed_of_f32<P>(a, sh);
    if (got != want) ++fbad;
}

// every sh that keeps |a 2^sh| <= 2^(23 + P), and one far below
template <int P, bool NARROW>
static void fixed_cases_f32(float a) {
    const int e = a == 0.0f ? -149 : std::ilogb(a) + 1;  // |a| < 2^e
    const int top = 23 + P - e;
    for (int d = 0; d < 40; ++d) check_fixed_f32<P, NARROW>(a, top - d);
    check_fixed_f32<P, NARROW>(a, top - 100);
}

static void all_f32(float a) {
    fixed_cases_f32<0, true>(a);   // one digit
    fixed_cases_f32<3, true>(a);   // two digits
    fixed_cases_f32<6, true>(a);   // three digits (F = 29)
    fixed_cases_f32<12, false>(a);
    fixed_cases_f32<21, false>(a);
    fixed_cases_f32<24, false>(a);  // the FP8 mode's fixed point (F = 47)
    fixed_cases_f32<30, false>(a);
}

int main() {
    const int64_t specials[] = {0, 1, -1, 2, 3, INT64_MAX, INT64_MIN, INT64_MIN + 1, (1ll << 53) - 1, 1ll << 53,
                                (1ll << 53) + 1, (1ll << 54) + 2, (1ll << 54) + 6, (1ll << 60) + (1ll << 7)};
    for (int64_t T : specials)
        for (int e = -1100; e <= 1100; e += 7) check(T, e);
    for (int i = 0; i < 2000000; ++i) {
        const uint64_t r = next();
        const int bits = 1 + static_cast<int>(next() % 63);
        int64_t T = static_cast<int64_t>(r >> (64 - bits));
        const int kind = static_cast<int>(next() % 4);
        if (kind == 1 && bits > 54) {  // an exact tie at the double rounding point
            const int drop = bits - 53;
            T = (T >> drop << drop) | (int64_t(1) << (drop - 1));
        }
        if (next() & 1) T = -T;
        int e = static_cast<int>(next() % 200) - 100;
        if (kind == 2) e = static_cast<int>(next() % 2300) - 1150;  // range edges
        check(T, e);
    }
    const double fspecial[] = {0.0, -0.0, 1.0, -1.0, 0.5, 1.5, 2.5, -2.5, 0x1p-1074, -0x1p-1074, 0x1.8p-1073,
                               0x1.fffffffffffffp+1023, -0x1.fffffffffffffp-1023, 0x1p-1022};
    for (double a : fspecial) {
        fixed_cases<0>(a);
        fixed_cases<1>(a);
    }
    for (int i = 0; i < 200000; ++i) {
        const int pick = static_cast<int>(next() % 8);
        const int eb = pick == 0 ? 0 : pick == 1 ? 1 + static_cast<int>(next() % 2046)
                                                : 1023 + static_cast<int>(next() % 64) - 32;
        const double a = make_double(eb, next() & 1);
        fixed_cases<0>(a);
        fixed_cases<1>(a);
    }
    const float f32special[] = {0.0f, -0.0f, 1.0f, -1.0f, 0.5f, 1.5f, 2.5f, -2.5f, 0x1p-149f, -0x1p-149f,
                                0x1.8p-148f, 0x1.fffffep+127f, -0x1.fffffep-127f, 0x1p-126f};
    for (float a : f32special) all_f32(a);
    for (int i = 0; i < 100000; ++i) {
        const int pick = static_cast<int>(next() % 8);
        const uint32_t eb = pick == 0 ? 0u : pick == 1 ? 1u + static_cast<uint32_t>(next() % 254)
                                                      : 127u + static_cast<uint32_t>(next() % 32) - 16u;
        const uint32_t bits = (static_cast<uint32_t>(next() & 1) << 31) | (eb << 23) |
                              static_cast<uint32_t>(next() & 0x7FFFFFu);
        float a;
        std::memcpy(&a, &bits, sizeof a);
        all_f32(a);
    }
    std::printf("%ld %ld %ld %ld %ld\n", cases, bad, missed, fcases, fbad);
    return 0;
}
