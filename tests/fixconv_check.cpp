// Checks the integer-only rounding of csrc/fixconv.h against the host's
// conversion: (double)T rounds to nearest, ties to even, and ldexp by a power
// of two is exact while the result stays normal.
// Prints "<cases> <mismatches> <missed>" and exits 0.
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
    std::printf("%ld %ld %ld\n", cases, bad, missed);
    return 0;
}
