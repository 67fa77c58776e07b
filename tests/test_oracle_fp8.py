"""Pins for the FP8 (E4M3) reference of the low-precision mode (oracle/fp8.py).

The E4M3 rounding is tied to the format's bit-field definition (every code
decodes to a fixed point of the rounding; midpoints go to the even code),
to hand-worked values, and to a library conversion (torch's float8_e4m3fn
cast).  The FP8 product is tied to the plain definition on inputs that E4M3
holds exactly, to exact rational arithmetic, and to the error bound the mode
states."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import fp8
from paper_2110_13042_gb300 import inputs


def finite_codes():
    return [c for c in range(256) if (c & 0x7F) != 0x7F]


def test_decode_table_structure():
    v = fp8.e4m3_decode(np.arange(256))
    assert v[0x00] == 0.0 and v[0x01] == 2.0 ** -9 and v[0x07] == 7 * 2.0 ** -9
    assert v[0x08] == 2.0 ** -6 and v[0x38] == 1.0 and v[0x7E] == 448.0
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    pos = v[0x00:0x7F]
    assert np.all(np.diff(pos) > 0)                 # codes 0x00..0x7E increase strictly
    assert np.array_equal(v[0x80:0xFF], -pos)       # sign bit


def test_round_fixes_every_code():
    for c in finite_codes():
        x = fp8.e4m3_decode(c)
        assert fp8.e4m3_round(x) == x


def test_round_midpoints_go_to_even_code():
    v = fp8.e4m3_decode(np.arange(0x7F))
    for c in range(0x7E):
        mid = (v[c] + v[c + 1]) / 2
        even = v[c] if c % 2 == 0 else v[c + 1]
        assert fp8.e4m3_round(mid) == even, hex(c)
        assert fp8.e4m3_round(-mid) == -even
        gap = (v[c + 1] - v[c]) / 64
        assert fp8.e4m3_round(mid - gap) == v[c]
        assert fp8.e4m3_round(mid + gap) == v[c + 1]


@pytest.mark.parametrize("x,want", [
    (1.0625, 1.0),            # tie between 1.0 (even) and 1.125
    (1.1875, 1.25),           # tie between 1.125 and 1.25 (even)
    (2.0 ** -10, 0.0),        # half the smallest subnormal: tie to zero
    (1.5 * 2.0 ** -10, 2.0 ** -9),
    (3 * 2.0 ** -10, 2.0 ** -8),   # 1.5 subnormal steps: tie to 2 steps
    (250.0, 256.0),           # spacing 16 between 128 and 256
    (232.0, 224.0),           # tie between 224 = 1.75 * 2^7 (code 0x76) and 240 (0x77)
    (447.0, 448.0),
    (-0.3, -0.3125),
])
def test_round_hand_values(x, want):
    assert fp8.e4m3_round(x) == want


def test_round_matches_library_cast():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    v = fp8.e4m3_decode(np.arange(0x7F))
    mids = (v[:-1] + v[1:]) / 2
    rng = np.random.default_rng(7)
    rand = rng.uniform(-440, 440, 20000) * 2.0 ** rng.integers(-14, 0, 20000)
    x = np.concatenate([v, -v, mids, -mids, rand]).astype(np.float32).astype(np.float64)
    got = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(fp8.e4m3_round(x), got)


def test_column_exponents():
    A = np.array([[1.0, 0.75, 0.0, -3.0], [0.5, -0.25, 0.0, 2.0]])
    assert list(fp8.column_exponents(A)) == [1, 0, 0, 2]
    Q, e = fp8.fp8_quantize(A)
    assert np.all(np.abs(Q) < 256)


def test_product_exact_on_integer_inputs():
    """|a| <= 8 has at most 4 significant bits, so E4M3 holds every scaled
    entry and the FP8 product is the plain definition."""
    A = inputs.integer_valued(301, 45, seed=17)
    C8, _ = fp8.fp8_ata_lower(A)
    assert np.array_equal(C8, np.tril(oracle.ata_full(A)))


def test_product_is_exact_sum_of_quantised_products():
    A = inputs.uniform(13, 6, seed=4)
    Q, e = fp8.fp8_quantize(A)
    C8, _ = fp8.fp8_ata_lower(A)
    for j in range(6):
        for k in range(j + 1):
            s = sum((Fraction(float(Q[i, j])) * Fraction(float(Q[i, k])) for i in range(13)), Fraction(0))
            assert C8[j, k] == float(s * Fraction(2) ** int(e[j] + e[k] - 16))


@pytest.mark.parametrize("maker", ["uniform", "column_scaled_normal"])
def test_product_within_stated_bound(maker):
    A = getattr(inputs, maker)(700, 90, seed=3)
    C8, _ = fp8.fp8_ata_lower(A)
    ref = np.tril(oracle.ata_full(A))
    B = fp8.fp8_error_bound(A, accum_terms=0)   # the reference itself is exact
    assert np.all(np.abs(C8 - ref) <= B)


def test_bound_is_nearly_reached():
    """Every entry just below the tie 1.0625 * 2^7 (scaled): each rounds down
    by almost u of its value, in the same direction, so the error approaches
    (2u - u^2) D against the bound's (2u + u^2) D."""
    A = np.full((64, 3), 1.0624)
    C8, _ = fp8.fp8_ata_lower(A)
    ref = np.tril(oracle.ata_full(A))
    B = fp8.fp8_error_bound(A, accum_terms=0)
    low = np.tril_indices(3)
    r = np.abs(C8 - ref)[low] / B[low]
    assert np.all(r <= 1) and np.all(r > 0.85)


def test_wrong_rounding_is_caught():
    """A round-half-away-from-zero variant differs from the pinned midpoints."""
    v = fp8.e4m3_decode(np.arange(0x7F))
    mids = (v[:-1] + v[1:]) / 2
    away = np.where(mids > 0, v[1:], v[:-1])
    assert not np.array_equal(fp8.e4m3_round(mids), away)
