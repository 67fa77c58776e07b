"""FP8 (E4M3) reference for the low-precision FP8 mode -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module; the product library never does.  Plain
numpy in FP64, written from the E4M3 format definition (OCP 8-bit floating
point specification: 1 sign bit, 4 exponent bits with bias 7, 3 fraction
bits; subnormals 2^-6 * f/8; largest finite value 448 = 1.75 * 2^8; no
infinities) and from the FP8 mode's arithmetic:

* every column j of A is scaled by 2^(8 - e_j), where 2^e_j is the smallest
  power of two above max_i |a_ij| (the column equilibration of the method's
  other modes), so every scaled entry lies in (-2^8, 2^8);
* each scaled entry is rounded to the nearest E4M3 value, ties to even;
* C_jk = 2^(e_j + e_k - 16) * sum_i q_ij q_ik.

The products q_ij q_ik have at most 8 significant bits and lie between
2^-18 and 2^16, so every partial sum of fewer than 2^19 of them is an exact
FP64 number: ``fp8_ata_lower`` is the EXACT product of the quantised columns,
whatever order the sum takes.  The GPU mode differs from it only by its FP32
accumulation.

Functions:

* ``e4m3_round(x)``        nearest E4M3 value of each element (ties to even).
* ``e4m3_decode(code)``    value of an 8-bit E4M3 code (NaN for 0x7F, 0xFF).
* ``column_exponents(A)``  e_j with 2^(e_j - 1) <= max_i |a_ij| < 2^e_j (0 for a zero column).
* ``fp8_quantize(A)``      (Q, e): Q = E4M3(A * 2^(8 - e)) column by column.
* ``fp8_ata_lower(A)``     low C of the FP8 mode, exact (see above); also
                           returns D8 = low(|Q|^T|Q|) scaled the same way.
* ``fp8_error_bound(A)``   componentwise bound on |C_fp8 - C_exact| at
                           Strassen depth 0 (derivation in the docstring).
"""
from __future__ import annotations

import numpy as np

__all__ = ["E4M3_MAX", "U8", "e4m3_round", "e4m3_decode", "column_exponents", "fp8_quantize",
           "fp8_ata_lower", "fp8_error_bound", "fp8_strassen_bound"]

E4M3_MAX = 448.0
U8 = 2.0 ** -4          # unit roundoff of a 4-significant-bit format
SUB_Q = 2.0 ** -9       # subnormal spacing (2^-6 * 1/8)
MIN_NORMAL = 2.0 ** -6


def e4m3_round(x):
    """Round to the nearest E4M3 value, ties to even, saturating at +-448.

    For |x| >= 2^-6 the spacing at x is 2^(E - 3) with 2^E <= |x| < 2^(E+1);
    below 2^-6 it is the subnormal spacing 2^-9.  Division by the spacing is
    exact (a power of two), and np.rint rounds half to even."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)                       # a = f 2^ex, f in [0.5, 1)
    E = ex - 1                                # 2^E <= a < 2^(E+1)
    spacing = np.where(a >= MIN_NORMAL, np.ldexp(1.0, E - 3), SUB_Q)
    r = np.rint(a / spacing) * spacing
    r = np.minimum(r, E4M3_MAX)
    return np.where(a == 0, 0.0, np.copysign(r, x))


def e4m3_decode(code):
    """Value of E4M3 code(s) 0..255 from the bit fields."""
    c = np.asarray(code, np.int64)
    s = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    f = (c & 0x7).astype(np.float64)
    val = np.where(e == 0, np.ldexp(f / 8.0, -6), np.ldexp(1.0 + f / 8.0, e - 7))
    val = np.where((c & 0x7F) == 0x7F, np.nan, val)
    return s * val


def column_exponents(A):
    A = np.asarray(A, np.float64)
    mx = np.max(np.abs(A), axis=0) if A.shape[0] else np.zeros(A.shape[1])
    _, e = np.frexp(mx)                       # mx = f 2^e, f in [0.5, 1) -> 2^(e-1) <= mx < 2^e
    return np.where(mx > 0, e, 0).astype(np.int64)


def fp8_quantize(A):
    A = np.asarray(A, np.float64)
    e = column_exponents(A)
    return e4m3_round(A * np.ldexp(1.0, 8 - e)[None, :]), e


def fp8_ata_lower(A):
    """(C8, D8): low(C) of the FP8 mode and low(|Q|^T|Q|), both scaled by
    2^(e_j + e_k - 16).  Exact for m < 2^19 (see the module docstring)."""
    Q, e = fp8_quantize(A)
    m = Q.shape[0]
    assert m < 2 ** 19
    sc = np.ldexp(1.0, e - 8)
    C = (Q.T @ Q) * sc[:, None] * sc[None, :]
    D = (np.abs(Q).T @ np.abs(Q)) * sc[:, None] * sc[None, :]
    return np.tril(C), np.tril(D)


def fp8_error_bound(A, accum_terms=None):
    """Componentwise bound on |C_fp8 - A^T A| at Strassen depth 0.

    Per entry, in the scaled units x = a 2^(8 - e): |E4M3(x) - x| <= u |x|
    (normal range, u = 2^-4) or <= 2^-10 (subnormal range), so in A's units
    d_ij = |q_ij 2^(e_j - 8) - a_ij| <= u |a_ij| + 2^(e_j - 18).  Then
      |sum_i (q q' - a a')| <= sum_i (|a_ij| d_ik + |a_ik| d_ij + d_ij d_ik)
        <= (2u + u^2) D_jk + (1 + u)(2^(e_k - 18) S_j + 2^(e_j - 18) S_k)
           + m 2^(e_j + e_k - 36),
    S_j = sum_i |a_ij|, D = |A|^T|A|.  FP32 accumulation of the exact
    products adds at most ``accum_terms`` * 2^-24 * |Q|^T|Q| (default:
    512 additions in the tensor core, m / 512 in the epilogue, one final
    rounding), bounded with |Q|^T|Q| <= (1 + u)^2 D + the subnormal terms."""
    A = np.asarray(A, np.float64)
    m = A.shape[0]
    e = column_exponents(A)
    Aa = np.abs(A)
    D = Aa.T @ Aa
    S = np.sum(Aa, axis=0)
    s = np.ldexp(1.0, e - 18)
    u = U8
    rnd = (2 * u + u * u) * D + (1 + u) * (s[None, :] * S[:, None] + s[:, None] * S[None, :]) + \
        m * s[:, None] * s[None, :]
    if accum_terms is None:
        accum_terms = 512 + m / 512.0 + 2
    QQ = (1 + u) ** 2 * D + rnd
    return np.tril(rnd + accum_terms * 2.0 ** -24 * QQ)


def fp8_strassen_bound(A, depth):
    """Normwise bound on max |C_fp8 - A^T A| / 2^(e_j + e_k) with Strassen on
    the off-diagonal blocks to the given depth (any split points).

    In the scaled matrix Ahat = A diag(2^-e) every output entry is a sum of
    products M_r = U_r^T V_r whose operands are exact sums of blocks of Ahat,
    each rounded once to E4M3 in units 2^-t (t <= depth) of the sum; the pairs
    (block of U_r, block of V_r) over all products that reach one output
    block number 12 per level (M1 + M4 - M5 + M7 and M1 - M2 + M3 + M6: 4 + 2
    + 2 + 4 pairs), so at most 12^depth.  Each pair contributes at most
    (2u + u^2) max_p Dhat_pp (Cauchy-Schwarz on |X|^T|Y|) plus the subnormal
    terms 2 (1 + u) 2^(t - 18) max_p Shat_p + m 2^(2t - 36), and the FP32
    accumulation as in fp8_error_bound.  Returns that scalar bound."""
    A = np.asarray(A, np.float64)
    m = A.shape[0]
    e = column_exponents(A)
    Ah = np.abs(A) * np.ldexp(1.0, -e)[None, :]
    dmax = float(np.max(np.sum(Ah * Ah, axis=0))) if A.size else 0.0
    smax = float(np.max(np.sum(Ah, axis=0))) if A.size else 0.0
    u, t = U8, depth
    pairs = 12.0 ** depth
    per_pair = (2 * u + u * u) * dmax + 2 * (1 + u) * 2.0 ** (t - 18) * smax + m * 2.0 ** (2 * t - 36)
    accum = (512 + m / 512.0 + 2 + 8 * (depth + 1)) * 2.0 ** -24 * ((1 + u) ** 2 * dmax + per_pair)
    return pairs * (per_pair + accum)
