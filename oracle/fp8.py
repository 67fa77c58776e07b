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
* ``fp8_strassen_atb(X, Y, depth)``  the FP8 mode's Strassen product X^T Y of two
                           equilibrated panels: ``depth`` levels of Strassen's
                           algorithm (Section 3.1, Section 3.3 splits), every
                           leaf operand an exact sum of blocks rounded once to
                           E4M3; returns the product and the matching |Q|^T|Q|
                           magnitude sum (for the FP32-accumulation tolerance).
* ``fp8_ata_lower_blocks(A, blocks)``  low C of the FP8 mode for a given AtA
                           block layout: depth-0 entries everywhere, Strassen
                           on each listed off-diagonal block.
* ``fp8_strassen_bound(A, depth)``  scalar normwise bound at Strassen depth > 0.

With Strassen the operands are signed sums of blocks of the equilibrated
matrix Ahat = A diag(2^-e).  An operand of t' nonempty terms is scaled by
2^(8 - t), t = ceil(log2 t'), so it stays below 2^8 in magnitude; each term is
first rounded to FP8_FIX = 47 fraction bits of that scale (half away from
zero; exact for every FP32 entry at or above 2^-21 of its column scale), the
terms are summed exactly, and the sum is rounded once to E4M3.  Leaf products
Q_u^T Q_v are exact in FP64 as above; the Strassen result sums are FP64 sums.
"""
from __future__ import annotations

import numpy as np

__all__ = ["E4M3_MAX", "U8", "e4m3_round", "e4m3_decode", "column_exponents", "fp8_quantize",
           "fp8_ata_lower", "fp8_error_bound", "fp8_strassen_atb", "fp8_ata_lower_blocks",
           "fp8_strassen_bound"]

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


def _row_regions(m, depth):
    """The contraction-row regions after ``depth`` ceil-first halvings
    (Section 3.3 rounds up; a second half past the end is zero padding)."""
    regs, N = [(0, m)], m
    for _ in range(depth):
        Nc = (N + 1) // 2
        regs = [x for off, ext in regs for x in ((off, min(Nc, ext)), (off + Nc, max(0, ext - Nc)))]
        N = Nc
    return regs, N


def fp8_strassen_bound(A, depth):
    """Normwise bound on max |C_fp8 - A^T A| / 2^(e_j + e_k) with Strassen on
    the off-diagonal blocks to the given depth (any column split points; the
    contraction rows split ceil-first).

    In the scaled matrix Ahat = A diag(2^-e) every output entry is a sum of
    products M_r = U_r^T V_r whose operands are exact sums of blocks of Ahat,
    each rounded once to E4M3 in units 2^-t (t <= depth) of the sum, so
    |Qhat_r - U_r| <= u |U_r| + 2^(t - 18) elementwise and
      |Qu^T Qv - U^T V| <= (2u + u^2) |U|^T |V| + (1 + u) 2^(t - 18) (|U|^T 1 + 1^T |V|)
                           + R 2^(2t - 36)
    over the R = ceil^depth(m) rows of one leaf.  |U|^T|V| is at most the sum
    over the (block of U_r, block of V_r) pairs, and the pairs over all
    products that reach one output block number 12 per level (M1 + M4 - M5 + M7
    and M1 - M2 + M3 + M6: 4 + 2 + 2 + 4), so at most 12^depth.  Every block
    of a pair lies in one contraction-row region of the depth's row split, so
    by Cauchy-Schwarz a pair is at most dmax = the largest sum over one region
    of Ahat_ij^2 for one column (and a row sum of |U| at most smax, the
    largest such sum of |Ahat_ij|).  The FP32 accumulation adds
    (512 + R / 512 + 2 + 8 (depth + 1)) 2^-24 of the rounded magnitudes.
    Returns that scalar bound."""
    A = np.asarray(A, np.float64)
    m = A.shape[0]
    if A.size == 0:
        return 0.0
    e = column_exponents(A)
    Ah = np.abs(A) * np.ldexp(1.0, -e)[None, :]
    regs, R = _row_regions(m, depth)
    dmax = max(float(np.max(np.sum(Ah[o:o + x] ** 2, axis=0))) for o, x in regs if x > 0)
    smax = max(float(np.max(np.sum(Ah[o:o + x], axis=0))) for o, x in regs if x > 0)
    u, t = U8, depth
    pairs = 12.0 ** depth
    per_pair = (2 * u + u * u) * dmax + 2 * (1 + u) * 2.0 ** (t - 18) * smax + R * 2.0 ** (2 * t - 36)
    accum = (512 + R / 512.0 + 2 + 8 * (depth + 1)) * 2.0 ** -24 * ((1 + u) ** 2 * dmax + per_pair)
    return pairs * (per_pair + accum)


# ------------------------------------------------------------ Strassen --
FP8_FIX = 47      # fraction bits of an operand sum before its E4M3 rounding

# Strassen's algorithm (Strassen 1969, the form the paper uses in Section 3.1)
# written for C = X^T Y.  X_ab is the block of contraction half a and column
# half b (0 = first); products M1..M7 and result sums
#   M1 = (X11 + X22)^T (Y11 + Y22)     M5 = (X11 + X21)^T Y22
#   M2 = (X12 + X22)^T Y11             M6 = (X12 - X11)^T (Y11 + Y12)
#   M3 = X11^T (Y12 - Y22)             M7 = (X21 - X22)^T (Y21 + Y22)
#   M4 = X22^T (Y21 - Y11)
#   C11 = M1 + M4 - M5 + M7   C12 = M3 + M5   C21 = M2 + M4   C22 = M1 - M2 + M3 + M6
# Each operand is a tuple of (coef, a, b); each result a tuple of (coef, product).
_M = (
    (((1, 0, 0), (1, 1, 1)), ((1, 0, 0), (1, 1, 1))),
    (((1, 0, 1), (1, 1, 1)), ((1, 0, 0),)),
    (((1, 0, 0),), ((1, 0, 1), (-1, 1, 1))),
    (((1, 1, 1),), ((1, 1, 0), (-1, 0, 0))),
    (((1, 0, 0), (1, 1, 0)), ((1, 1, 1),)),
    (((1, 0, 1), (-1, 0, 0)), ((1, 0, 0), (1, 0, 1))),
    (((1, 1, 0), (-1, 1, 1)), ((1, 1, 0), (1, 1, 1))),
)
_C = {(0, 0): ((1, 0), (1, 3), (-1, 4), (1, 6)),
      (0, 1): ((1, 2), (1, 4)),
      (1, 0): ((1, 1), (1, 3)),
      (1, 1): ((1, 0), (-1, 1), (1, 2), (1, 5))}


def _block(terms, R, P, a, b):
    """Terms of block (a, b) of an operand of nominal size R x P given as terms
    (coef, row0, col0, rows, cols) of a panel.  Halving is ceil-first; a second
    half that runs past a term's extent is zero padding (clipped, possibly to
    nothing), as Section 3.1 handles odd sizes."""
    R1, P1 = (R + 1) // 2, (P + 1) // 2
    out = []
    for coef, r0, c0, rows, cols in terms:
        rr0, rr = (r0, min(R1, rows)) if a == 0 else (r0 + R1, max(0, rows - R1))
        cc0, cc = (c0, min(P1, cols)) if b == 0 else (c0 + P1, max(0, cols - P1))
        if rr > 0 and cc > 0:
            out.append((coef, rr0, cc0, rr, cc))
    return out


def _operand(terms, R, P, combo):
    """Terms of a signed sum of blocks, e.g. X11 + X22."""
    out = []
    for coef, a, b in combo:
        out += [(coef * c, r0, c0, rr, cc) for c, r0, c0, rr, cc in _block(terms, R, P, a, b)]
    return out


def _round_half_away(x):
    return np.copysign(np.floor(np.abs(x) + 0.5), x)


def _e4m3_operand(panel, terms, R, P):
    """(Q, t): the operand sum of `terms` scaled by 2^(8 - t) and rounded to
    E4M3 (see the module docstring)."""
    t = int(np.ceil(np.log2(len(terms)))) if len(terms) > 1 else 0
    V = np.zeros((R, P), np.float64)          # integer values, |V| < 2^47: exact
    for coef, r0, c0, rr, cc in terms:
        V[:rr, :cc] += coef * _round_half_away(panel[r0:r0 + rr, c0:c0 + cc] * 2.0 ** (FP8_FIX - t))
    return e4m3_round(V * 2.0 ** (8 - FP8_FIX)), t


def _strassen(X, Y, xt, yt, R, P, Q, depth):
    if depth == 0:
        Qu, tu = _e4m3_operand(X, xt, R, P)
        Qv, tv = _e4m3_operand(Y, yt, R, Q)
        sc = 2.0 ** (tu + tv - 16)
        return (Qu.T @ Qv) * sc, (np.abs(Qu).T @ np.abs(Qv)) * sc
    R1, P1, Q1 = (R + 1) // 2, (P + 1) // 2, (Q + 1) // 2
    prods = [_strassen(X, Y, _operand(xt, R, P, ux), _operand(yt, R, Q, vy), R1, P1, Q1, depth - 1)
             for ux, vy in _M]
    M = np.zeros((P, Q))
    D = np.zeros((P, Q))
    for (a, b), combo in _C.items():
        rows = slice(0, P1) if a == 0 else slice(P1, P)
        cols = slice(0, Q1) if b == 0 else slice(Q1, Q)
        pr, pc = rows.stop - rows.start, cols.stop - cols.start
        acc = np.zeros((P1, Q1))
        dacc = np.zeros((P1, Q1))
        for coef, r in combo:
            acc += coef * prods[r][0]
            dacc += prods[r][1]
        M[rows, cols] = acc[:pr, :pc]
        D[rows, cols] = dacc[:pr, :pc]
    return M, D


def fp8_strassen_atb(Xh, Yh, depth):
    """FP8-mode Strassen product of two equilibrated panels (Xh r x p, Yh r x q,
    columns already scaled by 2^-e): (M, D) with M ~ Xh^T Yh computed by
    ``depth`` levels of Strassen with E4M3 leaf operands, and
    D = sum over the products reaching each entry of |Q_u|^T |Q_v| (scaled
    like M), the magnitude the FP32 accumulation error is relative to."""
    Xh = np.asarray(Xh, np.float64)
    Yh = np.asarray(Yh, np.float64)
    r, p = Xh.shape
    r2, q = Yh.shape
    assert r == r2 and r < 2 ** 19
    return _strassen(Xh, Yh, [(1, 0, 0, r, p)] if r and p else [],
                     [(1, 0, 0, r, q)] if r and q else [], r, p, q, depth)


def fp8_ata_lower_blocks(A, blocks):
    """(C8, D8) of the FP8 mode for an AtA block layout.  ``blocks`` lists the
    off-diagonal blocks (r0, p, c0, q, depth): C[r0:r0+p, c0:c0+q] =
    A[:, r0:r0+p]^T A[:, c0:c0+q] by ``depth`` Strassen levels; every other
    entry (diagonal panels, depth-0 blocks) is the plain FP8 product."""
    A = np.asarray(A, np.float64)
    C, D = fp8_ata_lower(A)
    e = column_exponents(A)
    Ah = A * np.ldexp(1.0, -e)[None, :]
    for r0, p, c0, q, d in blocks:
        if d == 0:
            continue
        M, Dm = fp8_strassen_atb(Ah[:, r0:r0 + p], Ah[:, c0:c0 + q], d)
        sc = np.ldexp(1.0, e[r0:r0 + p])[:, None] * np.ldexp(1.0, e[c0:c0 + q])[None, :]
        C[r0:r0 + p, c0:c0 + q] = M * sc
        D[r0:r0 + p, c0:c0 + q] = Dm * sc
    return C, D
