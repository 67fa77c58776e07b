// Host planner (see plan.h).
//
// The AtA recursion of Algorithm 1 (Section 3.1) is applied to column panels
// with the full contraction height m: splitting n floor-first into n1, n2,
//   C11 = A[:, :n1]^T A[:, :n1]        (AtA on the left panel)
//   C22 = A[:, n1:]^T A[:, n1:]        (AtA on the right panel)
//   C21 = A[:, n1:]^T A[:, :n1]        (one A^T B product)
// which equals Eq. "Cij" with its two A^T A calls per diagonal block and two
// Strassen calls for C21 merged along the contraction (A11^T A11 + A21^T A21
// is the panel product A[:, :n1]^T A[:, :n1]).  Panels of at most `cutoff`
// columns are leaves (the '?syrk' base case).  Every C21 block is computed by
// `depth` levels of Strassen's algorithm in its A^T B form, splitting every
// dimension ceil-first and treating the smaller block as zero-padded
// (Sections 3.1 and 3.3), with classical tiles at the leaves.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <numeric>
#include <queue>
#include <string>

namespace ata {
namespace {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Strassen's seven products in the A^T B form C = X^T Y (X r x p, Y r x q).
// Quadrant index = 2 * (contraction half) + (column half) for X and Y, and
// 2 * (row half) + (column half) for C.
//   M1 = (X11 + X22)^T (Y11 + Y22)     M5 = (X11 + X21)^T Y22
//   M2 = (X12 + X22)^T Y11             M6 = (X12 - X11)^T (Y11 + Y12)
//   M3 = X11^T (Y12 - Y22)             M7 = (X21 - X22)^T (Y21 + Y22)
//   M4 = X22^T (Y21 - Y11)
//   C11 = M1 + M4 - M5 + M7   C12 = M3 + M5   C21 = M2 + M4
//   C22 = M1 - M2 + M3 + M6
const int kU[7][4] = {{1, 0, 0, 1}, {0, 1, 0, 1}, {1, 0, 0, 0}, {0, 0, 0, 1},
                      {1, 0, 1, 0}, {-1, 1, 0, 0}, {0, 0, 1, -1}};
const int kV[7][4] = {{1, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, -1}, {-1, 0, 1, 0},
                      {0, 0, 0, 1}, {1, 1, 0, 0}, {0, 0, 1, 1}};
const int kW[7][4] = {{1, 0, 0, 1}, {0, 0, 1, -1}, {0, 1, 0, 1}, {1, 0, 1, 0},
                      {-1, 1, 0, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}};

// Winograd's variant (7 products, 15 block additions when the sums are
// chained: Winograd 1971), written out for C = X^T Y in the same indexing.
// With S1 = X12 + X22, S2 = S1 - X11, S3 = X11 - X12, S4 = X21 - S2 and
// T1 = Y12 - Y11, T2 = Y22 - T1, T3 = Y22 - Y12, T4 = T2 - Y21:
//   M1 = X11^T Y11   M2 = X21^T Y21   M3 = S4^T Y22   M4 = X22^T T4
//   M5 = S1^T T1     M6 = S2^T T2     M7 = S3^T T3
//   C11 = M1 + M2              C12 = M1 + M6 + M5 + M3
//   C21 = M1 + M6 + M7 - M4    C22 = M1 + M6 + M7 + M5
// Here every operand is formed directly from the quadrants (the chained
// sums flattened), so an operand has up to four terms.
const int wU[7][4] = {{1, 0, 0, 0}, {0, 0, 1, 0}, {1, -1, 1, -1}, {0, 0, 0, 1},
                      {0, 1, 0, 1}, {-1, 1, 0, 1}, {1, -1, 0, 0}};
const int wV[7][4] = {{1, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}, {1, -1, -1, 1},
                      {-1, 1, 0, 0}, {1, -1, 0, 1}, {0, -1, 0, 1}};
const int wW[7][4] = {{1, 1, 1, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, -1, 0},
                      {0, 1, 0, 1}, {0, 1, 1, 1}, {0, 0, 1, 1}};

struct Region {
    int64_t off, ext;
};

// The 2^d regions of a dimension of size D after d ceil-first halvings, in
// bit order (first split = most significant bit).  A second half that is
// smaller than the first is zero-padded: its extent is clipped, possibly to
// zero.  *nominal receives the common padded size ceil^d(D).
std::vector<Region> split_regions(int64_t D, int d, int64_t *nominal) {
    std::vector<Region> cur{{0, D}};
    int64_t N = D;
    for (int l = 0; l < d; ++l) {
        int64_t Nc = (N + 1) / 2;
        std::vector<Region> nxt;
        nxt.reserve(cur.size() * 2);
        for (const Region &r : cur) {
            nxt.push_back({r.off, std::min(Nc, r.ext)});
            nxt.push_back({r.off + Nc, std::max<int64_t>(0, r.ext - Nc)});
        }
        cur.swap(nxt);
        N = Nc;
    }
    *nominal = N;
    return cur;
}

int bit(int64_t idx, int l, int d) { return static_cast<int>((idx >> (d - 1 - l)) & 1); }

int log2_ceil(int64_t x) {
    int t = 0;
    while ((int64_t(1) << t) < x) ++t;
    return t;
}

struct Builder {
    Plan &P;
    bool digits;
    bool fp8;    // one E4M3 plane per operand, FP32 accumulation
    int kalign;  // contraction rows of one leaf K step
    bool reuse_quadrants = true;
    // coefficient tables of the chosen variant (Strassen or Winograd)
    const int (*tU)[4] = kU;
    const int (*tV)[4] = kV;
    const int (*tW)[4] = kW;
    int64_t prod_elems = 0;
    int split_k = 1;  // contraction chunks per plain tile (split contraction)
    double comb_bound_max = 0;  // largest worst-case combine sum, units 2^smin
    // Tail split: plain tiles from number tail_from on (generation order) are
    // computed as tail_parts contraction chunks (see make_plan).
    int64_t n_plain = 0, tail_from = -1;
    int tail_parts = 1;
    // Per operand (index in P.ops): the group its prep may be fused with
    // (one side of one Strassen block; at depth >= 2 also one outer-level
    // product pattern), -1 for none.  See fuse_group.
    std::vector<int64_t> op_key;
    int64_t n_strassen_blocks = 0;

    int tn;  // leaf tile columns

    explicit Builder(Plan &p)
        : P(p), digits(p.p.mode != MODE_F64), fp8(p.p.mode == MODE_F32_FP8), kalign(kstep_rows(p.p.mode)),
          tn(tile_cols(p.p.mode)) {}

    int family_for(int64_t K_nominal) {
        int64_t Kp = round_up(std::max<int64_t>(K_nominal, 1), PREP_K);
        for (size_t i = 0; i < P.families.size(); ++i)
            if (P.families[i].K_pitch == Kp && !(i == 0 && digits)) return static_cast<int>(i);
        Family f{};
        f.K_pitch = Kp;
        f.cols = 0;
        P.families.push_back(f);
        return static_cast<int>(P.families.size()) - 1;
    }

    // Add an operand descriptor; returns its first column in the family.
    int64_t add_op(int fam, const std::vector<OpTerm> &terms, int64_t P_nominal, int64_t key = -1) {
        op_key.push_back(key);
        OpDesc o{};
        o.family = fam;
        int nonempty = 0;
        for (const OpTerm &t : terms)
            if (t.rows > 0 && t.cols > 0) ++nonempty;
        o.t_shift = log2_ceil(std::max(1, nonempty));
        o.first_term = static_cast<int32_t>(P.terms.size());
        for (const OpTerm &t : terms)
            if (t.rows > 0 && t.cols > 0) P.terms.push_back(t);
        o.nterms = static_cast<int32_t>(P.terms.size()) - o.first_term;
        o.K_pitch = static_cast<int32_t>(P.families[fam].K_pitch);
        o.P_pad = static_cast<int32_t>(round_up(std::max<int64_t>(P_nominal, 1), TILE));
        o.out_col = P.families[fam].cols;
        P.families[fam].cols += o.P_pad;
        P.ops.push_back(o);
        return o.out_col;
    }

    void plain_tile(int64_t r0, int64_t c0, int64_t rows, int64_t cols) {
        const bool tail = tail_from >= 0 && n_plain >= tail_from;
        ++n_plain;
        if (split_k > 1 || tail) {
            split_tile(r0, c0, rows, cols, split_k > 1 ? split_k : tail_parts);
            return;
        }
        LeafTask t{};
        t.fam_u = digits ? 0 : -1;
        t.fam_v = t.fam_u;
        t.col_u = static_cast<int32_t>(r0);
        t.col_v = static_cast<int32_t>(c0);
        t.k0 = 0;
        t.klen = static_cast<int32_t>(P.p.m);
        t.rows = static_cast<int32_t>(rows);
        t.cols = static_cast<int32_t>(cols);
        // The tile crosses the diagonal if its last column lies right of its
        // first row: then only entries with c0 + col <= r0 + row are written.
        t.diag = (c0 + cols - 1 > r0) ? 1 : 0;
        t.diag_off = static_cast<int32_t>(r0 - c0);
        if (P.p.mode == MODE_F64) {
            t.kind = OUT_C_F64;
            t.eu = t.ev = -1;  // native FP64 works on A unscaled
        } else {
            t.kind = (P.p.mode == MODE_F64_EMU) ? OUT_C_F64 : OUT_C_F32;
            t.eu = static_cast<int32_t>(r0);
            t.ev = static_cast<int32_t>(c0);
        }
        t.shift = 0;
        t.hbits = fp8 ? 0 : hbits_for(P.p.m);
        if (P.p.packed) {  // packed lower triangle: the store computes each row's offset
            t.out_off = r0;
            t.out_ld = c0;
        } else {
            t.out_off = r0 * P.p.ldc + c0;
            t.out_ld = P.p.ldc;
        }
        t.unit = P.n_units - 1;
        P.tasks.push_back(t);
        P.plain_madds += static_cast<double>(P.p.m) * TILE_M * tn;
        P.leaf_madds += static_cast<double>(P.p.m) * TILE_M * tn;
    }

    // Tiles of the diagonal panel [c0, c0 + w) that hold lower-triangle entries.
    void diag_panel(int64_t c0, int64_t w) {
        P.n_panels++;
        P.n_units++;  // one recursion unit
        for (int64_t J = 0; J < ceil_div(w, TILE_M); ++J) {
            const int64_t rows = std::min<int64_t>(TILE_M, w - J * TILE_M);
            for (int64_t K = 0; K * tn < w && K * tn <= J * TILE_M + rows - 1; ++K)
                plain_tile(c0 + J * TILE_M, c0 + K * tn, rows,
                           std::min<int64_t>(tn, w - K * tn));
        }
    }

    // Classical tiles of the off-diagonal block rows [r0, r0+p) x cols [c0, c0+q).
    void classical_block(int64_t r0, int64_t p, int64_t c0, int64_t q) {
        P.n_units++;  // one recursion unit
        for (int64_t J = 0; J < ceil_div(p, TILE_M); ++J)
            for (int64_t K = 0; K < ceil_div(q, tn); ++K)
                plain_tile(r0 + J * TILE_M, c0 + K * tn, std::min<int64_t>(TILE_M, p - J * TILE_M),
                           std::min<int64_t>(tn, q - K * tn));
    }

    int block_depth(int64_t p, int64_t q) const {
        int d = 0;
        int64_t pp = p, qq = q, mm = P.p.m;
        while (d < P.depth) {
            if (pp < P.strassen_min || qq < P.strassen_min || pp < 2 || qq < 2 || mm < 2) break;
            int64_t np = (pp + 1) / 2, nq = (qq + 1) / 2, nm = (mm + 1) / 2;
            pp = np;
            qq = nq;
            mm = nm;
            ++d;
        }
        return d;
    }

    // Where a Strassen product reads one operand.
    struct Operand {
        int fam;
        int64_t col, k0;
        int t_shift;
    };

    // A Strassen operand.  A single +1 term whose region is aligned to the
    // digit images, and whose zero padding (if any) lies beyond the end of A,
    // is read straight from the planes of A (family 0) at its row and column
    // offsets; any other operand gets its own planes in family `fam`.
    Operand operand(int fam, const std::vector<OpTerm> &tt, int64_t nominal_cols, int64_t rn, int64_t key) {
        if (digits && reuse_quadrants && tt.size() == 1 && tt[0].coef == 1) {
            const OpTerm &t = tt[0];
            const Family &f0 = P.families[0];
            const int64_t f0_cols = round_up(std::max<int64_t>(P.p.n, 1), TILE) + std::max(TILE, tn);
            // The leaf reads whole K steps: the rows from rn up to the next
            // step boundary must be zero, i.e. rn is a whole number of steps,
            // or the region ends at the end of A (family 0 is zero below m).
            const bool rows_ok = (t.rows == rn && rn % kalign == 0) ||
                                 (t.row0 + t.rows == P.p.m && t.row0 + rn <= f0.K_pitch);
            const bool cols_ok = t.cols == nominal_cols || t.col0 + t.cols == P.p.n;
            if (t.row0 % kalign == 0 && t.col0 % BLOCK_COLS == 0 && rows_ok && cols_ok &&
                t.col0 + round_up(nominal_cols, TILE) <= f0_cols) {
                P.n_reused++;
                return {0, t.col0, t.row0, 0};
            }
        }
        const size_t o = P.ops.size();
        const int64_t col = add_op(fam, tt, nominal_cols, key);
        return {fam, col, 0, P.ops[o].t_shift};
    }

    // C[r0:r0+p, c0:c0+q] = A[:, r0:r0+p]^T A[:, c0:c0+q] by d Strassen levels.
    void strassen_block(int64_t r0, int64_t p, int64_t c0, int64_t q, int d) {
        int64_t rn, pn, qn;
        std::vector<Region> kreg = split_regions(P.p.m, d, &rn);
        std::vector<Region> preg = split_regions(p, d, &pn);
        std::vector<Region> qreg = split_regions(q, d, &qn);
        const int64_t nsub = int64_t(1) << d;
        int64_t nprod = 1;
        for (int l = 0; l < d; ++l) nprod *= 7;
        int fam = family_for(rn);
        ++n_strassen_blocks;

        std::vector<int64_t> prod_off(nprod);
        std::vector<int> prod_shift(nprod);
        for (int64_t r = 0; r < nprod; ++r) {
            int digit[8];
            int64_t rr = r;
            for (int l = d - 1; l >= 0; --l) {
                digit[l] = static_cast<int>(rr % 7);
                rr /= 7;
            }
            std::vector<OpTerm> ut, vt;
            for (int64_t ia = 0; ia < nsub; ++ia) {
                for (int64_t ib = 0; ib < nsub; ++ib) {
                    int cu = 1, cv = 1;
                    for (int l = 0; l < d; ++l) {
                        int quad = 2 * bit(ia, l, d) + bit(ib, l, d);
                        cu *= tU[digit[l]][quad];
                        cv *= tV[digit[l]][quad];
                    }
                    if (cu != 0)
                        ut.push_back({kreg[ia].off, r0 + preg[ib].off,
                                      static_cast<int32_t>(kreg[ia].ext),
                                      static_cast<int32_t>(preg[ib].ext), cu, 0});
                    if (cv != 0)
                        vt.push_back({kreg[ia].off, c0 + qreg[ib].off,
                                      static_cast<int32_t>(kreg[ia].ext),
                                      static_cast<int32_t>(qreg[ib].ext), cv, 0});
                }
            }
            // fuse keys: this block, the side, the outermost product digit
            const int64_t kb = n_strassen_blocks * 64 + (d >= 2 ? digit[0] : 0) * 2;
            Operand U = operand(fam, ut, pn, rn, kb), V = operand(fam, vt, qn, rn, kb + 1);
            // Product unit: 2^(-43 - h + t_u + t_v); the combine sees it as
            // 2^(-43 + shift) with shift = t_u + t_v - h.  (FP8: the leaf
            // writes the product in units of the scaled columns, shift =
            // t_u + t_v.)
            const int hb = fp8 ? 0 : hbits_for(rn);
            int shift = U.t_shift + V.t_shift - hb;
            prod_shift[r] = shift;
            prod_off[r] = prod_elems;
            prod_elems += pn * qn;
            P.n_products++;
            const int32_t unit = P.n_units++;  // every product is one recursion unit
            for (int64_t J = 0; J < ceil_div(pn, TILE_M); ++J) {
                for (int64_t K = 0; K < ceil_div(qn, tn); ++K) {
                    LeafTask t{};
                    t.fam_u = U.fam;
                    t.fam_v = V.fam;
                    t.col_u = static_cast<int32_t>(U.col + J * TILE_M);
                    t.col_v = static_cast<int32_t>(V.col + K * tn);
                    t.k0 = static_cast<int32_t>(U.k0);
                    t.k0v = static_cast<int32_t>(V.k0);
                    t.klen = static_cast<int32_t>(rn);
                    t.rows = static_cast<int32_t>(std::min<int64_t>(TILE_M, pn - J * TILE_M));
                    t.cols = static_cast<int32_t>(std::min<int64_t>(tn, qn - K * tn));
                    t.diag = 0;
                    t.kind = digits && !fp8 ? OUT_M_I64 : OUT_M_F64;
                    t.shift = shift;
                    t.hbits = hb;
                    t.eu = t.ev = -1;
                    t.out_off = prod_off[r] + J * TILE_M * qn + K * tn;
                    t.out_ld = qn;
                    t.unit = unit;
                    P.tasks.push_back(t);
                    P.leaf_madds += static_cast<double>(rn) * TILE_M * tn;
                }
            }
        }
        P.plain_madds += static_cast<double>(P.p.m) * ceil_div(p, TILE_M) * ceil_div(q, tn) * TILE_M * tn;

        // Result sums, one per (row region, column region) of the C block.
        for (int64_t ir = 0; ir < nsub; ++ir) {
            for (int64_t ic = 0; ic < nsub; ++ic) {
                if (preg[ir].ext == 0 || qreg[ic].ext == 0) continue;
                std::vector<CombTerm> terms;
                for (int64_t r = 0; r < nprod; ++r) {
                    int64_t rr = r;
                    int w = 1;
                    for (int l = d - 1; l >= 0; --l) {
                        int dg = static_cast<int>(rr % 7);
                        rr /= 7;
                        w *= tW[dg][2 * bit(ir, l, d) + bit(ic, l, d)];
                    }
                    if (w != 0) terms.push_back({prod_off[r], static_cast<int32_t>(qn), w, prod_shift[r], 0});
                }
                add_comb(r0 + preg[ir].off, c0 + qreg[ic].off, preg[ir].ext, qreg[ic].ext, terms,
                         std::vector<int64_t>(terms.size(), rn), false);
            }
        }
    }

    // One combine region C[r0:r0+rows, c0:c0+cols] = sum of `terms` (products
    // in the workspace; term i over a contraction of klen[i] rows).  The exact
    // products are summed exactly in units 2^smin.  The result is an entry of
    // A^T A over m rows of column-scaled values below 1, so |result| <= m,
    // i.e. <= g m 2^(T_BOUND_LOG2 - smin) in those units.  g covers the
    // rounding of the operands: a product whose operands sum 2^t_u and 2^t_v
    // blocks (t = t_u + t_v = shift + h) is off by at most
    // K 2^t (2^(t_u - F) + 2^(t_v - F)) <= m 2^(2t + 1 - F) (F fraction bits
    // of the digits at the planned digit count, which an added digit only
    // makes finer), plus 1% for the leaf's rounded last accumulator.  Below
    // 2^63 the kernel sums modulo 2^64, which
    // is exact however large the terms; else in int128 (wide), whose worst
    // case (|T| <= 1.004 K 2^(T_BOUND_LOG2 + h) per product, scaled by its
    // shift) is checked against 2^125 once the plan is built.  diag: the
    // region crosses the diagonal, only entries with col <= row + (r0 - c0)
    // are written.
    void add_comb(int64_t r0, int64_t c0, int64_t rows, int64_t cols, const std::vector<CombTerm> &terms,
                  const std::vector<int64_t> &klen, bool diag) {
        CombDesc c{};
        c.c_off = r0 * P.p.ldc + c0;
        c.rows = static_cast<int32_t>(rows);
        c.cols = static_cast<int32_t>(cols);
        c.e_row0 = static_cast<int32_t>(r0);
        c.e_col0 = static_cast<int32_t>(c0);
        c.diag = diag ? 1 : 0;
        c.diag_off = static_cast<int32_t>(r0 - c0);
        c.first_term = static_cast<int32_t>(P.cterms.size());
        P.cterms.insert(P.cterms.end(), terms.begin(), terms.end());
        c.nterms = static_cast<int32_t>(terms.size());
        int smin = 1 << 20;
        for (const CombTerm &t : terms) smin = std::min(smin, t.shift);
        c.wide = 0;
        if (digits && !fp8) {
            double bound = 0;
            for (size_t i = 0; i < terms.size(); ++i)
                bound += 1.004 * static_cast<double>(klen[i]) *
                         std::ldexp(1.0, T_BOUND_LOG2 + hbits_for(klen[i]) + terms[i].shift - smin);
            const int F = DIGIT_TOP_BITS + DIGIT_BITS * (P.slices - 1);
            double g = 1.01;
            for (size_t i = 0; i < terms.size(); ++i)
                g += std::ldexp(1.0, 2 * (terms[i].shift + hbits_for(klen[i])) + 1 - F);
            const double result_bound = g * static_cast<double>(P.p.m) * std::ldexp(1.0, T_BOUND_LOG2 - smin);
            c.wide = result_bound >= std::ldexp(1.0, 63) ? 1 : 0;
            if (c.wide) comb_bound_max = std::max(comb_bound_max, bound);
        }
        c.smin = smin;
        c.tile_base = P.comb_tiles;
        P.comb_tiles += ceil_div(c.rows, COMB_ROWS) * ceil_div(c.cols, COMB_COLS);
        P.combs.push_back(c);
    }

    // A plain tile computed as `parts` contraction chunks (rows a multiple of
    // 256, so every chunk drains its accumulators on the same row boundaries
    // as the whole): each chunk's exact partial product goes to the product
    // workspace, and one combine region sums them in chunk order into C.
    void split_tile(int64_t r0, int64_t c0, int64_t rows, int64_t cols, int parts) {
        // (parts chunks of a multiple of 256 rows; the last may be shorter)
        const int64_t m = P.p.m;
        const int64_t chunk = round_up(ceil_div(m, parts), 256);
        std::vector<CombTerm> terms;
        std::vector<int64_t> klen;
        for (int64_t k0 = 0; k0 < m; k0 += chunk) {
            const int64_t kl = std::min(chunk, m - k0);
            LeafTask t{};
            t.fam_u = t.fam_v = 0;
            t.col_u = static_cast<int32_t>(r0);
            t.col_v = static_cast<int32_t>(c0);
            t.k0 = t.k0v = static_cast<int32_t>(k0);
            t.klen = static_cast<int32_t>(kl);
            t.rows = static_cast<int32_t>(rows);
            t.cols = static_cast<int32_t>(cols);
            t.diag = 0;  // the combine masks the diagonal
            t.kind = fp8 ? OUT_M_F64 : OUT_M_I64;
            t.hbits = fp8 ? 0 : hbits_for(kl);
            t.shift = fp8 ? 0 : -t.hbits;  // a product of single-term operands
            t.eu = t.ev = -1;
            t.out_off = prod_elems;
            t.out_ld = tn;
            t.unit = P.n_units - 1;
            P.tasks.push_back(t);
            terms.push_back({prod_elems, tn, 1, t.shift, 0});
            klen.push_back(kl);
            prod_elems += static_cast<int64_t>(TILE_M) * tn;
            P.leaf_madds += static_cast<double>(kl) * TILE_M * tn;
        }
        P.plain_madds += static_cast<double>(m) * TILE_M * tn;
        add_comb(r0, c0, rows, cols, terms, klen, c0 + cols - 1 > r0);
    }

    // Leaf K-steps of the lower triangle of a w-wide panel under the default
    // (middle) splits with classical off-diagonal blocks: the cost model used
    // to place a Strassen split.
    int64_t panel_steps(int64_t w) const {
        const int64_t ks = ceil_div(P.p.m, KSTEP);
        if (w <= P.cutoff || w <= 1) {
            int64_t t = 0;
            for (int64_t J = 0; J < ceil_div(w, TILE_M); ++J) {
                const int64_t rows = std::min<int64_t>(TILE_M, w - J * TILE_M);
                t += std::min<int64_t>(ceil_div(w, tn), (J * TILE_M + rows - 1) / tn + 1);
            }
            return t * ks;
        }
        const int64_t n1 = (w / (2 * SPLIT_ALIGN)) * SPLIT_ALIGN;
        if (n1 == 0) return panel_steps(P.cutoff);
        return panel_steps(n1) + panel_steps(w - n1) + ceil_div(w - n1, TILE_M) * ceil_div(n1, tn) * ks;
    }

    int64_t strassen_steps(int64_t p, int64_t q, int d) const {
        int64_t rn, pn, qn, prods = 1;
        split_regions(P.p.m, d, &rn);
        split_regions(p, d, &pn);
        split_regions(q, d, &qn);
        for (int l = 0; l < d; ++l) prods *= 7;
        return prods * ceil_div(pn, TILE_M) * ceil_div(qn, tn) * ceil_div(rn, KSTEP);
    }

    void recurse(int64_t c0, int64_t w) {
        if (w <= P.cutoff || w <= 1) {
            diag_panel(c0, w);
            return;
        }
        // Split near the middle on a SPLIT_ALIGN boundary, so every diagonal
        // panel and classical tile starts on a digit-image column block (the
        // identity C = [C11 C12; C21 C22] holds for any split point).
        int64_t n1 = (w / (2 * SPLIT_ALIGN)) * SPLIT_ALIGN, n2 = w - n1;
        if (n1 == 0) {
            diag_panel(c0, w);
            return;
        }
        // Where C21 goes to Strassen, move the split (within w/8 of the
        // middle) to the point with the fewest predicted leaf steps: product
        // blocks that are whole multiples of the 128 x 96 tile waste nothing.
        const int d0 = block_depth(n2, n1);
        if (digits && P.p.split_search && d0 > 0) {
            int64_t best = -1, best_n1 = n1;
            for (int64_t c = ((w / 2 - w / 8) / SPLIT_ALIGN) * SPLIT_ALIGN; c <= w / 2 + w / 8; c += SPLIT_ALIGN) {
                if (c < (int64_t(1) << d0) || w - c < (int64_t(1) << d0)) continue;
                const int64_t cost = panel_steps(c) + panel_steps(w - c) + strassen_steps(w - c, c, d0);
                if (best < 0 || cost < best) {
                    best = cost;
                    best_n1 = c;
                }
            }
            n1 = best_n1;
            n2 = w - n1;
        }
        recurse(c0, n1);
        recurse(c0 + n1, n2);
        P.n_blocks++;
        int d = digits && P.p.split_search ? d0 : block_depth(n2, n1);
        P.blocks.push_back({c0 + n1, n2, c0, n1, d, 0});
        if (d == 0)
            classical_block(c0 + n1, n2, c0, n1);
        else
            strassen_block(c0 + n1, n2, c0, n1, d);
    }
};

}  // namespace

// The busiest CTA's K steps when tiles of the given step counts are laid out
// longest-first on G persistent CTAs (as balance_task_list does), counting
// each tile's final drains and stores as 3 steps.
static int64_t lpt_makespan(std::vector<int64_t> steps, int G) {
    std::sort(steps.begin(), steps.end(), std::greater<int64_t>());
    std::priority_queue<int64_t, std::vector<int64_t>, std::greater<int64_t>> heap;
    for (int b = 0; b < G; ++b) heap.push(0);
    int64_t mx = 0;
    for (int64_t v : steps) {
        int64_t l = heap.top() + v + 3;
        heap.pop();
        heap.push(l);
        mx = std::max(mx, l);
    }
    return mx;
}

// Distinct source blocks of operand j, appended to `src` (by row0, col0).
// Returns false if a block appears with two different extents.
static bool add_sources(const Plan &P, size_t j, std::vector<OpTerm> *src) {
    const OpDesc &o = P.ops[j];
    for (int t = 0; t < o.nterms; ++t) {
        const OpTerm &tm = P.terms[static_cast<size_t>(o.first_term + t)];
        bool found = false;
        for (const OpTerm &sb : *src) {
            if (sb.row0 == tm.row0 && sb.col0 == tm.col0) {
                if (sb.rows != tm.rows || sb.cols != tm.cols) return false;
                found = true;
            }
        }
        if (!found) src->push_back(tm);
    }
    return true;
}

// Fuse a group of digit operands of one family and shape: split it into
// sub-groups by the planner's fuse key (the operand sums of one side of one
// Strassen block; at depth >= 2, of one outer-level product pattern), each
// drawing on at most FUSE_MAX_SRC distinct blocks of A (the four quadrants
// of a side at depth 1) with at most FUSE_MAX_OPS operands, put each
// sub-group's blocks in the plan's source list, give every term its block's
// index, and mark the operands.  *subs
// receives the sub-groups (member lists).  Returns false (nothing changed)
// when some operand has no key or some sub-group is too large, or no
// sub-group would have two operands.
static bool fuse_group(Plan &P, const std::vector<size_t> &members, const std::vector<int64_t> &key,
                       std::vector<std::vector<size_t>> *subs) {
    std::vector<std::vector<size_t>> groups;
    std::vector<std::vector<OpTerm>> srcs;
    std::vector<int64_t> gkey;
    for (size_t j : members) {
        if (key[j] < 0) return false;
        size_t gi = 0;
        while (gi < gkey.size() && gkey[gi] != key[j]) ++gi;
        if (gi == gkey.size()) {
            if (groups.size() == static_cast<size_t>(FUSE_MAX_SUBGROUPS)) return false;  // too many
            groups.emplace_back();
            srcs.emplace_back();
            gkey.push_back(key[j]);
        }
        if (!add_sources(P, j, &srcs[gi]) || srcs[gi].size() > static_cast<size_t>(FUSE_MAX_SRC) ||
            groups[gi].size() == static_cast<size_t>(FUSE_MAX_OPS))
            return false;
        groups[gi].push_back(j);
    }
    bool any_pair = false;
    for (const auto &g : groups) any_pair = any_pair || g.size() > 1;
    // (the prep kernel locates a tile's sub-group by walking the range's
    // sub-groups: a few dozen at most, as at Strassen depth <= 2)
    if (!any_pair || groups.size() > static_cast<size_t>(FUSE_MAX_SUBGROUPS)) return false;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const std::vector<OpTerm> &src = srcs[gi];
        const int32_t first = static_cast<int32_t>(P.fsrc.size());
        bool uni = true;
        for (size_t j : groups[gi]) {
            OpDesc &o = P.ops[j];
            uint32_t packed = 0;
            for (int t = 0; t < o.nterms; ++t) {
                OpTerm &tm = P.terms[static_cast<size_t>(o.first_term + t)];
                for (size_t q = 0; q < src.size(); ++q)
                    if (src[q].row0 == tm.row0 && src[q].col0 == tm.col0) tm.src = static_cast<int32_t>(q);
                packed |= (static_cast<uint32_t>(tm.coef) & 3u) << (2 * tm.src);
            }
            o.fuse_src = first;
            o.fuse_ns = static_cast<int16_t>(src.size());
            o.fuse_coef = static_cast<int32_t>(packed);
            o.fuse_isub = static_cast<int16_t>(gi);
            o.fuse_nsub = static_cast<int16_t>(groups.size());
            uni = uni && o.t_shift == P.ops[groups[gi][0]].t_shift;
        }
        for (size_t j : groups[gi]) P.ops[j].fuse_uni = uni ? 1 : 0;
        for (OpTerm sb : src) {
            sb.coef = 1;
            sb.src = 0;
            P.fsrc.push_back(sb);
        }
        P.n_fused++;
    }
    *subs = groups;
    return true;
}

// Longest-first greedy assignment of the tiles to the leaf's G persistent
// CTAs, laid out so that the kernel's round-robin walk (task i on CTA i % G)
// realises it; CTAs with fewer tiles get empty fillers (klen = 0, nothing
// stored).  Equal-length tiles run in waves of G, and a wave reads every
// operand block it touches over the whole contraction once from DRAM (a
// block's K extent does not stay in L2 from one wave to the next).  With
// `raster`, equal-length tiles that read the same operand families are
// ordered in bands of GM tile rows (column by column within a band), so a
// wave is a patch of about GM x G / GM tiles: GM minimises the patch's
// operand columns 128 GM + 96 G / GM (GM = 11 for 152 CTAs; an L2 model of
// the 8192^2 plan read 5.2 GB per launch in this order against 10.5 GB in
// generation order, whose waves span 2 tile rows and every column).
static void balance_task_list(std::vector<LeafTask> &tasks, int G, bool raster) {
    constexpr int64_t TASK_OVERHEAD_STEPS = 3;  // final drains and stores
    const size_t n = tasks.size();
    std::vector<size_t> order(n);
    std::iota(order.begin(), order.end(), size_t(0));
    const int GM = std::max(1, static_cast<int>(std::lround(std::sqrt(double(G) * TILE_N / TILE_M))));
    auto band_key = [&](const LeafTask &t) {
        return std::make_tuple(t.fam_u, t.fam_v, t.k0, t.k0v, t.col_u / (TILE_M * GM), t.col_v, t.col_u);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        if (tasks[a].klen != tasks[b].klen) return tasks[a].klen > tasks[b].klen;
        return raster && band_key(tasks[a]) < band_key(tasks[b]);
    });
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < G; ++b) heap.push({0, b});
    std::vector<std::vector<size_t>> per(G);
    for (size_t i : order) {
        Load l = heap.top();
        heap.pop();
        per[l.second].push_back(i);
        l.first += ceil_div(tasks[i].klen, KSTEP) + TASK_OVERHEAD_STEPS;
        heap.push(l);
    }
    size_t rounds = 0;
    for (const auto &v : per) rounds = std::max(rounds, v.size());
    LeafTask filler{};
    filler.kind = OUT_C_F64;
    std::vector<LeafTask> out(rounds * G, filler);
    for (int b = 0; b < G; ++b)
        for (size_t r = 0; r < per[b].size(); ++r) out[r * G + b] = tasks[per[b][r]];
    tasks.swap(out);
}

void balance_tasks(Plan &P, int G) { balance_task_list(P.tasks, G, true); }

// Static partition of the recursion over `streams` leaf launches: the
// counterpart of the paper's shared-memory AtA (Section 4.1-4.2, Algorithm 3),
// which simulates the recursion up front and gives each thread whole subtrees.
// Here the units are the recursion's leaves (a diagonal panel, a classical
// block, one Strassen product), assigned longest-first to the least-loaded
// group; every group gets a share of the CTAs proportional to its load and
// its tiles laid out for them as in balance_tasks.
void partition_units(Plan &P, int streams, int num_ctas) {
    constexpr int64_t TASK_OVERHEAD_STEPS = 3;
    const int G = std::max(1, streams);
    std::vector<double> unit_steps(static_cast<size_t>(std::max(P.n_units, 1)), 0.0);
    for (const LeafTask &t : P.tasks)
        unit_steps[static_cast<size_t>(t.unit)] += static_cast<double>(ceil_div(t.klen, KSTEP) + TASK_OVERHEAD_STEPS);
    std::vector<int> order(unit_steps.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return unit_steps[a] > unit_steps[b]; });
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int g = 0; g < G; ++g) heap.push({0.0, g});
    std::vector<int> group_of(unit_steps.size(), 0);
    std::vector<double> load(G, 0.0);
    for (int u : order) {
        Load l = heap.top();
        heap.pop();
        group_of[u] = l.second;
        l.first += unit_steps[u];
        load[l.second] = l.first;
        heap.push(l);
    }
    std::vector<std::vector<LeafTask>> per(G);
    for (const LeafTask &t : P.tasks) per[group_of[t.unit]].push_back(t);
    double total = 0;
    for (double x : load) total += x;
    const int ctas_all = std::max(num_ctas, G);
    std::vector<LeafTask> out;
    P.groups.clear();
    int given = 0;
    for (int g = 0; g < G; ++g) {
        if (per[g].empty()) continue;
        int c = total > 0 ? static_cast<int>(ctas_all * load[g] / total) : 1;
        c = std::max(1, std::min(c, ctas_all - given));
        given += c;
        if (per[g].size() > static_cast<size_t>(c)) balance_task_list(per[g], c, true);
        LeafGroup lg{};
        lg.first = static_cast<int64_t>(out.size());
        lg.count = static_cast<int64_t>(per[g].size());
        lg.ctas = c;
        lg.steps = load[g];
        out.insert(out.end(), per[g].begin(), per[g].end());
        P.groups.push_back(lg);
    }
    P.tasks.swap(out);
}

bool make_batch_plan(int mode, int slices, int num_ctas, int64_t count, const int64_t *m, const int64_t *n,
                     const int64_t *lda, const int64_t *ldc, const void *const *A, void *const *C,
                     BatchPlan *plan, std::string *err) {
    BatchPlan &B = *plan;
    B = BatchPlan();
    if (mode != MODE_F64_EMU && mode != MODE_F32 && mode != MODE_F32_BF16) {
        if (err) *err = "batched calls take F64_EMU, F32 or F32_BF16";
        return false;
    }
    B.mode = mode;
    B.slices = slices > 0 ? slices : default_slices(mode, 0);
    if (B.slices < 1 || B.slices > MAX_SLICES) {
        if (err) *err = "slices out of range";
        return false;
    }
    B.count = count;
    B.probs.resize(static_cast<size_t>(count));
    int64_t col_off = 0, plane_off = 0, prep = 0;
    for (int64_t i = 0; i < count; ++i) {
        // A and C may be absent (pointers that only the device holds): then
        // they are not checked here and the table's pointers stay null.
        if (m[i] < 0 || n[i] < 0 || m[i] > MAX_DIGIT_K || n[i] > (int64_t(1) << 30) ||
            (n[i] > 0 && (ldc[i] < n[i] || (C && !C[i]))) ||
            (n[i] > 0 && m[i] > 0 && (lda[i] < n[i] || (A && !A[i])))) {
            if (err) *err = "invalid problem " + std::to_string(i);
            return false;
        }
        BatchProb &q = B.probs[static_cast<size_t>(i)];
        q.A = A ? A[i] : nullptr;
        q.C = C ? C[i] : nullptr;
        q.m = m[i];
        q.n = n[i];
        q.lda = lda[i];
        q.ldc = ldc[i];
        q.col_off = col_off;
        q.plane_off = plane_off;
        q.prep_base = prep;
        if (n[i] == 0 || m[i] == 0) continue;
        q.K_pitch = round_up(m[i], PREP_K);
        // Only columns < n feed stored outputs: prep writes whole image
        // blocks up to n; the leaf's tile overhang reads (unwritten) memory
        // that stays inside the allocation and only reaches rows and columns
        // that are not stored.
        q.P_pad = round_up(n[i], BLOCK_COLS);
        q.tc = batch_tile_cols(q.P_pad);
        const int64_t cols = round_up(n[i], TILE) + TILE;
        q.ncb = cols / BLOCK_COLS;
        col_off += n[i];
        plane_off += q.K_pitch * cols * 2 * B.slices;
        prep += batch_prep_tiles(q.K_pitch, q.P_pad, q.tc);
        B.max_col_chunks = std::max<int64_t>(B.max_col_chunks, ceil_div(n[i], 64));
        const int kind = mode == MODE_F64_EMU ? OUT_C_F64 : OUT_C_F32;
        const int hb = hbits_for(m[i]);
        for (int64_t J = 0; J < ceil_div(n[i], TILE_M); ++J) {
            const int64_t rows = std::min<int64_t>(TILE_M, n[i] - J * TILE_M);
            for (int64_t K = 0; K * TILE_N < n[i] && K * TILE_N <= J * TILE_M + rows - 1; ++K) {
                const int64_t r0 = J * TILE_M, c0 = K * TILE_N;
                const int64_t cols_t = std::min<int64_t>(TILE_N, n[i] - c0);
                LeafTask t{};
                t.fam_u = t.fam_v = 0;
                t.col_u = static_cast<int32_t>(r0);
                t.col_v = static_cast<int32_t>(c0);
                t.klen = static_cast<int32_t>(m[i]);
                t.rows = static_cast<int32_t>(rows);
                t.cols = static_cast<int32_t>(cols_t);
                t.diag = (c0 + cols_t - 1 > r0) ? 1 : 0;
                t.diag_off = static_cast<int32_t>(r0 - c0);
                t.kind = kind;
                t.eu = static_cast<int32_t>(q.col_off + r0);
                t.ev = static_cast<int32_t>(q.col_off + c0);
                t.out_off = r0 * ldc[i] + c0;
                t.out_ld = ldc[i];
                t.hbits = hb;
                t.prob = static_cast<int32_t>(i);
                B.tasks.push_back(t);
                B.leaf_madds += static_cast<double>(m[i]) * TILE_M * TILE_N;
            }
        }
    }
    if (col_off > 0x7FFFFFFF) {
        if (err) *err = "batch has more than 2^31 columns";
        return false;
    }
    B.total_cols = col_off;
    B.plane_bytes = plane_off;
    B.prep_tiles = prep;
    B.n_tiles = static_cast<int64_t>(B.tasks.size());
    if (num_ctas > 1 && B.tasks.size() > static_cast<size_t>(num_ctas)) balance_task_list(B.tasks, num_ctas, false);
    return true;
}

int default_slices(int mode, int64_t m) {
    (void)m;
    switch (mode) {
        case MODE_F64_EMU: return 6;
        case MODE_F32: return 3;
        case MODE_F32_BF16: return 1;
        case MODE_F32_FP8: return 1;
        default: return 0;
    }
}

bool make_plan(const PlanParams &pp, Plan *plan, std::string *err) {
    Plan &P = *plan;
    P = Plan();
    P.p = pp;
    // A's leading dimension spans the operand's columns, or (transposed
    // operand) its contraction rows; a packed C has none.
    const int64_t lda_min = std::max<int64_t>(pp.trans ? pp.m : pp.n, 1);
    if (pp.m < 0 || pp.n < 0 || pp.lda < lda_min || (!pp.packed && pp.ldc < std::max<int64_t>(pp.n, 1))) {
        if (err) *err = "invalid dimensions";
        return false;
    }
    if (pp.m > (int64_t(1) << 30) || pp.n > (int64_t(1) << 30)) {
        if (err) *err = "dimension beyond the 2^30 limit";
        return false;
    }
    if (pp.mode != MODE_F64 && pp.mode != MODE_F64_EMU && pp.mode != MODE_F32 &&
        pp.mode != MODE_F32_BF16 && pp.mode != MODE_F32_FP8) {
        if (err) *err = "unknown mode";
        return false;
    }
    P.slices = pp.slices > 0 ? pp.slices : default_slices(pp.mode, pp.m);
    if (pp.mode == MODE_F64) P.slices = 0;
    if (pp.mode == MODE_F32_FP8) P.slices = 1;  // one E4M3 plane whatever the digit setting
    if (pp.mode != MODE_F64 && (P.slices < 1 || P.slices > MAX_SLICES)) {
        if (err) *err = "slices out of range";
        return false;
    }
    // Automatic depth: one Strassen level from n = 4096 in the FP64 modes.
    // A level saves 1/8 of the top block's leaf work and adds operand sums and
    // exact products that are written and summed again, in proportion to the
    // block's area, not its contraction: measured on GB300, it pays for
    // F64_EMU only with m >= 4096 (2048 x 65536: 61.2 with, 61.9 TFLOP/s
    // without), and the cheaper FP32, one-digit and FP8 leaves lost at 8192^2
    // (141 / 312 / 303 against 146 / 361 / 512 TFLOP/s), so there it is 0.
    // Native FP64 leaves are slow enough for any level to pay.
    if (pp.depth >= 0)
        P.depth = pp.depth;
    else if (pp.mode == MODE_F64)
        P.depth = pp.n >= 4096 ? 1 : 0;
    else if (pp.mode == MODE_F64_EMU)
        P.depth = pp.n >= 4096 && pp.m >= 4096 ? 1 : 0;
    else
        P.depth = 0;
    if (P.depth > MAX_STRASSEN_DEPTH) P.depth = MAX_STRASSEN_DEPTH;
    if (pp.variant != VARIANT_STRASSEN && pp.variant != VARIANT_WINOGRAD) {
        if (err) *err = "unknown Strassen variant";
        return false;
    }
    // The FP8 mode's stated bounds are Strassen's: it always uses Strassen.
    P.variant = pp.mode == MODE_F32_FP8 ? VARIANT_STRASSEN : pp.variant;
    if (P.depth == 0)
        P.cutoff = static_cast<int>(std::max<int64_t>(pp.n, 1));
    else
        P.cutoff = pp.cutoff > 0 ? pp.cutoff : static_cast<int>(std::max<int64_t>(pp.n / 4, 256));
    // A Strassen level on an N-wide block saves 1/8 of its leaf work but adds
    // ~14 operand sums of (m/2) x (N/2); on GB300 the extra HBM traffic only
    // pays for blocks of a few thousand columns (see the design notes).
    P.strassen_min = pp.strassen_min > 0 ? pp.strassen_min : 4096;
    if (pp.mode != MODE_F64 && pp.m > MAX_DIGIT_K) {
        if (err) *err = "contraction length beyond the exact-accumulation limit";
        return false;
    }

    // Build the task lists, with `split` contraction chunks per plain tile.
    std::unique_ptr<Builder> Bp;
    int tn_use = tile_cols(pp.mode);
    auto build = [&](int split, int64_t tail_from, int tail_parts) {
        P.families.clear();
        P.ops.clear();
        P.terms.clear();
        P.tasks.clear();
        P.combs.clear();
        P.cterms.clear();
        P.blocks.clear();
        P.n_panels = P.n_blocks = P.n_products = P.n_reused = 0;
        P.n_units = 0;
        P.comb_tiles = 0;
        P.leaf_madds = P.plain_madds = 0;
        Bp.reset(new Builder(P));
        Builder &B = *Bp;
        B.tn = tn_use;
        B.split_k = split;
        B.tail_from = tail_from;
        B.tail_parts = tail_parts;
        if (P.variant == VARIANT_WINOGRAD) {
            B.tU = wU;
            B.tV = wV;
            B.tW = wW;
        }
        if (B.digits) {
            // Family 0: digit planes of A itself (diagonal panels, classical tiles).
            Family f0{};
            f0.K_pitch = round_up(std::max<int64_t>(pp.m, 1), PREP_K);
            P.families.push_back(f0);
            B.add_op(0, {OpTerm{0, 0, static_cast<int32_t>(pp.m), static_cast<int32_t>(pp.n), 1, 0}},
                     pp.n);
        }
        if (pp.n > 0 && pp.m > 0) B.recurse(0, pp.n);
    };
    // The tile layout: whole tiles, then an automatic split contraction and
    // tail split (below); for the one-digit BF16 mode, redone with 96-column
    // tiles if a leaf contraction came out longer than its wide tiles' 32-bit
    // sums allow.
    const int ctas = pp.num_ctas > 1 ? pp.num_ctas : 152;
    auto layout = [&]() {
        // Split contraction (digit modes): when the plan has too few tiles to keep
        // every CTA busy and the contraction is long, or when asked for.
        int split = 1;
        const bool can_split = pp.mode != MODE_F64;
        if (can_split && pp.split_k > 1) split = std::min(pp.split_k, SPLITK_MAX);
        build(split, -1, 1);
        if (can_split && pp.split_k == 0 && static_cast<int64_t>(P.tasks.size()) < SPLITK_TILES_PER_CTA * ctas &&
            pp.m >= 2 * SPLITK_MIN_ROWS) {
            int64_t s = 2;
            while (s < SPLITK_MAX && static_cast<int64_t>(P.tasks.size()) * s < SPLITK_TILES_PER_CTA * ctas &&
                   pp.m / (2 * s) >= SPLITK_MIN_ROWS)
                s *= 2;
            // one BF16 digit on wide tiles: chunks short enough for 32-bit sums
            if (pp.mode == MODE_F32_BF16 && tn_use != TILE_N)
                while (s < SPLITK_MAX && round_up(ceil_div(pp.m, s), 256) > ONE_DIGIT_WIDE_MAX_K) s *= 2;
            build(static_cast<int>(s), -1, 1);
        }
        // Tail split: when the plain tiles (all of contraction m) leave the last
        // wave of the persistent CTAs partly idle, the last q of them (q = plain
        // tiles mod CTAs) are computed as contraction chunks, which the
        // longest-first layout spreads over the idle CTAs; chosen by simulating
        // the layout, and kept only if it shortens the busiest CTA by >= 0.5%.
        if (can_split && pp.split_k == 0 && Bp->split_k == 1 && pp.streams <= 1 && Bp->n_plain > 0) {
            const int64_t q = Bp->n_plain % ctas;
            const int64_t m_steps = ceil_div(pp.m, KSTEP);
            std::vector<int64_t> steps;
            for (const LeafTask &t : P.tasks) steps.push_back(ceil_div(t.klen, KSTEP));
            const int64_t base = lpt_makespan(steps, ctas);
            int best_parts = 1;
            int64_t best = base;
            for (int parts : {2, 3, 4, 6, 8}) {
                const int64_t chunk = round_up(ceil_div(pp.m, parts), 256);
                if (q == 0 || chunk < 1024 || chunk >= pp.m) continue;
                std::vector<int64_t> st;
                int64_t removed = 0;
                for (int64_t v : steps) {
                    if (v == m_steps && removed < q) {
                        ++removed;
                        for (int64_t k0 = 0; k0 < pp.m; k0 += chunk)
                            st.push_back(ceil_div(std::min(chunk, pp.m - k0), KSTEP));
                    } else {
                        st.push_back(v);
                    }
                }
                const int64_t ms = lpt_makespan(st, ctas);
                if (ms < best) {
                    best = ms;
                    best_parts = parts;
                }
            }
            if (best_parts > 1 && best * 200 <= base * 199) build(1, Bp->n_plain - q, best_parts);
        }
    };
    layout();
    if (pp.mode == MODE_F32_BF16 && tn_use != TILE_N) {
        int64_t kmax = 0;
        for (const LeafTask &t : P.tasks) kmax = std::max<int64_t>(kmax, t.klen);
        if (kmax > ONE_DIGIT_WIDE_MAX_K) {
            tn_use = TILE_N;
            layout();
        }
    }
    Builder &B = *Bp;
    P.split_k = B.split_k;
    P.tile_n = B.tn;
    if (B.comb_bound_max >= std::ldexp(1.0, 125)) {  // the int128 sum keeps 2 bits of margin
        if (err) *err = "internal: a combine sum could overflow 128 bits";
        return false;
    }

    P.n_tiles = static_cast<int64_t>(P.tasks.size());
    if (pp.streams > 1 && !P.tasks.empty())
        partition_units(P, pp.streams, pp.num_ctas > 1 ? pp.num_ctas : 152);
    else if (B.digits && pp.num_ctas > 1 && P.tasks.size() > static_cast<size_t>(pp.num_ctas))
        balance_tasks(P, pp.num_ctas);

    // Every digit-family tile must start on a column block: the leaf loads
    // whole 1 KB images with bulk copies.
    if (B.digits) {
        for (const LeafTask &t : P.tasks) {
            if (t.col_u % BLOCK_COLS != 0 || t.col_v % BLOCK_COLS != 0 || t.k0 % B.kalign != 0 ||
                t.k0v % B.kalign != 0) {
                if (err) *err = "internal: leaf tile not aligned to a digit-image block";
                return false;
            }
        }
    }

    // An operand summed from 2^t nonempty blocks is held with t fewer fraction
    // bits, so a product of two such operands is t_u + t_v bits coarser than a
    // plain tile.  Deep recursion (and Winograd's four-term operands) can lose
    // more than the accuracy target leaves spare: with the digit count on auto,
    // such a plan gets one more 9-bit digit (F64_EMU: 6 bits spare at 6 digits
    // for the 1e-13 target; F32: 8 bits at 3 digits for 5e-5).
    if (pp.slices == 0 && (pp.mode == MODE_F64_EMU || pp.mode == MODE_F32)) {
        int tmax = 0;
        for (const LeafTask &t : P.tasks)
            if (t.kind == OUT_M_I64) tmax = std::max(tmax, t.shift + t.hbits);
        const int spare = pp.mode == MODE_F64_EMU ? 6 : 8;
        if (tmax > spare && P.slices < MAX_SLICES) P.slices += 1;
    }

    // Workspace layout.
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        int64_t o = off;
        off += round_up(std::max<int64_t>(bytes, 0), 1024);
        return o;
    };
    P.off_colmax = take(pp.n * 8);
    P.off_expo = take(pp.n * 4);
    for (Family &f : P.families) {
        f.cols += std::max(TILE, B.tn);  // padding: a leaf box may extend a tile's width past the last operand
        f.plane_elems = f.cols * f.K_pitch;
        int64_t bytes = B.fp8 ? f.plane_elems : B.digits ? f.plane_elems * 2 * P.slices : f.plane_elems * 8;
        f.offset = take(bytes);
    }
    P.product_bytes = B.prod_elems * 8;
    P.off_products = take(P.product_bytes);
    // Prep tiles: operands of one family and shape are grouped (in order of
    // first appearance) and share an interleaved tile range (OpDesc::ilv_n).
    // Fused groups (fuse_group) take the first tiles, [0, fused_tiles): the
    // prep launches one kernel for them and one for the rest.
    {
        std::vector<std::vector<size_t>> groups;
        std::vector<bool> taken(P.ops.size(), false);
        for (size_t i = 0; i < P.ops.size(); ++i) {
            if (taken[i]) continue;
            const OpDesc &key = P.ops[i];
            std::vector<size_t> members;
            for (size_t j = i; j < P.ops.size(); ++j)
                if (!taken[j] && P.ops[j].family == key.family && P.ops[j].K_pitch == key.K_pitch &&
                    P.ops[j].P_pad == key.P_pad) {
                    members.push_back(j);
                    taken[j] = true;
                }
            groups.push_back(members);
        }
        P.prep_tiles = 0;
        P.fused_tiles = 0;
        P.fsrc.clear();
        P.n_fused = 0;
        std::vector<bool> fused(groups.size(), false);
        std::vector<std::vector<std::vector<size_t>>> subs(groups.size());
        for (size_t g = 0; g < groups.size(); ++g)
            fused[g] = B.digits && !B.fp8 && fuse_group(P, groups[g], B.op_key, &subs[g]);
        // The planes of A from the same reads: when fused sub-groups whose
        // source blocks tile A exactly (the top block's two sides, at depth 1),
        // every block starting on a K step, write family 0 too, and drop its
        // own operand (one pass over A instead of two).
        bool skip_f0 = false;
        if (B.digits && !B.fp8 && pp.m > 0 && pp.n > 0) {
            std::vector<std::pair<size_t, size_t>> chosen;  // (group, sub-group)
            std::vector<OpTerm> cover;
            int64_t area = 0;
            for (size_t g = groups.size(); g-- > 0 && area < pp.m * pp.n;) {
                if (!fused[g]) continue;
                for (size_t k = subs[g].size(); k-- > 0 && area < pp.m * pp.n;) {
                    const OpDesc &o = P.ops[subs[g][k][0]];
                    bool ok = true;
                    int64_t a = 0;
                    for (int q = 0; q < o.fuse_ns && ok; ++q) {
                        const OpTerm &sb = P.fsrc[static_cast<size_t>(o.fuse_src + q)];
                        ok = sb.row0 % KSTEP == 0 && sb.row0 + sb.rows <= pp.m && sb.col0 + sb.cols <= pp.n;
                        for (const OpTerm &c : cover)
                            ok = ok && (sb.row0 + sb.rows <= c.row0 || c.row0 + c.rows <= sb.row0 ||
                                        sb.col0 + sb.cols <= c.col0 || c.col0 + c.cols <= sb.col0);
                        a += static_cast<int64_t>(sb.rows) * sb.cols;
                    }
                    if (!ok) continue;
                    for (int q = 0; q < o.fuse_ns; ++q) cover.push_back(P.fsrc[static_cast<size_t>(o.fuse_src + q)]);
                    area += a;
                    chosen.push_back({g, k});
                }
            }
            if (area == pp.m * pp.n) {
                for (const auto &gk : chosen)
                    for (size_t j : subs[gk.first][gk.second]) P.ops[j].fuse_f0 = 1;
                skip_f0 = true;
                P.f0_zero = true;
            }
        }
        std::vector<OpDesc> grouped;
        grouped.reserve(P.ops.size());
        for (int pass = 0; pass < 2; ++pass) {
            for (size_t g = 0; g < groups.size(); ++g) {
                if (fused[g] != (pass == 0)) continue;
                const OpDesc &key = P.ops[groups[g][0]];
                if (skip_f0 && key.family == 0) continue;  // written by the fused groups
                if (fused[g]) {  // sub-groups back to back, sharing one interleaved tile range
                    for (const std::vector<size_t> &members : subs[g])
                        for (size_t k = 0; k < members.size(); ++k) {
                            OpDesc o = P.ops[members[k]];
                            o.tile_base = P.prep_tiles;
                            o.ilv_n = static_cast<int32_t>(members.size());
                            o.ilv_i = static_cast<int32_t>(k);
                            grouped.push_back(o);
                        }
                    P.prep_tiles += fused_tiles_for(key.K_pitch, key.P_pad) *
                                    static_cast<int64_t>(subs[g].size());
                    continue;
                }
                const std::vector<size_t> &members = groups[g];
                const int64_t per = prep_tiles_for(B.digits, key.K_pitch, key.P_pad, B.fp8);
                for (size_t k = 0; k < members.size(); ++k) {
                    OpDesc o = P.ops[members[k]];
                    o.tile_base = P.prep_tiles;
                    o.ilv_n = static_cast<int32_t>(members.size());
                    o.ilv_i = static_cast<int32_t>(k);
                    grouped.push_back(o);
                }
                P.prep_tiles += per * static_cast<int64_t>(members.size());
            }
            if (pass == 0) P.fused_tiles = P.prep_tiles;
        }
        P.ops.swap(grouped);
    }
    P.t_ops = 0;
    P.t_terms = round_up(P.t_ops + static_cast<int64_t>(P.ops.size() * sizeof(OpDesc)), 256);
    P.t_tasks = round_up(P.t_terms + static_cast<int64_t>(P.terms.size() * sizeof(OpTerm)), 256);
    P.t_combs = round_up(P.t_tasks + static_cast<int64_t>(P.tasks.size() * sizeof(LeafTask)), 256);
    P.t_cterms = round_up(P.t_combs + static_cast<int64_t>(P.combs.size() * sizeof(CombDesc)), 256);
    P.t_fsrc = round_up(P.t_cterms + static_cast<int64_t>(P.cterms.size() * sizeof(CombTerm)), 256);
    P.table_bytes = round_up(P.t_fsrc + static_cast<int64_t>(P.fsrc.size() * sizeof(OpTerm)), 256);
    P.off_tables = take(P.table_bytes);
    P.workspace_bytes = off;
    return true;
}

void pack_tables(const Plan &P, std::vector<uint8_t> *buf) {
    buf->assign(static_cast<size_t>(P.table_bytes), 0);
    auto put = [&](int64_t at, const void *src, size_t bytes) {
        if (bytes) std::memcpy(buf->data() + at, src, bytes);
    };
    put(P.t_ops, P.ops.data(), P.ops.size() * sizeof(OpDesc));
    put(P.t_terms, P.terms.data(), P.terms.size() * sizeof(OpTerm));
    put(P.t_tasks, P.tasks.data(), P.tasks.size() * sizeof(LeafTask));
    put(P.t_combs, P.combs.data(), P.combs.size() * sizeof(CombDesc));
    put(P.t_cterms, P.cterms.data(), P.cterms.size() * sizeof(CombTerm));
    put(P.t_fsrc, P.fsrc.data(), P.fsrc.size() * sizeof(OpTerm));
}

}  // namespace ata
