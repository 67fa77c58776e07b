// Host planner: flattens the AtA recursion (Algorithm 1) and the Strassen
// trees of its off-diagonal blocks into flat, phase-ordered task lists that
// the device kernels execute.  Host-only C++ (no CUDA), shared with the
// kernels through the plain structs below.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ata {

constexpr int TILE = 128;        // column padding unit of operand families
constexpr int TILE_M = 128;      // leaf output tile rows (U-operand columns)
constexpr int TILE_N = 96;       // leaf output tile columns (V-operand columns)
// The one-digit modes' tiles (FP8, and BF16 when every contraction is short
// enough) are twice as wide (one accumulator, whose two TMEM buffers take
// 2 x 192 of the 512 columns): their leaf is bound by operand delivery, and a
// 128 x 192 tile moves 10 KB instead of 2 x 7 KB per K step of the same work.
constexpr int TILE_N8 = 2 * TILE_N;
inline int tile_cols(int mode);
constexpr int KSTEP = 16;        // contraction rows per pipeline stage (one MMA K step)
constexpr int CHUNK_STEPS = 4;   // stages per exact-accumulation chunk (64 rows)
// The leaf's exact int64 sum T is in units of 2^-T_FRAC of the leading digit
// product; |T| <= 1.004 * K * 2^T_BOUND_LOG2 for a contraction of K rows.
constexpr int T_FRAC = 27;
constexpr int T_BOUND_LOG2 = 43;
constexpr int DIGIT_TOP_BITS = 8;   // first digit: |x_1| <= 2^8
constexpr int DIGIT_BITS = 9;       // every further digit carries 9 bits
constexpr int64_t MAX_DIGIT_K = int64_t(1) << 19;  // keeps |T| < 2^63
constexpr int BLOCK_COLS = 32;   // digit-plane image: 32 columns x KSTEP rows = 1 KB
constexpr int BLOCK_BYTES = BLOCK_COLS * KSTEP * 2;
constexpr int SPLIT_ALIGN = 32;  // AtA column splits are multiples of this
constexpr int PREP_K = 64;       // contraction pitch unit; native-FP64 prep tile rows
constexpr int PREP_C = 64;       // native-FP64 prep tile columns
// Digit-plane prep tile: 16 contraction rows (one K step) x 256 columns, so
// a tile reads 2 KB row segments of A and writes 8 KB image runs per digit.
constexpr int PREP_TK = KSTEP;
constexpr int PREP_TC = 256;
constexpr int MAX_FAMILIES = 6;  // operand families (tensor maps) per launch
constexpr int MAX_SLICES = 7;
// Strassen levels per off-diagonal block: a budget; a level splits a block
// only while both its sides are >= strassen_min, so a large budget recurses
// to that size cutoff (the paper's FastStrassen recursion to its base case).
constexpr int MAX_STRASSEN_DEPTH = 8;
enum Variant : int { VARIANT_STRASSEN = 0, VARIANT_WINOGRAD = 1 };

enum Mode : int { MODE_F64 = 0, MODE_F64_EMU = 1, MODE_F32 = 2, MODE_F32_BF16 = 4, MODE_F32_FP8 = 5 };

// FP8 mode: one E4M3 plane per operand.  A column scaled by 2^(FP8_TOP - e)
// has |value| < 2^FP8_TOP <= 448 (E4M3's largest finite value), so no value
// saturates.  An operand sum is first formed exactly in fixed point with
// FP8_FIX fraction bits (every FP32 entry at or above 2^-18 of its column
// scale, i.e. every entry that does not round to zero, is exact there),
// then rounded once to E4M3.  One K step of an FP8 plane is 32 contraction
// rows (the 32-byte image row holds 32 one-byte values).
constexpr int FP8_TOP = 8;
constexpr int FP8_FIX = 47;
constexpr int KSTEP8 = 32;
// FP8 prep tiles: 32 contraction rows (one FP8 K step) x 128 columns.
constexpr int PREP8_TK = KSTEP8;
constexpr int PREP8_TC = 128;
inline int tile_cols(int mode) { return mode == MODE_F32_FP8 || mode == MODE_F32_BF16 ? TILE_N8 : TILE_N; }
// The one-digit BF16 mode's wide tiles keep their exact sums in 32 bits: each
// 256-row chunk adds at most 2^24 (in units of the digit product), so a
// contraction of up to 16384 rows stays below 2^30.  A plan with a longer
// leaf contraction uses the 96-column tiles and 64-bit sums.
constexpr int64_t ONE_DIGIT_WIDE_MAX_K = 16384;
inline int kstep_rows(int mode) { return mode == MODE_F32_FP8 ? KSTEP8 : KSTEP; }

// One term of a (possibly summed) Strassen operand: a sub-block of A.
struct OpTerm {
    int64_t row0;   // first contraction row in A
    int64_t col0;   // first column in A
    int32_t rows;   // valid rows (contraction extent); rows beyond are zero
    int32_t cols;   // valid columns; columns beyond are zero
    int32_t coef;   // +1 or -1
    int32_t src;    // fused groups: index of the term's block in the group's
                    // source list (OpDesc::fuse_src); 0 otherwise
};

// Operand generator: writes
//   U[k][c] = sum_t coef_t * A[row0_t + k][col0_t + c] * 2^-e(col0_t + c)
// for k < K_pitch, c < P_pad (zero outside every term's extent) into the
// family: either `slices` BF16 digit planes, stored as 1 KB images of
// 32 columns x 16 contraction rows in exactly the order the leaf kernel's
// shared memory needs them (K-major rows of 32 bytes, 32-byte swizzle;
// image (kstep, digit, colblock) at ((kstep * S + digit) * ncb + colblock) KB),
// or one E4M3 plane of 1 KB images of 32 columns x 32 rows (FP8 mode,
// image (kstep, colblock) at (kstep * ncb + colblock) KB),
// or one FP64 array ([k][col], row-major) for the native FP64 mode.
struct OpDesc {
    int32_t family;
    int32_t t_shift;     // |U| < 2^t_shift (t = log2 of the term count)
    int32_t nterms;
    int32_t first_term;
    int64_t out_col;     // first column of this operand inside the family
    int32_t K_pitch;     // contraction rows written (multiple of PREP_K)
    int32_t P_pad;       // columns written (multiple of TILE)
    int64_t tile_base;   // prefix count of prep tiles (flat grid)
    // Operands of one family and shape share a tile range, interleaved: tile
    // tile_base + i of the range is tile i / ilv_n of the group's operand
    // i mod ilv_n, so operand sums that read the same blocks of A read them
    // at about the same time (L2 hits).  ilv_i: this operand's index in its
    // group (0 .. ilv_n - 1; ilv_n <= 1: not interleaved).
    int32_t ilv_n;
    int32_t ilv_i;
    // Fused group (fuse_ns > 0): the group's operands (ilv_n of them, this
    // one ilv_i-th) draw on the same fuse_ns <= FUSE_MAX_SRC blocks of A
    // (entries fuse_src .. of the plan's source list), and one prep tile
    // writes tile `local` of every operand of the group from one read of
    // those blocks.  fuse_nsub groups of one family and shape share a tile
    // range, interleaved (tile i of the range: group i mod fuse_nsub, local
    // tile i / fuse_nsub; this one is group fuse_isub), so groups that read
    // the same blocks read them at about the same time.  fuse_uni: every
    // operand of the group has the same t_shift, so each block is converted
    // to fixed point once.  fuse_f0: the group also writes the digit planes
    // of A (family 0) for the elements of its source blocks (the top block's
    // two sides, whose quadrants tile A; see Plan::f0_zero).
    int32_t fuse_src;
    int16_t fuse_ns;
    int8_t fuse_uni;
    int8_t fuse_f0;
    int32_t fuse_coef;   // coefficient of source q (-1, 0, +1) in bits 2q, 2q + 1
    int16_t fuse_isub, fuse_nsub;
};

// Source blocks of a fused prep group: the four quadrants of one side of a
// depth-1 block.  (Depth-2 groups of up to eight blocks, with four lanes of 4
// rows per column, measured slower than the one-operand path: 12.3 against
// 8.3 ms of prep at 16384^2.)
constexpr int FUSE_MAX_SRC = 4;
constexpr int FUSE_MAX_OPS = 8;   // operands of a fused prep group
constexpr int FUSE_MAX_SUBGROUPS = 32;  // fused groups sharing one tile range

// Fused prep tiles are 16 contraction rows x FUSED_TC columns: two lanes of
// 8 rows each share a column.
constexpr int FUSED_TC = 128;
inline int64_t fused_tiles_for(int64_t K_pitch, int64_t P_pad) {
    return (K_pitch / KSTEP) * ((P_pad + FUSED_TC - 1) / FUSED_TC);
}

struct Family {
    int64_t K_pitch;     // contraction pitch in elements (multiple of PREP_K)
    int64_t cols;        // total columns (multiple of TILE, plus TILE of padding)
    int64_t offset;      // byte offset of the family in the workspace
    int64_t plane_elems; // elements per digit plane = cols * K_pitch
};

// One leaf output tile (TILE x TILE), all digit pairs (or one FP64 product).
struct LeafTask {
    int32_t fam_u, fam_v;   // operand families (-1: A itself, native FP64 only)
    int32_t col_u, col_v;   // first column of the tile's rows / columns
    int32_t k0, klen;       // contraction offset of the row operand, length
    int32_t rows, cols;     // valid output rows / columns (<= TILE)
    int32_t diag;           // 1: tile crosses the diagonal (see diag_off)
    int32_t kind;           // OUT_* below
    int32_t shift;          // product unit exponent adjustment (t_u + t_v)
    int32_t eu, ev;         // exponent index of tile row 0 / column 0 (-1: none)
    int32_t diag_off;       // with diag: write only where col <= row + diag_off
    int64_t out_off;        // element offset of the tile origin in the output
    int64_t out_ld;         // output leading dimension (elements)
                            // (packed lower-triangular C: out_off = first row,
                            //  out_ld = first column of the tile in C)
    int32_t hbits;          // extra fraction bits of T for short contractions
    int32_t k0v;            // contraction offset of the column operand (k0: row operand)
    int32_t prob;           // batched calls: problem index (planes and C of that problem)
    int32_t unit;           // node of the recursion the tile belongs to (a diagonal
                            // panel, a classical block or one Strassen product)
};

// One problem of a batched call (device table, one entry per problem).
struct BatchProb {
    const void *A;          // A_i (device)
    void *C;                // C_i (device)
    int64_t m, n, lda, ldc;
    int64_t col_off;        // first column of this problem in the batch's exponent array
    int64_t plane_off;      // byte offset of its digit planes in the planes block
    int64_t ncb;            // 32-column image blocks per digit plane
    int64_t K_pitch;        // contraction rows of its planes (multiple of PREP_K)
    int64_t P_pad;          // columns written by prep: n rounded up to an image block
    int64_t prep_base;      // first prep tile of this problem (prefix over problems)
    int32_t tc;             // prep tile columns for this problem (64, 128 or 256)
    int32_t pad;
};

// Batched problems: the prep tile width (64, 128 or 256 columns, with 4096 /
// width rows) that wastes the fewest columns on P_pad, and its tile count.
inline int batch_tile_cols(int64_t P_pad) {
    int best = 256;
    int64_t best_cols = ((P_pad + 255) / 256) * 256;
    for (int tc : {128, 64}) {
        const int64_t c = ((P_pad + tc - 1) / tc) * tc;
        if (c < best_cols) best = tc, best_cols = c;
    }
    return best;
}
inline int64_t batch_prep_tiles(int64_t K_pitch, int64_t P_pad, int tc) {
    return (K_pitch / (4096 / tc)) * ((P_pad + tc - 1) / tc);
}

// Prep tiles of one operand of K_pitch rows and P_pad columns.
inline int64_t prep_tiles_for(bool digits, int64_t K_pitch, int64_t P_pad, bool fp8 = false) {
    if (fp8) return (K_pitch / PREP8_TK) * ((P_pad + PREP8_TC - 1) / PREP8_TC);
    return digits ? (K_pitch / PREP_TK) * ((P_pad + PREP_TC - 1) / PREP_TC) : (K_pitch / PREP_K) * (P_pad / PREP_C);
}

// Extra fraction bits of the leaf's int64 sum for a contraction of K rows:
// T is kept in units of 2^-(T_FRAC + h) of the leading digit product, which
// stays below 2^63 while K * 2^(T_BOUND_LOG2 + h) < 2^62.
inline int hbits_for(int64_t K) {
    int lg = 0;
    while ((int64_t(1) << lg) < K) ++lg;
    int h = 19 - lg;
    return h < 0 ? 0 : (h > 9 ? 9 : h);
}

enum OutKind : int {
    OUT_C_F64 = 0,   // double into C, scaled by 2^(e_row + e_col)
    OUT_C_F32 = 1,   // float into C, scaled by 2^(e_row + e_col)
    OUT_M_I64 = 2,   // exact int64 partial into the product workspace
    OUT_M_F64 = 3    // double into the product workspace (native FP64, FP8)
};

// One Strassen result sum: region of C = sum_r coef_r * M_r (clipped).
struct CombTerm {
    int64_t src_off;  // element offset of M_r's origin in the product workspace
    int32_t ld;       // M_r leading dimension
    int32_t coef;     // +1 / -1
    int32_t shift;    // unit exponent of M_r (t_u + t_v)
    int32_t pad;
};

struct CombDesc {
    int64_t c_off;       // element offset in C of the region origin
    int32_t rows, cols;  // region extent
    int32_t e_row0;      // A column of region row 0 (exponent index)
    int32_t e_col0;      // A column of region column 0
    int32_t first_term, nterms;
    int64_t tile_base;   // prefix count of combine tiles (COMB_ROWS x COMB_COLS)
    int32_t wide;        // 1: the result bound reaches 2^63: summed in int128
                         //    (else modulo 2^64, exact as the result fits)
    int32_t smin;        // smallest term shift; products are summed in units 2^smin
    int32_t diag;        // 1: the region crosses the diagonal: write only where
    int32_t diag_off;    //    col <= row + diag_off (split contraction of a diagonal tile)
};

// Split contraction: plain tiles of a plan with few tiles and a long
// contraction are computed as this many contraction chunks (exact partial
// products in the product workspace) summed by the combine in a fixed order,
// when the tile count is below SPLITK_TILES_PER_CTA x the CTA count and
// every chunk keeps at least SPLITK_MIN_ROWS rows.
constexpr int SPLITK_TILES_PER_CTA = 4;
constexpr int64_t SPLITK_MIN_ROWS = 4096;
constexpr int SPLITK_MAX = 16;
constexpr int COMB_ROWS = 64;  // combine tile: 64 rows x 32 columns, 8 rows per thread
constexpr int COMB_COLS = 32;

// One off-diagonal block of the AtA recursion: C[r0:r0+p, c0:c0+q] =
// A[:, r0:r0+p]^T A[:, c0:c0+q] by `depth` Strassen levels (0: classical tiles).
struct BlockInfo {
    int64_t r0, p, c0, q;
    int32_t depth;
    int32_t pad;
};

struct PlanParams {
    int64_t m = 0, n = 0, lda = 0, ldc = 0;
    int mode = MODE_F64_EMU;
    int cutoff = 0;          // 0 = auto
    int depth = -1;          // -1 = auto
    int slices = 0;          // 0 = auto
    int strassen_min = 0;    // Strassen splits a (sub)block only while both its
                             // sides are >= strassen_min (0 = auto)
    int split_search = 1;    // 1: place Strassen splits by the leaf-step cost
                             // model; 0: always split at the aligned middle
    int num_ctas = 0;        // > 1: lay the tile list out for this many
                             // persistent leaf CTAs (longest-first balance)
    int trans = 0;           // 1: the operand is the transpose of a row-major
                             // n x m array (A A^T of that array): element (i, j)
                             // of the m x n operand at A[j * lda + i], lda >= m
    int packed = 0;          // 1: C is stored as a packed lower triangle, entry
                             // (j, k) at j (j + 1) / 2 + k (ldc unused)
    int variant = VARIANT_STRASSEN;  // coefficient tables of the off-diagonal products
    int streams = 1;         // > 1: static partition of the recursion's units over
                             // this many leaf launches on their own streams
    int split_k = 0;         // contraction chunks per plain tile: 0 = automatic
                             // (few tiles, long contraction), 1 = never, > 1 = that many
};

// One leaf launch of a static partition: tasks [first, first + count) of the
// plan's task list, laid out for `ctas` persistent CTAs.
struct LeafGroup {
    int64_t first, count;
    int32_t ctas;
    int32_t pad;
    double steps;            // K steps of its tiles (the load the partition balances)
};

// Element offset of entry (j, k), k <= j, of a packed lower triangle.
inline int64_t packed_index(int64_t j, int64_t k) { return j * (j + 1) / 2 + k; }

struct Plan {
    PlanParams p;
    int cutoff = 0, depth = 0, slices = 0, strassen_min = 0, variant = VARIANT_STRASSEN;
    int split_k = 1;       // contraction chunks per plain tile (1: none)
    int tile_n = TILE_N;   // leaf tile columns (tile_cols of the mode)
    int64_t n_panels = 0, n_blocks = 0, n_products = 0;
    int64_t n_reused = 0;  // Strassen operands read from the planes of A
    int64_t n_tiles = 0;   // leaf tiles (tasks also holds empty balance fillers)
    std::vector<Family> families;       // [0] = plain digits of A (if used)
    std::vector<OpDesc> ops;
    std::vector<OpTerm> terms;
    std::vector<OpTerm> fsrc;           // source blocks of the fused prep groups
    int64_t n_fused = 0;                // fused prep groups
    std::vector<LeafTask> tasks;
    std::vector<CombDesc> combs;
    std::vector<CombTerm> cterms;
    std::vector<BlockInfo> blocks;      // off-diagonal blocks, in recursion order
    std::vector<LeafGroup> groups;      // static partition (PlanParams::streams > 1), else empty
    int32_t n_units = 0;                // recursion units the tiles belong to
    int64_t prep_tiles = 0, comb_tiles = 0;
    int64_t fused_tiles = 0;            // prep tiles [0, fused_tiles) belong to fused groups
    // The planes of A are written by the top block's fused groups, which
    // cover A's rows and columns but not the planes' zero padding: the
    // padding is zeroed once when the plan's tables are loaded into the
    // workspace, and nothing else writes family 0 while they stay loaded.
    bool f0_zero = false;
    // workspace layout (byte offsets)
    int64_t off_colmax = 0, off_expo = 0, off_products = 0, product_bytes = 0;
    int64_t off_tables = 0, table_bytes = 0, workspace_bytes = 0;
    // byte offsets of the task tables inside the table block
    int64_t t_ops = 0, t_terms = 0, t_tasks = 0, t_combs = 0, t_cterms = 0, t_fsrc = 0;
    double leaf_madds = 0, plain_madds = 0;   // per digit pair / per FP64 product
    bool uses_digits() const { return p.mode != MODE_F64; }
};

// Plan of a batched call: every problem as plain lower-triangle tiles of
// its own digit planes, all tiles in one task list.
struct BatchPlan {
    int mode = MODE_F32;
    int slices = 0;
    int64_t count = 0;
    std::vector<BatchProb> probs;
    std::vector<LeafTask> tasks;
    int64_t n_tiles = 0;
    int64_t total_cols = 0;     // exponent entries
    int64_t plane_bytes = 0;    // digit planes of all problems
    int64_t prep_tiles = 0;
    int64_t max_col_chunks = 0; // max over problems of ceil(n / 64) (exponent blocks)
    double leaf_madds = 0;
};

// Build the batched plan for `count` problems (host arrays m, n, lda, ldc, A,
// C).  Problems with n == 0 or m == 0 get no tiles (m == 0 is zero-filled by
// the caller).  Returns false with *err set on invalid input.
bool make_batch_plan(int mode, int slices, int num_ctas, int64_t count, const int64_t *m, const int64_t *n,
                     const int64_t *lda, const int64_t *ldc, const void *const *A, void *const *C,
                     BatchPlan *plan, std::string *err);

// Digits per column for a mode (slices == 0 -> default).
int default_slices(int mode, int64_t m);
// Build the full plan.  Returns false (and sets *err) on invalid parameters.
bool make_plan(const PlanParams &pp, Plan *plan, std::string *err);
// Copy the task tables into a contiguous host buffer laid out as
// plan.t_* describe (size plan.table_bytes).
void pack_tables(const Plan &plan, std::vector<uint8_t> *buf);

// Reorders plan.tasks for num_ctas persistent leaf CTAs (longest first,
// greedy least-loaded), padding with empty tasks; make_plan calls it when
// PlanParams::num_ctas > 1.
void balance_tasks(Plan &plan, int num_ctas);

// Reorders plan.tasks into `streams` static groups of whole recursion units
// (plan.groups), each laid out for its share of num_ctas CTAs; make_plan
// calls it when PlanParams::streams > 1.
void partition_units(Plan &plan, int streams, int num_ctas);

}  // namespace ata
