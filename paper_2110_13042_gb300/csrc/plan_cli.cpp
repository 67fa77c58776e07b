// Host-only planner inspector (used by the CPU tests): builds the plan for
//   plan_cli m n mode cutoff depth slices [strassen_min [split_search [num_ctas [variant [streams]]]]]
// and prints key=value statistics, including a coverage check that every
// lower-triangle entry of C is produced exactly once (by a diagonal/classical
// tile or by one Strassen result sum) and no upper entry is produced.
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "plan.h"

using namespace ata;

int main(int argc, char **argv) {
    if (argc < 7) return 2;
    PlanParams pp;
    pp.m = std::atoll(argv[1]);
    pp.n = std::atoll(argv[2]);
    pp.lda = pp.ldc = pp.n > 0 ? pp.n : 1;
    pp.mode = std::atoi(argv[3]);
    pp.cutoff = std::atoi(argv[4]);
    pp.depth = std::atoi(argv[5]);
    pp.slices = std::atoi(argv[6]);
    pp.strassen_min = argc > 7 ? std::atoi(argv[7]) : 1;
    pp.split_search = argc > 8 ? std::atoi(argv[8]) : 1;
    pp.num_ctas = argc > 9 ? std::atoi(argv[9]) : 0;
    pp.variant = argc > 10 ? std::atoi(argv[10]) : 0;
    pp.streams = argc > 11 ? std::atoi(argv[11]) : 1;
    pp.split_k = argc > 12 ? std::atoi(argv[12]) : 0;
    Plan P;
    std::string err;
    if (!make_plan(pp, &P, &err)) {
        std::fprintf(stderr, "%s\n", err.c_str());
        return 1;
    }
    const int64_t n = pp.n, ldc = pp.ldc;
    std::vector<uint8_t> cov(static_cast<size_t>(n * n), 0);
    double s_leaf = 0, s_plain = 0;
    // K-steps per leaf CTA under the kernel's round-robin walk
    const int G = pp.num_ctas > 1 ? pp.num_ctas : 152;
    std::vector<int64_t> cta(G, 0);
    for (size_t i = 0; i < P.tasks.size(); ++i) cta[i % G] += (P.tasks[i].klen + KSTEP - 1) / KSTEP;
    int64_t cta_max = 0, cta_sum = 0;
    for (int64_t v : cta) cta_max = std::max(cta_max, v), cta_sum += v;
    for (const LeafTask &t : P.tasks) {
        if (t.kind == OUT_M_I64 || t.kind == OUT_M_F64) {
            s_leaf += static_cast<double>(t.klen) * t.rows * t.cols;
            continue;
        }
        const int64_t r0 = t.out_off / ldc, c0 = t.out_off % ldc;
        for (int r = 0; r < t.rows; ++r)
            for (int c = 0; c < t.cols; ++c)
                if (!t.diag || c <= r + t.diag_off) cov[(r0 + r) * n + c0 + c]++;
    }
    for (const CombDesc &d : P.combs) {
        const int64_t r0 = d.c_off / ldc, c0 = d.c_off % ldc;
        s_plain += static_cast<double>(pp.m) * d.rows * d.cols;
        for (int r = 0; r < d.rows; ++r)
            for (int c = 0; c < d.cols; ++c)
                if (!d.diag || c <= r + d.diag_off) cov[(r0 + r) * n + c0 + c]++;
    }
    // Prep tiles: walk the flat tile range the way the prep kernels map it
    // (last operand with tile_base <= tile, then the interleaved group) and
    // check that every tile of every operand is produced exactly once.
    bool prep_ok = true;
    int64_t groups = 0;
    {
        const bool digits = pp.mode != MODE_F64, fp8 = pp.mode == MODE_F32_FP8;
        std::vector<std::vector<uint8_t>> seen(P.ops.size());
        for (size_t i = 0; i < P.ops.size(); ++i) {
            seen[i].assign(static_cast<size_t>(P.ops[i].fuse_ns > 0
                                                   ? fused_tiles_for(P.ops[i].K_pitch, P.ops[i].P_pad)
                                                   : prep_tiles_for(digits, P.ops[i].K_pitch, P.ops[i].P_pad, fp8)),
                           0);
            if (P.ops[i].ilv_i == 0) groups++;
            if (P.ops[i].ilv_n < 1 || P.ops[i].ilv_i >= P.ops[i].ilv_n) prep_ok = false;
            if (P.ops[i].ilv_i > 0 && (P.ops[i].tile_base != P.ops[i - 1].tile_base ||
                                       P.ops[i].K_pitch != P.ops[i - 1].K_pitch ||
                                       P.ops[i].P_pad != P.ops[i - 1].P_pad ||
                                       P.ops[i].family != P.ops[i - 1].family))
                prep_ok = false;
        }
        for (int64_t tile = 0; tile < P.prep_tiles && prep_ok; ++tile) {
            size_t i = 0;
            for (size_t j = 0; j < P.ops.size(); ++j)
                if (P.ops[j].tile_base <= tile) i = j;
            const int64_t g = tile - P.ops[i].tile_base;
            const int64_t nn = P.ops[i].ilv_n;
            if (P.ops[i].fuse_ns > 0) {  // fused range: sub-group g mod nsub, tile g / nsub of every member
                const int64_t nsub = P.ops[i].fuse_nsub, sub = g % nsub, lt = g / nsub;
                size_t last = i;  // last operand of sub-group `sub`
                while (P.ops[last].fuse_isub > sub) last -= static_cast<size_t>(P.ops[last].ilv_i) + 1;
                if (P.ops[last].fuse_isub != sub || tile >= P.fused_tiles) prep_ok = false;
                const size_t lead = last - static_cast<size_t>(P.ops[last].ilv_i);
                for (int64_t mi = 0; mi < P.ops[last].ilv_n && prep_ok; ++mi) {
                    const size_t op = lead + static_cast<size_t>(mi);
                    if (P.ops[op].fuse_ns != P.ops[last].fuse_ns || P.ops[op].tile_base != P.ops[i].tile_base ||
                        P.ops[op].fuse_isub != sub || lt >= static_cast<int64_t>(seen[op].size()) || seen[op][lt]++)
                        prep_ok = false;
                }
                continue;
            }
            if (tile < P.fused_tiles) prep_ok = false;
            const size_t op = nn > 1 ? i - P.ops[i].ilv_i + static_cast<size_t>(g % nn) : i;
            const int64_t local = nn > 1 ? g / nn : g;
            if (local < 0 || local >= static_cast<int64_t>(seen[op].size()) || seen[op][local]++) prep_ok = false;
        }
        for (const auto &v : seen)
            for (uint8_t x : v)
                if (x != 1) prep_ok = false;
        // fused groups: every term names a source block that is the term's region
        for (const OpDesc &o : P.ops) {
            if (o.fuse_ns <= 0) continue;
            if (o.fuse_ns > FUSE_MAX_SRC || o.fuse_src + o.fuse_ns > static_cast<int64_t>(P.fsrc.size()))
                prep_ok = false;
            for (int t = 0; t < o.nterms && prep_ok; ++t) {
                const OpTerm &tm = P.terms[static_cast<size_t>(o.first_term + t)];
                if (tm.src < 0 || tm.src >= o.fuse_ns) {
                    prep_ok = false;
                    break;
                }
                const OpTerm &sb = P.fsrc[static_cast<size_t>(o.fuse_src + tm.src)];
                if (sb.row0 != tm.row0 || sb.col0 != tm.col0 || sb.rows != tm.rows || sb.cols != tm.cols)
                    prep_ok = false;
            }
        }
    }
    // Combine tiles: COMB_ROWS x COMB_COLS per block, prefix tile_base.
    bool comb_ok = true;
    {
        int64_t expect = 0;
        for (const CombDesc &d : P.combs) {
            if (d.tile_base != expect) comb_ok = false;
            expect += ((d.rows + COMB_ROWS - 1) / COMB_ROWS) * ((d.cols + COMB_COLS - 1) / COMB_COLS);
        }
        if (expect != P.comb_tiles) comb_ok = false;
    }
    int64_t covered = 0, overlap = 0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t k = 0; k < n; ++k) {
            const int v = cov[j * n + k];
            if (k <= j && v == 1) covered++;
            if (v > 1 || (k > j && v > 0)) overlap++;
        }
    // Static partition: groups are consecutive, cover the task list, use at
    // most the CTAs given, and every recursion unit lies in one group.
    bool groups_ok = true;
    int64_t group_steps_max = 0;
    if (!P.groups.empty()) {
        int64_t next = 0, ctas = 0;
        std::vector<int> unit_group(static_cast<size_t>(P.n_units), -1);
        for (size_t g = 0; g < P.groups.size(); ++g) {
            const LeafGroup &lg = P.groups[g];
            if (lg.first != next || lg.count <= 0 || lg.ctas < 1) groups_ok = false;
            next = lg.first + lg.count;
            ctas += lg.ctas;
            std::vector<int64_t> per(static_cast<size_t>(lg.ctas), 0);
            for (int64_t i = lg.first; i < lg.first + lg.count; ++i) {
                const LeafTask &t = P.tasks[static_cast<size_t>(i)];
                per[static_cast<size_t>((i - lg.first) % lg.ctas)] += (t.klen + KSTEP - 1) / KSTEP;
                if (t.klen == 0) continue;  // balance filler
                int &ug = unit_group[static_cast<size_t>(t.unit)];
                if (ug >= 0 && ug != static_cast<int>(g)) groups_ok = false;
                ug = static_cast<int>(g);
            }
            for (int64_t v : per) group_steps_max = std::max(group_steps_max, v);
        }
        if (next != static_cast<int64_t>(P.tasks.size()) || ctas > G) groups_ok = false;
    }
    // Execute the plan's tables in plain FP64 on a small-integer A (every
    // step exact): operand sums into the families, leaf tiles over them
    // (family 0 is A itself), the result sums; compare with A^T A.
    double verify_err = -1.0;
    bool bounds_ok = true;  // every leaf read stays inside its family's rows
    if (argc > 13 && std::atoi(argv[13]) == 1 && pp.mode != MODE_F64) {
        const int64_t m = pp.m;
        std::vector<double> A(static_cast<size_t>(m * n));
        uint64_t z = 2110;
        for (double &a : A) {
            z = z * 6364136223846793005ull + 1442695040888963407ull;
            a = static_cast<double>(static_cast<int>((z >> 33) % 9) - 4);
        }
        std::vector<std::vector<double>> fam(P.families.size());
        for (size_t f = 0; f < P.families.size(); ++f)
            fam[f].assign(static_cast<size_t>(P.families[f].K_pitch * P.families[f].cols), 0.0);
        for (const OpDesc &o : P.ops) {
            const Family &F = P.families[static_cast<size_t>(o.family)];
            if (o.fuse_f0) {  // the group also writes family 0 for its source blocks
                const Family &F0 = P.families[0];
                for (int q = 0; q < o.fuse_ns; ++q) {
                    const OpTerm &sb = P.fsrc[static_cast<size_t>(o.fuse_src + q)];
                    for (int k = 0; k < sb.rows; ++k)
                        for (int c = 0; c < sb.cols; ++c)
                            fam[0][static_cast<size_t>((sb.row0 + k) * F0.cols + sb.col0 + c)] =
                                A[static_cast<size_t>((sb.row0 + k) * n + sb.col0 + c)];
                }
            }
            for (int t = 0; t < o.nterms; ++t) {
                const OpTerm &tm = P.terms[static_cast<size_t>(o.first_term + t)];
                for (int k = 0; k < tm.rows; ++k)
                    for (int c = 0; c < tm.cols; ++c)
                        fam[static_cast<size_t>(o.family)][static_cast<size_t>(k * F.cols + o.out_col + c)] +=
                            tm.coef * A[static_cast<size_t>((tm.row0 + k) * n + tm.col0 + c)];
            }
        }
        std::vector<double> Cv(static_cast<size_t>(n * n), 0.0), M(static_cast<size_t>(P.product_bytes / 8 + 1), 0.0);
        for (const LeafTask &t : P.tasks) {
            if (t.klen == 0) continue;
            const Family &FU = P.families[static_cast<size_t>(t.fam_u)], &FV = P.families[static_cast<size_t>(t.fam_v)];
            const std::vector<double> &U = fam[static_cast<size_t>(t.fam_u)], &V = fam[static_cast<size_t>(t.fam_v)];
            // the leaf loads whole TILE_M x tile_n boxes: inside the families' columns
            if (t.col_u + TILE_M > FU.cols || t.col_v + P.tile_n > FV.cols || t.cols > P.tile_n) bounds_ok = false;
            for (int r = 0; r < t.rows; ++r)
                for (int c = 0; c < t.cols; ++c) {
                    if (t.diag && c > r + t.diag_off) continue;
                    // the leaf reads whole K steps of `ks` rows, inside the families
                    const int ks = kstep_rows(pp.mode);
                    const int kread = (t.klen + ks - 1) / ks * ks;
                    if (t.k0 + kread > FU.K_pitch || t.k0v + kread > FV.K_pitch) bounds_ok = false;
                    double s = 0;
                    for (int k = 0; k < kread && t.k0 + k < FU.K_pitch && t.k0v + k < FV.K_pitch; ++k)
                        s += U[static_cast<size_t>((t.k0 + k) * FU.cols + t.col_u + r)] *
                             V[static_cast<size_t>((t.k0v + k) * FV.cols + t.col_v + c)];
                    if (t.kind == OUT_M_I64 || t.kind == OUT_M_F64)
                        M[static_cast<size_t>(t.out_off + r * t.out_ld + c)] = s;
                    else
                        Cv[static_cast<size_t>(t.out_off + r * t.out_ld + c)] = s;
                }
        }
        for (const CombDesc &d : P.combs)
            for (int r = 0; r < d.rows; ++r)
                for (int c = 0; c < d.cols; ++c) {
                    if (d.diag && c > r + d.diag_off) continue;
                    double s = 0;
                    for (int i = 0; i < d.nterms; ++i) {
                        const CombTerm &ct = P.cterms[static_cast<size_t>(d.first_term + i)];
                        s += ct.coef * M[static_cast<size_t>(ct.src_off + r * ct.ld + c)];
                    }
                    Cv[static_cast<size_t>(d.c_off + r * ldc + c)] = s;
                }
        verify_err = 0.0;
        for (int64_t j = 0; j < n; ++j)
            for (int64_t k = 0; k <= j; ++k) {
                double s = 0;
                for (int64_t i = 0; i < m; ++i) s += A[static_cast<size_t>(i * n + j)] * A[static_cast<size_t>(i * n + k)];
                verify_err = std::max(verify_err, std::abs(s - Cv[static_cast<size_t>(j * n + k)]));
            }
    }
    int64_t wide = 0;  // combine regions summed in int128
    for (const CombDesc &d : P.combs) wide += d.wide;
    std::printf("verify_err=%g verify_bounds_ok=%d wide_regions=%lld fused_groups=%lld fused_tiles=%lld f0_fused=%d ",
                verify_err, bounds_ok ? 1 : 0, static_cast<long long>(wide), static_cast<long long>(P.n_fused),
                static_cast<long long>(P.fused_tiles), P.f0_zero ? 1 : 0);
    std::printf("cutoff=%d depth=%d slices=%d panels=%lld blocks=%lld products=%lld tiles=%zu "
                "covered=%lld overlap=%lld cterms=%zu ops=%zu families=%zu workspace=%lld "
                "strassen_leaf_madds=%.0f strassen_plain_madds=%.0f reused=%lld cta_steps_max=%lld "
                "cta_steps_sum=%lld prep_tiles=%lld prep_groups=%lld prep_map_ok=%d comb_map_ok=%d "
                "units=%d leaf_groups=%zu groups_ok=%d group_steps_max=%lld\n",
                P.cutoff, P.depth, P.slices, (long long)P.n_panels, (long long)P.n_blocks,
                (long long)P.n_products, (size_t)P.n_tiles, (long long)covered, (long long)overlap,
                P.cterms.size(), P.ops.size(), P.families.size(), (long long)P.workspace_bytes, s_leaf,
                s_plain, (long long)P.n_reused, (long long)cta_max, (long long)cta_sum, (long long)P.prep_tiles,
                (long long)groups, prep_ok ? 1 : 0, comb_ok ? 1 : 0, P.n_units, P.groups.size(), groups_ok ? 1 : 0,
                (long long)group_steps_max);
    return 0;
}
