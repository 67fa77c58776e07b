"""CPU checks of the static partition over streams (ata_config.streams, the
counterpart of the paper's static task tree, Section 4.1-4.2): the planner's
groups cover the task list, keep every recursion unit (diagonal panel,
classical block, Strassen product) in one group, use no more CTAs than the
persistent launch, and leave the produced entries unchanged."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cli(tmp_path_factory):
    src = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc")
    out = str(tmp_path_factory.mktemp("cli") / "plan_cli")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", src, os.path.join(src, "plan_cli.cpp"),
                    os.path.join(src, "plan.cpp"), "-o", out], check=True)

    def run(m, n, mode, cutoff, depth, smin, streams, variant=0, split=0, verify=0):
        r = subprocess.run([out, str(m), str(n), str(mode), str(cutoff), str(depth), "0", str(smin), "1", "152",
                            str(variant), str(streams), str(split), str(verify)], capture_output=True, text=True,
                           check=True)
        return {k: float(v) for k, v in (kv.split("=") for kv in r.stdout.split())}
    return run


@pytest.mark.parametrize("streams", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin", [
    (8192, 8192, 1, 0, 1, 4096), (3000, 5000, 2, 0, 2, 512), (700, 1300, 5, 200, 2, 2),
    (500, 900, 0, 128, 1, 2), (1000, 300, 1, 0, 0, 4096)])
def test_partition_covers_and_keeps_units_whole(cli, streams, m, n, mode, cutoff, depth, smin):
    one = cli(m, n, mode, cutoff, depth, smin, 1, split=1)  # no tail split: the same tiles
    part = cli(m, n, mode, cutoff, depth, smin, streams, split=1)
    assert part["covered"] == n * (n + 1) // 2 and part["overlap"] == 0
    assert part["groups_ok"] == 1
    assert 1 <= part["leaf_groups"] <= min(streams, part["units"])
    assert part["tiles"] == one["tiles"] and part["products"] == one["products"]
    assert part["cta_steps_sum"] == one["cta_steps_sum"]


def test_partition_is_a_static_comparison_not_a_speedup(cli):
    """Whole units per group cannot balance as finely as tiles over one
    persistent grid: the busiest CTA of the partition carries at least the
    persistent layout's load (the paper's AtA-S has the same limit)."""
    one = cli(8192, 8192, 1, 0, 1, 4096, 1)
    for s in (2, 4, 8):
        part = cli(8192, 8192, 1, 0, 1, 4096, s)
        assert part["group_steps_max"] >= one["cta_steps_max"]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin,streams,split", [
    (531, 700, 1, 350, 1, 2, 1, 0), (250, 330, 1, 0, 2, 16, 1, 0), (129, 515, 4, 0, 8, 16, 1, 0),
    (300, 257, 2, 32, 1, 2, 4, 0), (1300, 200, 1, 0, 0, 4096, 1, 4), (701, 300, 5, 64, 1, 2, 3, 3),
    (333, 401, 2, 100, 3, 8, 2, 2)])
def test_plan_tables_compute_the_product(cli, variant, m, n, mode, cutoff, depth, smin, streams, split):
    """plan_cli's interpreter executes the plan's operand, leaf and combine
    tables in FP64 on a small-integer A (every step exact), reading whole K
    steps as the leaf does, and compares with the direct A^T A: a wrong
    coefficient, offset, term, sum or contraction tail anywhere in the planner
    shows as a nonzero error (an odd m with both operands of a Winograd
    product read in place from A caught one such tail)."""
    r = cli(m, n, mode, cutoff, depth, smin, streams, variant=variant, split=split, verify=1)
    assert r["verify_err"] == 0.0 and r["verify_bounds_ok"] == 1


@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin,variant,split,expect_wide", [
    (600, 1111, 1, 300, 8, 64, 1, 0, False),   # Winograd down to 64 columns: huge terms, small result
    (8192, 8192, 1, 0, 1, 4096, 0, 1, False),  # the Strassen result sums (no chunked tiles)
    (262144, 2048, 1, 0, 0, 4096, 0, 0, True),  # 4 contraction chunks of 65536 rows: result up to 2^64
    (700, 900, 5, 0, 2, 2, 0, 0, False)])       # FP8 sums products in FP64
def test_wide_combine_regions(cli, m, n, mode, cutoff, depth, smin, variant, split, expect_wide):
    """The combine sums exactly: modulo 2^64 where the result (an entry of
    A^T A, at most m in scaled units, plus the operands' rounding) fits in
    int64 however large its terms, in int128 (wide) only where it may not."""
    r = cli(m, n, mode, cutoff, depth, smin, 1, variant=variant, split=split)
    assert (r["wide_regions"] > 0) == expect_wide


@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin,variant,expect", [
    (8192, 8192, 1, 2048, 1, 4096, 0, 2),   # both sides of the top block's sums, four quadrants each
    (8192, 8192, 1, 2048, 2, 2048, 0, 2),   # depth 2 (up to eight blocks): not fused; a depth-1 block is
    (531, 700, 1, 350, 1, 2, 1, 4),         # Winograd: mixed term counts, two blocks
    (1000, 1100, 2, 0, 1, 64, 0, 8),
    (250, 330, 1, 0, 2, 16, 0, 0),
    (700, 900, 5, 0, 1, 2, 0, 0)])          # FP8 planes are not fused
def test_fused_prep_groups(cli, m, n, mode, cutoff, depth, smin, variant, expect):
    """Operand sums that draw on the same four quadrants of A (one side of a
    depth-1 block) are written from one read of them (a fused prep group);
    the prep tile map still produces every tile of every operand exactly
    once and every term names its own source block."""
    r = cli(m, n, mode, cutoff, depth, smin, 1, variant=variant)
    assert r["fused_groups"] == expect
    assert r["prep_map_ok"] == 1
    assert (r["fused_tiles"] > 0) == (expect > 0)


@pytest.mark.parametrize("m,n,mode,cutoff", [(8192, 8192, 1, 8192), (4096, 4096, 2, 4096), (8192, 8192, 5, 8192)])
def test_tail_split_balances_the_last_wave(cli, m, n, mode, cutoff):
    """Plain tiles that leave the last wave of the 152 persistent CTAs partly
    idle: the last (tiles mod 152) are computed as contraction chunks, and the
    busiest CTA carries within 1% of the average load (without the split,
    up to one whole tile more)."""
    r = cli(m, n, mode, cutoff, 0, 4096, 1)
    avg = r["cta_steps_sum"] / 152
    assert r["cta_steps_max"] <= 1.01 * avg + 8
    assert r["comb_map_ok"] == 1 and r["covered"] == n * (n + 1) // 2 and r["overlap"] == 0


def test_tail_split_plan_computes_the_product(cli):
    r = cli(2048, 600, 1, 0, 0, 4096, 1, verify=1)
    assert r["wide_regions"] > 0  # the split tiles' chunks
    assert r["verify_err"] == 0.0 and r["verify_bounds_ok"] == 1


@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin,variant,f0", [
    (8192, 8192, 1, 2048, 1, 4096, 0, 1),  # the top block's quadrants tile A
    (512, 384, 1, 0, 1, 2, 0, 1),
    (512, 384, 2, 0, 1, 2, 1, 1),          # Winograd, FP32
    (513, 385, 1, 0, 1, 2, 0, 0),          # second row block starts off a K step: A keeps its own pass
    (8192, 8192, 1, 8192, 0, 4096, 0, 0),  # no Strassen block
    (700, 900, 5, 0, 1, 2, 0, 0)])         # FP8 is not fused
def test_planes_of_a_from_the_fused_reads(cli, m, n, mode, cutoff, depth, smin, variant, f0):
    """Where the fused groups' source blocks tile A exactly (the top block's
    two sides at depth 1), they also write the digit planes of A, and A's own
    prep pass is dropped; the plan still computes the product (interpreter,
    small cases) and produces every prep tile once."""
    verify = 1 if m * n <= 600 * 600 else 0
    r = cli(m, n, mode, cutoff, depth, smin, 1, variant=variant, verify=verify)
    assert r["f0_fused"] == f0 and r["prep_map_ok"] == 1
    if verify:
        assert r["verify_err"] == 0.0 and r["verify_bounds_ok"] == 1


@pytest.mark.parametrize("m,expect_wide", [(300, True), (16384, True), (16385, False), (40000, False)])
def test_one_digit_bf16_tile_width(cli, m, expect_wide):
    """One BF16 digit runs on 128 x 192 tiles with 32-bit sums only while
    every leaf contraction is at most 16384 rows (each 256-row chunk adds at
    most 2^24); longer plans keep the 96-column tiles and 64-bit sums."""
    n = 700
    wide = cli(m, n, 4, 0, 0, 4096, 1, split=1)
    narrow = cli(m, n, 2, 0, 0, 4096, 1, split=1)  # FP32 (3 digits): always 96 columns
    assert (wide["tiles"] < narrow["tiles"]) == expect_wide
    assert wide["covered"] == n * (n + 1) // 2 and wide["overlap"] == 0
