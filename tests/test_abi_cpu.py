"""CPU checks of the C-ABI library: it builds, loads, exports every symbol the
header declares, and its host planner (no GPU needed) produces the plans the
AtA recursion and Strassen's algorithm imply."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ata.h")


@pytest.fixture(scope="session")
def lib():
    from paper_2110_13042_gb300 import build as b
    b.build()
    import paper_2110_13042_gb300 as ata
    return ata


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(ata_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi():
    syms = declared_symbols()
    for s in ("ata_create", "ata_lower", "ata_batched", "ata_destroy", "ata_sync",
              "ata_status_string", "ata_plan_info", "ata_set_config", "ata_version"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ata_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    L = lib.load()
    for s in declared_symbols():
        assert hasattr(L, s)


def test_status_strings(lib):
    for code in range(7):
        assert lib.status_string(code)
    assert lib.status_string(99) == "unknown status"
    assert lib.version() >= 100


def test_no_torch_types_in_header():
    text = open(HEADER).read()
    assert "torch" not in text.lower().replace("(torch", "")
    assert "at::" not in text and "Tensor" not in text


@pytest.mark.skipif("torch" in sys.modules and __import__("torch").cuda.is_available(),
                    reason="only meaningful without a GPU")
def test_create_without_gpu_is_unsupported(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.load().ata_create(ctypes.byref(h), None) == 6


# ------------------------------------------------------------- planner ----

TM, TN = 128, 96   # leaf tile: 128 rows (j) x 96 columns (k)


def lower_tiles(n, tn=None):
    """Tiles of a TM x TN grid (TN x 2 in the FP8 mode) over an n x n matrix
    holding an entry k <= j."""
    tn = tn or TN
    count = 0
    for J in range(-(-n // TM)):
        rows = min(TM, n - J * TM)
        K = 0
        while K * tn < n and K * tn <= J * TM + rows - 1:
            count += 1
            K += 1
    return count


@pytest.mark.parametrize("n", [1, 64, 128, 129, 255, 1000, 4096])
@pytest.mark.parametrize("mode", [1, 2, 4, 5])
def test_plain_plan_is_all_lower_tiles(lib, n, mode):
    h = None
    info = lib.plan_info(300, n, mode, h)
    # depth 0 is only chosen automatically for small n
    if info["depth"] == 0:
        assert info["tiles"] == lower_tiles(n, 2 * TN if mode in (4, 5) else TN)  # one-digit modes: 192
        assert info["panels"] == 1 and info["products"] == 0
        assert info["leaf_madds"] == info["plain_madds"]


@pytest.fixture(scope="session")
def plan_cli(lib):
    src = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan_cli.cpp")
    out = os.path.join(ROOT, "paper_2110_13042_gb300", "_build", "plan_cli")
    plan_cpp = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan.cpp")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.dirname(src), src, plan_cpp, "-o", out],
                   check=True)

    def run(m, n, mode, cutoff, depth, slices=0, strassen_min=1, split_search=1, num_ctas=0, variant=0,
            split_k=0):
        r = subprocess.run([out, str(m), str(n), str(mode), str(cutoff), str(depth), str(slices),
                            str(strassen_min), str(split_search), str(num_ctas), str(variant), "1",
                            str(split_k)],
                           capture_output=True, text=True, check=True)
        return {k: int(v) for k, v in (kv.split("=") for kv in r.stdout.split())}
    return run


@pytest.mark.parametrize("n,cutoff", [(1024, 256), (2048, 512), (1000, 250), (777, 100)])
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_recursion_structure(plan_cli, n, cutoff, depth):
    # With the cost-model split placement off, every split is the aligned
    # middle: panels are the leaves of that column recursion, the split point
    # the largest multiple of 32 not above w/2 (a panel if that is 0).
    P = plan_cli(4096, n, 1, cutoff, depth, split_search=0, split_k=1)  # whole tiles only
    def split(w):
        return (w // 64) * 32

    def leaves(w):
        if w <= cutoff or split(w) == 0:
            return 1
        return leaves(split(w)) + leaves(w - split(w))

    def blocks(w):
        if w <= cutoff or split(w) == 0:
            return 0
        return 1 + blocks(split(w)) + blocks(w - split(w))

    if depth == 0:
        # Strassen depth 0 is plain tiled AtA: one panel, all lower tiles.
        assert P["panels"] == 1 and P["blocks"] == 0 and P["products"] == 0
        assert P["tiles"] == lower_tiles(n)
    else:
        assert P["panels"] == leaves(n)
        assert P["blocks"] == blocks(n)
    # every lower entry is produced exactly once
    assert P["covered"] == n * (n + 1) // 2
    assert P["overlap"] == 0


@pytest.mark.parametrize("m,n,cutoff,depth,smin", [(4096, 1000, 250, 1, 1), (777, 777, 100, 2, 1),
                                                    (8192, 8192, 0, 1, 4096), (513, 3001, 300, 3, 64),
                                                    (64, 16384, 0, 2, 4096)])
def test_split_search_keeps_coverage(plan_cli, m, n, cutoff, depth, smin):
    # Moving Strassen splits off the middle changes the tiling (and possibly
    # the recursion below), never the result: every lower entry is still
    # produced exactly once and no upper one.
    for search in (1, 0):
        P = plan_cli(m, n, 1, cutoff, depth, strassen_min=smin, split_search=search)
        assert P["covered"] == n * (n + 1) // 2
        assert P["overlap"] == 0


@pytest.mark.parametrize("m,n,depth,smin", [(8192, 8192, 1, 4096), (8192, 8192, 0, 4096),
                                            (3000, 5000, 2, 512), (100, 640, 1, 64)])
def test_task_balance_for_persistent_ctas(plan_cli, m, n, depth, smin):
    # The longest-first layout for 152 CTAs keeps every tile (fillers produce
    # nothing) and never loads the busiest CTA more than round-robin does.
    rr = plan_cli(m, n, 1, 0, depth, strassen_min=smin, num_ctas=0)
    bal = plan_cli(m, n, 1, 0, depth, strassen_min=smin, num_ctas=152)
    assert bal["tiles"] == rr["tiles"]
    assert bal["covered"] == n * (n + 1) // 2 and bal["overlap"] == 0
    assert bal["cta_steps_sum"] == rr["cta_steps_sum"]
    assert bal["cta_steps_max"] <= rr["cta_steps_max"]
    # greedy longest-first is within one task of the mean
    assert bal["cta_steps_max"] <= bal["cta_steps_sum"] / 152 + (m + 15) // 16 + 3


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_strassen_products_and_savings(plan_cli, depth):
    n, cutoff = 8192, 2048
    P = plan_cli(8192, n, 1, cutoff, depth, split_k=1)  # whole plain tiles: no chunk products
    assert P["products"] == 7 ** depth * P["blocks"]
    # Each Strassen level replaces 8 block products by 7 on the off-diagonal
    # blocks (Section 3.2): leaf work / classical work on those blocks = (7/8)^d.
    ratio = P["strassen_leaf_madds"] / P["strassen_plain_madds"]
    assert abs(ratio - (7 / 8) ** depth) < 1e-9


def test_combine_terms_match_strassen_counts(plan_cli):
    # depth 1: C11 and C22 have 4 terms, C12 and C21 have 2: 12 result terms
    # per block (the 8 result additions of Section 3.2 plus one term per quadrant).
    P = plan_cli(8192, 4096, 1, 2048, 1, split_search=0, split_k=1)
    assert P["blocks"] == 1
    assert P["cterms"] == 12
    P2 = plan_cli(8192, 4096, 1, 2048, 2, split_search=0, split_k=1)
    assert P2["cterms"] == 144


def test_invalid_parameters_rejected(plan_cli):
    with pytest.raises(subprocess.CalledProcessError):
        plan_cli(10, 10, 3, 0, 0)      # unknown mode
    with pytest.raises(subprocess.CalledProcessError):
        plan_cli(10, 10, 1, 0, 0, 9)   # too many digits


@pytest.mark.parametrize("m,n,depth", [(1056, 2048, 1), (1000, 1024, 1), (531, 777, 2), (4099, 2048, 2)])
def test_fp8_plan(plan_cli, m, n, depth):
    """FP8 mode: the same tiles (both one-digit modes use 128 x 192 tiles at
    these contraction lengths) and Strassen products as one BF16 digit, one
    byte per plane element (smaller workspace), and Strassen quadrants read
    from the planes of A only where their row offset falls on a 32-row FP8 K
    step (a 16-row offset that a BF16 plane could serve is not enough)."""
    # (middle splits: the cost model that places Strassen splits counts tiles)
    r8 = plan_cli(m, n, 5, n // 4, depth, split_search=0, split_k=1)
    rb = plan_cli(m, n, 4, n // 4, depth, split_search=0, split_k=1)
    assert r8["slices"] == 1
    for k in ("tiles", "products", "covered", "overlap", "cterms"):
        assert r8[k] == rb[k], k
    assert r8["workspace"] < rb["workspace"]
    assert r8["reused"] <= rb["reused"]
    if (m + 1) // 2 % 32 == 16:
        assert r8["reused"] < rb["reused"]


@pytest.mark.parametrize("mode", [1, 2, 0, 5])
@pytest.mark.parametrize("m,n,depth", [(1000, 1024, 1), (531, 777, 2), (4099, 2048, 2), (300, 900, 3)])
def test_prep_and_combine_tile_maps(plan_cli, mode, m, n, depth):
    """Operands of one family and shape share an interleaved tile range: the
    flat range, mapped the way the prep kernels map it, produces every tile
    of every operand exactly once; combine tiles (64 x 32) have consistent
    prefix bases."""
    r = plan_cli(m, n, mode, max(1, n // 4), depth)
    assert r["prep_map_ok"] == 1 and r["comb_map_ok"] == 1
    assert r["prep_groups"] <= r["ops"]
    if r["products"] > 0:
        assert r["prep_groups"] < r["ops"]  # Strassen operand sums were grouped


@pytest.fixture(scope="session")
def plan_cli_sanitized(lib, tmp_path_factory):
    """The planner inspector built with AddressSanitizer and UBSan (skipped
    where the compiler has no sanitizer runtime)."""
    src = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan_cli.cpp")
    plan_cpp = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan.cpp")
    out = str(tmp_path_factory.mktemp("san") / "plan_cli_san")
    r = subprocess.run(["g++", "-O1", "-g", "-std=c++17", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        "-I", os.path.dirname(src), src, plan_cpp, "-o", out], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no sanitizer runtime: " + r.stderr[:200])
    return out


SAN_SHAPES = [(1, 1), (1, 77), (129, 1), (2, 2), (37, 129), (300, 257), (531, 600), (97, 513), (600, 96)]


@pytest.mark.parametrize("m,n", SAN_SHAPES)
def test_planner_under_sanitizers(plan_cli_sanitized, m, n):
    """Every mode, Strassen depth and cutoff style on odd and degenerate
    shapes: no out-of-bounds access or undefined behaviour in the planner,
    every lower entry produced once, and consistent prep and combine tile
    maps."""
    for mode in (0, 1, 2, 5):  # (the one-digit BF16 mode plans like FP32)
        for depth in (0, 1, 3):
            for cutoff, smin in ((0, 4096), (max(1, n // 4), 2), (16, 1)):
                r = subprocess.run([plan_cli_sanitized, str(m), str(n), str(mode), str(cutoff), str(depth), "0",
                                    str(smin), "1", "152"], capture_output=True, text=True)
                assert r.returncode == 0, (mode, depth, cutoff, r.stderr[:500])
                kv = dict(x.split("=") for x in r.stdout.split())
                assert kv["overlap"] == "0" and kv["prep_map_ok"] == "1" and kv["comb_map_ok"] == "1"
                assert int(kv["covered"]) == n * (n + 1) // 2


@pytest.mark.parametrize("m,n,mode", [(8192, 8192, 1), (300, 5000, 2), (1000, 4096, 5), (64, 129, 1)])
def test_plan_blocks_describe_the_recursion(lib, m, n, mode):
    """ata_plan_blocks: one record per off-diagonal block of the plan
    (ata_plan_info's block count), each strictly below the diagonal, and
    together with the diagonal panels they cover the lower triangle once."""
    info = lib.plan_info(m, n, mode)
    blocks = lib.plan_blocks(m, n, mode)
    assert len(blocks) == info["blocks"]
    covered = 0
    for r0, p, c0, q, d in blocks:
        assert p > 0 and q > 0 and r0 >= c0 + q and r0 + p <= n and 0 <= d <= info["depth"]
        covered += p * q
    # the rest of the lower triangle is diagonal panels (w (w + 1) / 2 each)
    assert covered < n * (n + 1) // 2
    assert any(d > 0 for *_, d in blocks) == (info["products"] > 0)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("m,n,mode,cutoff,depth,smin", [
    (300, 257, 1, 32, 1, 2), (1000, 1000, 1, 0, 2, 64), (777, 901, 2, 64, 3, 64),
    (2000, 3001, 1, 0, 8, 64), (129, 515, 0, 0, 8, 16), (513, 700, 5, 100, 2, 2)])
def test_variants_and_recursion_to_cutoff_cover_the_triangle(plan_cli, variant, m, n, mode, cutoff, depth, smin):
    """Strassen's and Winograd's tables, and a depth budget large enough that
    only the size cutoff (strassen_min) stops the recursion: every lower
    entry produced exactly once, prep and combine maps consistent, and every
    Strassen block split while both its sides reach strassen_min."""
    r = plan_cli(m, n, mode, cutoff, depth, strassen_min=smin, variant=variant)
    assert r["covered"] == n * (n + 1) // 2 and r["overlap"] == 0
    assert r["prep_map_ok"] == 1 and r["comb_map_ok"] == 1
    assert r["products"] > 0


def test_winograd_products_and_terms(plan_cli):
    """Same product count per level (7); Winograd's result sums have more
    terms (2 + 4 + 4 + 4 = 14 per level against Strassen's 4 + 2 + 2 + 4 = 12)."""
    s = plan_cli(1024, 1024, 1, 0, 1, strassen_min=64, split_search=0, variant=0)
    w = plan_cli(1024, 1024, 1, 0, 1, strassen_min=64, split_search=0, variant=1)
    assert s["products"] == w["products"] == 7 * s["blocks"]
    assert s["cterms"] * 14 == w["cterms"] * 12


def test_recursion_to_cutoff_depth(plan_cli):
    """Depth budget 8 with strassen_min 256 on a 4096-column problem with the
    default cutoff (1024): the top block (2048 wide) splits while both sides
    are >= 256: 2048 -> 1024 -> 512 -> 256 -> 128, four levels."""
    r = plan_cli(4096, 4096, 1, 0, 8, strassen_min=256, split_search=0)
    assert r["depth"] == 8
    assert r["products"] >= 7 ** 4
