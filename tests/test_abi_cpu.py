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


def lower_tiles(n):
    """Tiles of a TM x TN grid over an n x n matrix holding an entry k <= j."""
    count = 0
    for J in range(-(-n // TM)):
        rows = min(TM, n - J * TM)
        K = 0
        while K * TN < n and K * TN <= J * TM + rows - 1:
            count += 1
            K += 1
    return count


@pytest.mark.parametrize("n", [1, 64, 128, 129, 255, 1000, 4096])
@pytest.mark.parametrize("mode", [1, 2, 4])
def test_plain_plan_is_all_lower_tiles(lib, n, mode):
    h = None
    info = lib.plan_info(300, n, mode, h)
    # depth 0 is only chosen automatically for small n
    if info["depth"] == 0:
        assert info["tiles"] == lower_tiles(n)
        assert info["panels"] == 1 and info["products"] == 0
        assert info["leaf_madds"] == info["plain_madds"]


@pytest.fixture(scope="session")
def plan_cli(lib):
    src = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan_cli.cpp")
    out = os.path.join(ROOT, "paper_2110_13042_gb300", "_build", "plan_cli")
    plan_cpp = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc", "plan.cpp")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.dirname(src), src, plan_cpp, "-o", out],
                   check=True)

    def run(m, n, mode, cutoff, depth, slices=0):
        r = subprocess.run([out, str(m), str(n), str(mode), str(cutoff), str(depth), str(slices)],
                           capture_output=True, text=True, check=True)
        return {k: int(v) for k, v in (kv.split("=") for kv in r.stdout.split())}
    return run


@pytest.mark.parametrize("n,cutoff", [(1024, 256), (2048, 512), (1000, 250), (777, 100)])
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_recursion_structure(plan_cli, n, cutoff, depth):
    P = plan_cli(4096, n, 1, cutoff, depth)
    # Panels: the leaves of the column recursion; the split point is the
    # largest multiple of 32 not above w/2 (a panel if that is 0).
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


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_strassen_products_and_savings(plan_cli, depth):
    n, cutoff = 8192, 2048
    P = plan_cli(8192, n, 1, cutoff, depth)
    assert P["products"] == 7 ** depth * P["blocks"]
    # Each Strassen level replaces 8 block products by 7 on the off-diagonal
    # blocks (Section 3.2): leaf work / classical work on those blocks = (7/8)^d.
    ratio = P["strassen_leaf_madds"] / P["strassen_plain_madds"]
    assert abs(ratio - (7 / 8) ** depth) < 1e-9


def test_combine_terms_match_strassen_counts(plan_cli):
    # depth 1: C11 and C22 have 4 terms, C12 and C21 have 2: 12 result terms
    # per block (the 8 result additions of Section 3.2 plus one term per quadrant).
    P = plan_cli(8192, 4096, 1, 2048, 1)
    assert P["blocks"] == 1
    assert P["cterms"] == 12
    P2 = plan_cli(8192, 4096, 1, 2048, 2)
    assert P2["cterms"] == 144


def test_invalid_parameters_rejected(plan_cli):
    with pytest.raises(subprocess.CalledProcessError):
        plan_cli(10, 10, 3, 0, 0)      # unknown mode
    with pytest.raises(subprocess.CalledProcessError):
        plan_cli(10, 10, 1, 0, 0, 9)   # too many digits
