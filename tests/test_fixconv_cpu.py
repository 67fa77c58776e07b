"""The integer-only conversions of csrc/fixconv.h: an exact sum T to T * 2^e in
FP64, checked against the host's correctly rounded int64 to double conversion
on random, tie and range-edge cases; and FP64 and FP32 values to the fixed point
round(a * 2^sh) (half away from zero), checked against the exact definition
over every shift the digit prep uses, subnormals and signed zeros included."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_rounding_matches_the_hosts_conversion(tmp_path):
    src = os.path.join(ROOT, "tests", "fixconv_check.cpp")
    inc = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc")
    exe = str(tmp_path / "fixconv_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    cases, bad, missed, fcases, fbad = map(int, out)
    assert cases > 2_000_000
    assert bad == 0, f"{bad} results differ from the host's rounding"
    assert missed == 0, f"{missed} normal results were handed to the fallback"
    assert fcases > 20_000_000
    assert fbad == 0, f"{fbad} fixed-point values differ from round(a * 2^sh)"
