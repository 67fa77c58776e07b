"""The integer-only conversion of an exact sum T to T * 2^e in FP64
(csrc/fixconv.h), checked against the host's correctly rounded int64 to
double conversion on random, tie and range-edge cases."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_rounding_matches_the_hosts_conversion(tmp_path):
    src = os.path.join(ROOT, "tests", "fixconv_check.cpp")
    inc = os.path.join(ROOT, "paper_2110_13042_gb300", "csrc")
    exe = str(tmp_path / "fixconv_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    cases, bad, missed = map(int, out)
    assert cases > 2_000_000
    assert bad == 0, f"{bad} results differ from the host's rounding"
    assert missed == 0, f"{missed} normal results were handed to the fallback"
