"""Build the CPU oracle (plain C, gcc) into ``oracle/_build/liboracle.so``.

Test infrastructure: compiled by ``__graft_entry__.build()`` so the checker
exists on every machine, but never linked into the product library.
``-ffp-contract=off`` keeps every multiply and add separately rounded (no FMA
contraction), so results match bit for bit across x86-64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ata_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")


def library_path() -> str:
    return os.path.join(_OUT_DIR, "liboracle.so")


def build_oracle(verbose: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    out = library_path()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o"]
    # OpenMP only parallelises over output rows; fall back to serial if absent.
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_OUT_DIR)
    os.close(fd)
    try:
        for extra in (["-fopenmp"], []):
            cmd = base + [tmp] + extra + ["-lm"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode == 0:
                os.replace(tmp, out)
                if verbose:
                    print(" ".join(cmd))
                return out
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    finally:
        if os.path.exists(tmp):
            os.unlink(tmp)


if __name__ == "__main__":
    print(build_oracle(verbose=True))
