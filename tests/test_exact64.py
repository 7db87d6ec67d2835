"""The integer binary64 products and roundings of the thermal-mass kernel
(exact64.cuh) against the host's IEEE double arithmetic, on random operands
of every magnitude the mass sums meet (compiled as plain C++, no GPU)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_binary64_matches_ieee_double(tmp_path):
    exe = tmp_path / "exact64_check"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                        "-I", os.path.join(ROOT, "paper_1912_04457_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "exact64_check.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe), "3000000"], capture_output=True, text=True, timeout=300)
    cases, bad = map(int, r.stdout.split())
    assert cases > 9_000_000
    assert bad == 0 and r.returncode == 0
