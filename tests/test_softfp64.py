"""The integer-pipe binary64 multiplication, addition and power-of-two scaling of the sweep kernels (csrc/softfp64.cuh) give the
correctly rounded IEEE 754 result: the header compiled as host C++ against the host's own arithmetic, bit
for bit, over seeded operands that cover cancellation, ties, exponent-range ends and special values."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("softfp64") / "softfp64_check")
    # -ffp-contract=off: the host reference must round every product and sum on its own
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(HERE, "softfp64_check.cpp"), "-o", exe],
                   check=True)
    return exe


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_integer_binary64_matches_the_host(checker, seed):
    out = subprocess.run([checker, "2000000", str(seed)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mul mismatches 0 add mismatches 0 pow2 mismatches 0" in out.stdout
