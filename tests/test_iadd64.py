"""The binary64 addition on the integer units (paper_1107_4650_gb300/csrc/iadd64.cuh, used by the FP64 step
kernel when int_unit_adds > 0) gives the same bits as the hardware addition: the checker compiles the header
for the host and compares it with the host's IEEE 754 addition and subtraction on several million operand
pairs chosen to reach every path (exponent differences 0-70, cancellation, ties, tiny, huge and special
operands)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1107_4650_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("iadd") / "iadd64_check")
    subprocess.check_call([gxx, "-O2", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "iadd64_check.cpp")])
    return exe


def test_integer_unit_addition_matches_hardware(checker):
    r = subprocess.run([checker, "3000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert "0 mismatches" in r.stdout
