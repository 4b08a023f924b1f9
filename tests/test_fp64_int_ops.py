"""The FP64 path divides and takes square roots in 64-bit integer fixed point
(csrc/wcns_f64int.cuh).  IEEE 754 fixes the correctly rounded quotient and
root, so the same source compiled for the host must reproduce the host's
division and sqrt bit for bit, on random operands over the whole exponent
range, exact quotients, squares and their neighbours, zeros, subnormals,
infinities and NaN, with the FP32 seeds moved by up to 64 ulps (the device
seeds come from approximate instructions)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1810_07806_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("f64int") / "host_f64int_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "host_f64int_check.cpp")], check=True)
    return exe


@pytest.mark.parametrize("ulps", [0, 2, 64])
def test_integer_division_and_sqrt_are_ieee(checker, ulps):
    out = subprocess.run([checker, "3000000", str(ulps)], check=True, capture_output=True, text=True).stdout
    f = out.split()
    assert f[f.index("div_mismatches") + 1] == "0", out
    assert f[f.index("sqrt_mismatches") + 1] == "0", out


def test_checker_detects_a_wrong_rounding(tmp_path, checker):
    """Plants a rounding mistake (ties and above-half no longer round up) in a
    copy of the header: the checker must report mismatches."""
    src = open(os.path.join(CSRC, "wcns_f64int.cuh")).read()
    rule = "if ((Q & 1ull) && (r != 0 || (M & 1ull))) ++M;"
    assert src.count(rule) == 2   # division and square root
    planted = src.replace(rule, "")
    d = tmp_path / "inc"
    d.mkdir()
    (d / "wcns_f64int.cuh").write_text(planted)
    exe = str(tmp_path / "bad")
    cxx = shutil.which("g++") or shutil.which("c++")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(d), "-o", exe,
                    os.path.join(HERE, "host_f64int_check.cpp")], check=True)
    out = subprocess.run([exe, "200000", "2"], check=True, capture_output=True, text=True).stdout
    f = out.split()
    assert int(f[f.index("div_mismatches") + 1]) > 0
    assert int(f[f.index("sqrt_mismatches") + 1]) > 0
