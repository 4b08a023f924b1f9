"""The FP32 path converts between FP64 and FP32 by integer arithmetic on the
IEEE-754 encodings (csrc/wcns_cvt.cuh).  IEEE 754 fixes the conversions:
compiled for the host, the header must reproduce the host's float(x)
(round to nearest even) and double(x) bit for bit, apart from the stated
flush of FP32 subnormals to signed zeros, on random encodings, exact ties,
the FLT_MIN and FLT_MAX edges, infinities and NaN."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1810_07806_gb300", "csrc")


def _build(inc, exe):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, "-o", exe,
                    os.path.join(HERE, "host_cvt_check.cpp")], check=True)


def _counts(exe, n):
    out = subprocess.run([exe, str(n)], check=True, capture_output=True, text=True).stdout.split()
    return {k: int(out[out.index(k) + 1]) for k in
            ("f64_to_f32_mismatches", "f32_to_f64_mismatches", "zero_mismatches")}


def test_integer_conversions_are_ieee(tmp_path):
    exe = str(tmp_path / "cvt")
    _build(CSRC, exe)
    assert _counts(exe, 4000000) == {"f64_to_f32_mismatches": 0, "f32_to_f64_mismatches": 0,
                                     "zero_mismatches": 0}


def test_checker_detects_round_half_up(tmp_path):
    """A planted mistake (ties rounded up instead of to even) is caught."""
    src = open(os.path.join(CSRC, "wcns_cvt.cuh")).read()
    rule = "(rest == 0x10000000u && (mant & 1u))"
    assert src.count(rule) == 1
    d = tmp_path / "inc"
    d.mkdir()
    (d / "wcns_cvt.cuh").write_text(src.replace(rule, "(rest == 0x10000000u)"))
    exe = str(tmp_path / "bad")
    _build(str(d), exe)
    assert _counts(exe, 200000)["f64_to_f32_mismatches"] > 0
