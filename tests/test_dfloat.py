"""The library's double-float arithmetic (csrc/dfloat.cuh: TwoSum, FastTwoSum,
FMA-based TwoProd, the accurate addition and the product) compiled as host
C++ with IEEE single-precision stand-ins for the round-to-nearest
intrinsics, against exact rational arithmetic: sums and products of random
pairs, including cancelling sums, to a few 2^-48 relative, and normalised
results (|lo| <= ulp(hi)/2)."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_02694_gb300", "csrc")

STAND_IN = r"""
#pragma once
#include <cmath>
#define __host__
#define __device__
#define __forceinline__ inline
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("needs a C++ compiler")
    d = tmp_path_factory.mktemp("dfloat")
    (d / "cuda_runtime.h").write_text(STAND_IN)
    exe = str(d / "dfloat_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-ffp-contract=off", "-fno-fast-math", "-I", str(d), "-I", CSRC,
                    os.path.join(ROOT, "tests", "dfloat_probe.cpp"), "-o", exe], check=True)
    return exe


def pair(rng, scale):
    v = rng.uniform(-1, 1) * scale
    hi = np.float32(v)
    lo = np.float32(v - float(hi))
    return float(hi), float(lo)


def exact(p):
    return Fraction(p[0]) + Fraction(p[1])


def test_double_float_sums_and_products(probe):
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(400):
        a = pair(rng, 10.0 ** rng.uniform(-3, 3))
        b = pair(rng, 10.0 ** rng.uniform(-3, 3))
        cases.append(("add", a, b))
        cases.append(("mul", a, b))
        # nearly cancelling sums: b close to -a
        c = pair(rng, 1e-6 * abs(a[0]) + 1e-30)
        neg = (-a[0], float(np.float32(-a[1] + c[0])))
        cases.append(("add", a, neg))
    text = "\n".join(f"{op} {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for op, x, y in cases)
    out = subprocess.run([probe], input=text + "\n", capture_output=True, text=True, check=True).stdout.split("\n")
    worst = 0.0
    for (op, x, y), line in zip(cases, out):
        hi, lo = (float.fromhex(t) for t in line.split())
        want = exact(x) + exact(y) if op == "add" else exact(x) * exact(y)
        got = Fraction(hi) + Fraction(lo)
        scale = abs(want)  # relative to the result: the accurate sum survives cancellation
        if scale == 0:
            assert got == 0
            continue
        err = float(abs(got - want) / scale)
        worst = max(worst, err)
        # normalised: hi is the float nearest hi + lo
        assert float(np.float32(hi + lo)) == hi or lo == 0.0
    assert worst <= 8 * 2.0 ** -48, worst


def test_exact_cancellation_and_zero(probe):
    cases = [("add", (1.5, 2.0 ** -30), (-1.5, -(2.0 ** -30))), ("mul", (0.0, 0.0), (3.0, 1e-9)),
             ("add", (0.0, 0.0), (0.0, 0.0))]
    text = "\n".join(f"{op} {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for op, x, y in cases)
    out = subprocess.run([probe], input=text + "\n", capture_output=True, text=True, check=True).stdout.split("\n")
    for line in out[:3]:
        hi, lo = (float.fromhex(t) for t in line.split())
        assert hi == 0.0 and lo == 0.0
