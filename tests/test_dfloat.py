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


def test_integer_split_equals_the_fp64_split(probe):
    # df_from_double_bits against df_from_double on bit patterns chosen to
    # reach every branch: exponents across the whole range and at the edges
    # of the integer path, remainders at the rounding tie (odd and even
    # kept mantissa), zero remainders, all-ones mantissas (carry into the
    # exponent), both signs, zeros, subnormals, infinities and NaN; and the
    # FP64 bits of |fl32(v)| from df_f64_bits_nonneg
    rng = np.random.default_rng(11)
    pats = []
    exps = list(range(940, 960)) + list(range(1130, 1150)) + list(rng.integers(0, 2048, 200)) + [1023] * 50
    for E in exps:
        for sign in (0, 1):
            for kind in range(6):
                m = int(rng.integers(0, 1 << 52, dtype=np.uint64))
                if kind == 1:
                    m = (m & ~((1 << 29) - 1)) | (1 << 28)  # tie
                elif kind == 2:
                    m = (m & ~((1 << 29) - 1))  # exact in FP32
                elif kind == 3:
                    m = (1 << 52) - 1  # carry into the exponent
                elif kind == 4:
                    m = (m & ~((1 << 29) - 1)) | (1 << 28) | (1 << 29)  # tie, odd kept mantissa
                pats.append((sign << 63) | (int(E) << 52) | m)
    pats += [0, 1 << 63, 0x7ff0000000000000, 0xfff0000000000000, 0x7ff8000000000000, 1, 0x000fffffffffffff,
             0x3ff0000000000000, 0x47efffffe0000000, 0x47efffffefffffff]
    pats += [int(b) for b in rng.integers(0, 1 << 63, 3000, dtype=np.uint64)]
    text = "\n".join(f"{p:x}" for p in pats)
    out = subprocess.run([probe, "split"], input=text + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    bad = [f"{p:x}" for p, line in zip(pats, out) if line.strip() != "1 1"]
    assert len(out) >= len(pats) and not bad, bad[:10]
