"""The FP32 moment rows the on-the-fly kernel forms (shifted_row in
csrc/monomials.cuh: each stencil cell's offset d = (x_j - x_i)/h_i and its
own central moments, binomially shifted) evaluated on the host and compared
with the oracle's exact moment rows, to FP32 rounding, in 1-D, 2-D and 3-D."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_02694_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = None
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(cand, "include")
            break
    if cxx is None or cuda_inc is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("shift") / "shifted_row_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-w", os.path.join(ROOT, "tests", "shifted_row_probe.cpp"),
                    "-I", CSRC, "-I", cuda_inc, "-o", exe], check=True)
    return exe


CASES = [
    ("tri8_p4", lambda: synth.tri_mesh(8, seed=4), 4, 2.0),
    ("tri8_p3", lambda: synth.tri_mesh(8, seed=5), 3, 1.0),
    ("tet3_p3", lambda: synth.tet_mesh(3, seed=15), 3, 2.0 / 3.0),
    ("line16_p5", lambda: synth.periodic_line_mesh(16, jitter=0.2, seed=6), 5, 2.0),
    ("line16_p3", lambda: synth.periodic_line_mesh(16, jitter=0.2, seed=7), 3, 1.0),
]


@pytest.mark.parametrize("name,make,p,ring", CASES, ids=[c[0] for c in CASES])
def test_shifted_rows_match_the_oracle(probe, name, make, p, ring):
    mesh = make()
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, min_rows=int(2 * ring + 1) if mesh.dim == 1 else 0)
    geo, kap, d = prob.geo, prob.kappas, prob.dim
    high = [k for k, kp in enumerate(kap) if sum(kp) >= 2]
    lines, want = [f"{d} {prob.m}"], []
    rng = np.random.default_rng(1)
    for i in rng.choice(prob.N, min(12, prob.N), replace=False):
        i = int(i)
        S = prob.stencils[i]
        A = prob.A(i)
        Ys = O.stencil_coords(geo, S, i, prob.period)
        for t, j in enumerate(S):
            cj = Ys[t].mean(axis=0)
            own = O.moment_row(Ys[t], cj, 1.0, kap)  # absolute units about x_j
            off = (cj - geo.centroid[i]) / geo.h[i]
            vals = list(off) + [1.0 / geo.h[i]] + [own[k] for k in high]
            lines.append(" ".join(repr(float(v)) for v in vals))
            want.append(A[t])
    out = subprocess.run([probe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.strip().split("\n")
    got = np.array([[float(v) for v in line.split()] for line in out])
    want = np.array(want)
    assert got.shape == want.shape
    # FP32 inputs and arithmetic: a few ulps of the row's largest entry
    scale = np.maximum(1.0, np.max(np.abs(want), axis=1))[:, None]
    assert np.max(np.abs(got - want) / scale) <= 2e-6
