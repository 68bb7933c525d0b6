"""The library's FP64 moment rows (csrc/moment_row.cuh: collapsed
Gauss-Legendre product quadrature on the simplex, Sec. 3.2 with the
h-normalisation of Sec. 3.3.2) evaluated on the host and compared with the
oracle's closed-form simplex moments, row by row, in 1-D, 2-D and 3-D."""
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
    exe = str(tmp_path_factory.mktemp("moments") / "moments_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-w", os.path.join(ROOT, "tests", "moments_probe.cpp"),
                    os.path.join(CSRC, "host_mesh.cpp"), "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", cuda_inc, "-o", exe], check=True)
    return exe


CASES = [
    ("tri6_p4_ring2", lambda: synth.tri_mesh(6, seed=4), 4, 2.0, 15),
    ("tri5_p3_open", lambda: synth.tri_mesh(5, periodic=False, seed=12), 3, 1.0, 9),
    ("tet3_p3", lambda: synth.tet_mesh(3, seed=15), 3, 2.0 / 3.0, 15),
    ("line12_p5", lambda: synth.periodic_line_mesh(12, jitter=0.2, seed=6), 5, 2.0, 5),
    ("line12_p3", lambda: synth.periodic_line_mesh(12, jitter=0.2, seed=7), 3, 2.0, 5),
]


@pytest.mark.parametrize("name,make,p,ring,min_rows", CASES, ids=[c[0] for c in CASES])
def test_moment_rows_match_the_oracle(probe, name, make, p, ring, min_rows):
    mesh = make()
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, min_rows=min_rows)
    d = mesh.vertices.shape[1]
    head = f"{d} {mesh.vertices.shape[0]} {mesh.cells.shape[0]} {p} {ring!r} 0.0 {min_rows} 0"
    body = " ".join(repr(float(x)) for x in np.asarray(mesh.period, dtype=np.float64).ravel())
    body += "\n" + " ".join(repr(float(x)) for x in mesh.vertices.ravel())
    body += "\n" + " ".join(str(int(x)) for x in mesh.cells.ravel())
    out = subprocess.run([probe], input=head + "\n" + body + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    assert out[0] == "rows"
    got = np.array([float(v) for v in out[2:]]).reshape(-1, prob.m)
    want = np.concatenate([prob.A(i) for i in range(prob.N)])
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, float(np.max(np.abs(want))))
